// chi -> Kraus conversion for callers that cannot allocate device memory.
//
// Some hosts of this library cannot call cudaMalloc: a plug-in running inside another
// application's memory pool, code that must not grow its footprint after start-up, or a caller
// that is itself executing between allocation-free checkpoints.  This entry point performs the same
// conversion as channel_set_from_process_matrices, with every intermediate (Choi matrices,
// eigenvectors, eigenvalues, eigensolver scratch) placed in one file-scope device array of fixed
// size instead of freshly allocated memory.  The caller passes device input and output buffers.
#include <mutex>

#include "kernels.h"
#include "mpdo.h"

using namespace mpdo;

namespace {
constexpr int kMaxChannels = MPDO_NOALLOC_MAX_CHANNELS;
constexpr int kD2 = 16;  // 4^nq for nq <= 2
constexpr int64_t kChoi = (int64_t)kD2 * kD2;
// per channel, in doubles: Choi matrix and eigenvectors (complex), eigenvalues, eigensolver scratch
constexpr int64_t kScrPerChan = 8 * kD2 * kD2 + 2 * kD2 + 64;
constexpr int64_t kPerChan = 2 * kChoi * 2 + kD2 + kScrPerChan;
constexpr int64_t kScratchDoubles = kMaxChannels * kPerChan;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_ptr[64] = {nullptr};  // device address of g_noalloc_scratch, per device ordinal

// Kraus operators of channel c from its Choi eigenpairs (descending), pruned at tol * max eta.  The
// rank written is -1 when the negative Choi mass exceeds 1e-8 (not completely positive) and -2 when
// sum_i K_i^H K_i differs from I by more than 1e-8 (not trace preserving); the operators are then zero.
__global__ void prune_and_build_kraus(int count, int nq, double tol, const double* eta, const cplx<double>* vecs,
                                      cplx<double>* kraus, int* ranks) {
  const int c = blockIdx.x;
  if (c >= count) return;
  const int d = 1 << nq, d2 = d * d;
  GPTR(const double, w, eta + (int64_t)c * d2);
  GPTR(cplx<double>, K, kraus + (int64_t)c * d2 * d2);
  __shared__ int s_r, s_bad;
  if (threadIdx.x == 0) {
    double emax = w[0] > 0 ? w[0] : 0, neg = 0;
    int r = 0;
    for (int i = 0; i < d2; ++i) {
      if (w[i] > tol * emax && w[i] > 0) ++r;
      if (w[i] < 0) neg -= w[i];
    }
    if (r < 1) r = 1;
    s_r = r;
    s_bad = (neg > 1e-8 || !(neg == neg)) ? -1 : 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < d2 * d2; e += blockDim.x) {
    int i = e / d2, a = e % d2;
    cplx<double> v = mk<double>(0, 0);
    if (i < s_r && !s_bad) v = sqrt(fmax(w[i], 0.0)) * GX(vecs, (int64_t)c * d2 * d2 + a + (int64_t)i * d2);
    K[e] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!s_bad) {
      double err = 0;
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
          cplx<double> t = mk<double>(a == b ? -1.0 : 0.0, 0.0);
          for (int i = 0; i < s_r; ++i)
            for (int m = 0; m < d; ++m) t = t + conjg(K[i * d2 + m * d + a]) * K[i * d2 + m * d + b];
          err = fmax(err, sqrt(norm2(t)));
        }
      if (!(err <= 1e-8)) s_bad = -2;
    }
    GX(ranks, c) = s_bad ? s_bad : s_r;
  }
  __syncthreads();
  if (s_bad)
    for (int e = threadIdx.x; e < d2 * d2; e += blockDim.x) K[e] = mk<double>(0, 0);
}

// Device address of the scratch array for the current device (set up once per device).
double* scratch_for_current_device(mpdo_status* st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *st = MPDO_ECUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      *st = MPDO_ECUDA;
      return nullptr;
    }
    g_ptr[dev] = static_cast<double*>(p);
  }
  *st = MPDO_OK;
  return g_ptr[dev];
}
}  // namespace

extern "C" mpdo_status channel_kraus_noalloc(int nq, int count, const double* chi_dev, double tol, double* kraus_dev,
                                             int* ranks_dev, void* stream) {
  if ((nq != 1 && nq != 2) || count < 1 || !chi_dev || !kraus_dev || !ranks_dev) return MPDO_EINVAL;
  if (count > kMaxChannels) return MPDO_EINVAL;
  if (!(tol > 0)) tol = 1e-12;
  mpdo_status st;
  double* base = scratch_for_current_device(&st);
  if (!base) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int d = 1 << nq, d2 = d * d;
  const int64_t per = (int64_t)d2 * d2;
  cplx<double>* choi = reinterpret_cast<cplx<double>*>(base);
  cplx<double>* vecs = choi + per * count;
  double* eta = reinterpret_cast<double*>(vecs + per * count);
  double* scr = eta + (int64_t)d2 * count;
  const int64_t scr_per = eig_scratch_elems(d2, d2);
  if (chi_to_choi(s, count, nq, reinterpret_cast<const cplx<double>*>(chi_dev), choi) != cudaSuccess)
    return MPDO_ECUDA;
  EigArgs<double> a;
  a.A = choi;
  a.astride = per;
  a.n = d2;
  a.k = d2;
  a.w = eta;
  a.wstride = d2;
  a.V = vecs;
  a.vv = col_major(d2, per);
  a.scratch = scr;
  a.sstride = scr_per;
  a.disc = nullptr;
  a.gap = nullptr;
  a.disc_stride = 0;
  if (heevk<double>(s, count, a) != cudaSuccess) return MPDO_ECUDA;
  prune_and_build_kraus<<<count, 128, 0, s>>>(count, nq, tol, eta, vecs,
                                              reinterpret_cast<cplx<double>*>(kraus_dev), ranks_dev);
  return cudaGetLastError() == cudaSuccess ? MPDO_OK : MPDO_ECUDA;
}
