// Internal launch interface of the sm_103a kernels (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cplx.cuh"

namespace mpdo {

template <typename R>
struct GemmArgs {
  int M, N, K;
  cplx<R> alpha, beta;  // beta == 0: C is written without being read
  const cplx<R>* A;
  View va;  // M x K
  const cplx<R>* B;
  View vb;  // K x N
  cplx<R>* C;
  View vc;  // M x N; vc.conj stores conj(result)
  int herm = 0;  // M == N and the result is Hermitian: only tiles on or below the diagonal are computed
  int allow_tc = 0;  // complex64 only: route to the tensor-core GEMM when the shape qualifies
  // optional workspace for split-K partial products (long reductions with few output tiles);
  // nullptr disables splitting
  cplx<R>* ws = nullptr;
  int64_t ws_elems = 0;
  int* status = nullptr;  // nullable: kStatusTimeout is or-ed in when a bounded wait runs out
  // complex64 only: workspaces for the tensor-core GEMM's split operand planes (floats, all batch
  // items); nullptr keeps every product on the CUDA cores
  float* tc_a = nullptr;
  float* tc_b = nullptr;
  int64_t tc_a_cap = 0, tc_b_cap = 0;
};

// bits of a handle's device status word (read and cleared by the host at synchronising calls)
constexpr int kStatusNoConv = 1;   // an eigensolver produced non-finite or collapsed eigenpairs
constexpr int kStatusTimeout = 2;  // a bounded wait inside a kernel ran out
template <typename R>
cudaError_t gemm(cudaStream_t s, int batch, const GemmArgs<R>& g);

// tensor-core (tcgen05, split TF32, compensated folding) complex64 GEMM for products with M >= 128,
// N >= 64, K >= 16 whose split planes fit the workspaces; plane sizes in floats per batch item
bool tc_gemm_applicable(const GemmArgs<float>& g, int batch);
cudaError_t tc_gemm(cudaStream_t s, int batch, const GemmArgs<float>& g);
int64_t tc_plane_floats_a(int M, int K);
int64_t tc_plane_floats_b(int N, int K);

template <typename R>
struct QrArgs {
  int m, n;
  const cplx<R>* in;
  View vin;
  cplx<R>* W;  // column-major m x n work matrix; R ends in its leading x rows
  int64_t wstride;
  cplx<R>* Qw;  // column-major m x x
  int64_t qstride;
  cplx<R>* qout;  // optional copy of Q through vq
  View vq;
};
template <typename R>
cudaError_t qr(cudaStream_t s, int batch, const QrArgs<R>& g);

template <typename R>
struct EigArgs {
  cplx<R>* A;  // column-major n x n Hermitian, overwritten
  int64_t astride;
  int n, k;
  R* w;  // top-k eigenvalues, descending (nullable)
  int64_t wstride;
  cplx<R>* V;  // n x k eigenvectors through vv
  View vv;
  R* scratch;
  int64_t sstride;  // >= eig_scratch_elems(n, k)
  double* disc;     // nullable: += (trace - sum of kept) / trace
  double* gap;      // nullable: min((w_{k-1} - w_k) / w_0)
  int64_t disc_stride;
  int* status = nullptr;  // nullable: kStatusNoConv is or-ed in on a non-finite or collapsed result
};
template <typename R>
cudaError_t heevk(cudaStream_t s, int batch, const EigArgs<R>& g);
int64_t eig_scratch_elems(int n, int k);

// ---- MPDO kernels (mpdo_kernels.cu)
// Choi matrix of each chi (Sec. III): L[a, b] = sum_mn chi_mn vec(s_m)[a] conj(vec(s_n)[b]),
// chi row-major (d2 x d2 complex), L column-major.
cudaError_t chi_to_choi(cudaStream_t s, int count, int nq, const cplx<double>* chi, cplx<double>* choi);
// K_i = sqrt(eta_i) unvec(psi_i) for i < r (eigenvectors column-major d2 x d2), padded with zeros to rmax.
cudaError_t choi_to_kraus(cudaStream_t s, int count, int nq, int rmax, const int* r_dev, const double* eta,
                          const cplx<double>* vecs, cplx<double>* kraus);
// max |sum_i K_i^H K_i - I| per channel
cudaError_t kraus_tp_error(cudaStream_t s, int count, int nq, int rmax, const cplx<double>* kraus, double* err);

template <typename R>
struct FuseArgs {
  int nq, rk;                    // rk = padded Kraus count
  cplx<double> U[64];            // used when Udev == nullptr (d x d, d <= 8)
  const cplx<double>* Udev;      // per instance d x d (row-major), stride d*d
  const cplx<double>* kraus;     // channel set: [chan][rk][d][d]
  int64_t chan_stride;
  const int* chan_idx;           // per instance channel index (nullable: channel 0)
  cplx<R>* Khat;                 // out per instance [rk][d][d]
  cplx<R>* Rt;                   // out per instance (2q only): 64 entries, see build_T
};
template <typename R>
cudaError_t fuse_gate(cudaStream_t s, int batch, const FuseArgs<R>& a);

// Keeps each chain's site near unit scale by an exact power of two, accumulated in exp2 (per chain,
// the stored state times 2^exp2 is the represented one); the site's entries are the first `elems`.
template <typename R>
cudaError_t renorm_sites(cudaStream_t s, int batch, int64_t elems, cplx<R>* site, int64_t stride, int* exp2);

// Three-qubit gate on a merged three-site tensor (one thread per output element):
//   T[x][p1'][p2'][n2][k][n3][p3'][r] = sum_{p1 p2 p3} Khat_k[(p1' p2' p3'), (p1 p2 p3)] T0[x][p1][p2][n2][p3][n3][r]
// Khat per instance [rk][8][8]; T0 and T the instance strides t0stride, tstride.
template <typename R>
cudaError_t gate3(cudaStream_t s, int batch, int X, int dn2, int dn3, int dr, int rk, const cplx<R>* Khat,
                  const cplx<R>* T0, int64_t t0stride, cplx<R>* T, int64_t tstride);

// T[c][a][c'][b] = sum_{p2, q2} Rt[(a,b),(p1,p2),(q1,q2)] E[(bb,p2),(bb',q2)], c = p1*dm + bb
template <typename R>
cudaError_t build_T(cudaStream_t s, int batch, int dm, const cplx<R>* Rt, const cplx<R>* E, int64_t estride,
                    cplx<R>* T, int64_t tstride);
// Y[((b'*2 + p2')*rk + k)][(bb*2 + p2)] = sum_{p1', p1} Khat_k[(p1' p2'), (p1 p2)] H[(b'*2 + p1')][(p1*dm + bb)]
template <typename R>
cudaError_t build_Y(cudaStream_t s, int batch, int kchi, int dm, int rk, const cplx<R>* Khat, const cplx<R>* H,
                    int64_t hstride, cplx<R>* Y, int64_t ystride);

// A new Kraus leg without forming the extended tensor (one-qubit gates, and the Kraus-first
// two-qubit update): the Kraus-leg Gram of X = (Khat (x) I) A from the Gram H of A over its bond
// indices, G[(k, n), (k', n')] = sum_{p, p''} (Khat_k^H Khat_k')[p, p''] H[(p, n), (p'', n')]
// (G column-major rk dn square, H row-major d dn square, d = 2 or 4 the gate dimension), and the kept
// directions V (column-major, ld vld) folded into the gate, W[(p', nu), (p, n)] = sum_k Khat_k[p', p]
// V[(k, n), nu] (row-major d kap x d dn).
template <typename R>
cudaError_t kraus_gram(cudaStream_t s, int batch, int d, int rk, int dn, const cplx<R>* Khat, const cplx<R>* H,
                       int64_t hstride, cplx<R>* G, int64_t gstride);
template <typename R>
cudaError_t kraus_fold(cudaStream_t s, int batch, int d, int rk, int dn, int kap, const cplx<R>* Khat,
                       const cplx<R>* V, int64_t vstride, int vld, cplx<R>* W, int64_t wstride);

// column scaling V[:, j] *= f[j] of a column-major n x n FP64 matrix
cudaError_t scale_cols(cudaStream_t s, int n, cplx<double>* V, const double* f);

// out(view) = in(view) for an M x N block, optional per-row scale by a diagonal d[row % dmod]
template <typename R>
cudaError_t copy_view(cudaStream_t s, int batch, int M, int N, const cplx<R>* in, View vin, cplx<R>* out, View vout);
// x[z][i] *= sgn for the rows i where ((i / div) % 2) == 1 (Z on the physical index)
template <typename R>
cudaError_t scale_odd(cudaStream_t s, int batch, int64_t len, int64_t div, R sgn, cplx<R>* x, int64_t stride);
// precision conversion
template <typename A, typename B>
cudaError_t convert(cudaStream_t s, int64_t count, const cplx<A>* in, cplx<B>* out);
// set the |0> product site: A[0,0,0,0] = 1, A[0,1,0,0] = 0 in `batch` slots
template <typename R>
cudaError_t init_zero_sites(cudaStream_t s, int count, cplx<R>* base, int64_t stride);
// sum_i conj(a[i]) b[i] per batch into out (FP64)
template <typename R>
cudaError_t dot_batch(cudaStream_t s, int batch, int64_t len, const cplx<R>* a, int64_t astride, const cplx<R>* b,
                      int64_t bstride, cplx<double>* out);
template <typename R>
cudaError_t fill(cudaStream_t s, int64_t count, cplx<R>* x, cplx<R> v);
// complete a column-major Hermitian n x n matrix from its lower triangle: A[i, j] = conj(A[j, i]), i < j
template <typename R>
cudaError_t herm_fill_upper(cudaStream_t s, int batch, int n, cplx<R>* A, int64_t stride);
// discarded-weight accumulators [batch][3] = (0, 0, +inf-like gap)
cudaError_t init_discarded(cudaStream_t s, int batch, double* d);
// generic permutation of a dense row-major tensor with up to 6 dims (batched)
template <typename R>
cudaError_t permute(cudaStream_t s, int batch, int nd, const int* dims, const int* perm, const cplx<R>* in,
                    int64_t istride, cplx<R>* out, int64_t ostride);

}  // namespace mpdo
