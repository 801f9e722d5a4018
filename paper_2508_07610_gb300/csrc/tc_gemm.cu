// Complex64 GEMM on the 5th-generation tensor cores (tcgen05, TF32 inputs, FP32 accumulators in
// tensor memory) for the largest contraction of the two-site update.
//
// Each complex product is four real products (Re = ArBr - AiBi, Im = ArBi + AiBr) and each real
// product is taken in three TF32 pieces (hi*hi + hi*lo + lo*hi, hi = x rounded to TF32, lo = the
// rest rounded to TF32), which keeps FP32-level accuracy.  A CTA of 128 threads owns a 128 x 128
// output tile: the real and imaginary accumulators occupy 2 x 128 TMEM columns.  Operands are read
// through the same strided views as the CUDA-core GEMM, split, and written to shared memory in the
// K-major no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix); one thread issues the
// twelve tcgen05.mma per k-step of 8 and commits them to an mbarrier per stage (two stages).  Every
// mbarrier wait is bounded: on timeout the kernel records an error flag and skips its output.
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels.h"
#include "mpdo.h"

namespace mpdo {

namespace {
constexpr int TM = 128, TN = 128, TK = 8, NTH = 128, STAGES = 2;
constexpr int TILE_BYTES = TM * TK * 4;          // one 128 x 8 TF32 operand tile: 4 KB
constexpr int STAGE_BYTES = 8 * TILE_BYTES;      // A: re hi/lo, im hi/lo; B: the same
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 256;
constexpr int TMEM_COLS = 2 * TN;
constexpr long long kWaitLimit = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm volatile("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// byte offset of element (row, k) of a 128 x 8 K-major tile: core matrices of 8 rows x 16 bytes,
// the two k-halves 128 bytes apart (leading-dimension offset), row groups 256 bytes apart (stride)
__device__ __forceinline__ int tile_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 256;
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, no swizzle
}
// kind::tf32 instruction descriptor: D F32, A/B TF32, both K-major, M = 128, N = TN
__device__ __forceinline__ uint32_t instr_desc(int negate_a) {
  uint32_t d = 0;
  d |= 1u << 4;                     // D format F32
  d |= 2u << 7;                     // A format TF32
  d |= 2u << 10;                    // B format TF32
  d |= (uint32_t)negate_a << 13;    // negate A
  d |= (uint32_t)(TN >> 3) << 17;   // N / 8
  d |= (uint32_t)(TM >> 4) << 24;   // M / 16
  return d;
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(NTH) tc_gemm_kernel(GemmArgs<float> g, int* err_flag) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* tiles = smem;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + STAGES * STAGE_BYTES + 64);
  int* s_fail = reinterpret_cast<int*>(smem + STAGES * STAGE_BYTES + 128);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int z = blockIdx.z;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const cplx<float>* A = g.A + view_batch(g.va, z);
  const cplx<float>* B = g.B + view_batch(g.vb, z);
  cplx<float>* C = g.C + view_batch(g.vc, z);

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])) : "memory");
    *s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int KT = (g.K + TK - 1) / TK;
  uint32_t phase[STAGES] = {0, 0};
  for (int kt = 0; kt < KT; ++kt) {
    const int s = kt % STAGES;
    unsigned char* st = tiles + s * STAGE_BYTES;
    if (kt >= STAGES) {  // the MMAs that read this stage two k-steps ago must be done
      if (!mbar_wait(smem_u32(&mbar[s]), phase[s])) *s_fail = 1;
      phase[s] ^= 1;
    }
    // stage the k-step: each thread splits 8 A elements and 8 B elements
    const int k0 = kt * TK;
    for (int e = tid; e < TM * TK; e += NTH) {
      const int row = e / TK, k = e % TK;
      const int i = m0 + row, kk = k0 + k;
      cplx<float> v = mk<float>(0.f, 0.f);
      if (i < g.M && kk < g.K) {
        v = A[view_row(g.va, i) + view_col(g.va, kk)];
        if (g.va.conj) v.y = -v.y;
      }
      const float rh = tf32_rna(v.x), ih = tf32_rna(v.y);
      const int o = tile_off(row, k);
      *reinterpret_cast<float*>(st + 0 * TILE_BYTES + o) = rh;
      *reinterpret_cast<float*>(st + 1 * TILE_BYTES + o) = tf32_rna(v.x - rh);
      *reinterpret_cast<float*>(st + 2 * TILE_BYTES + o) = ih;
      *reinterpret_cast<float*>(st + 3 * TILE_BYTES + o) = tf32_rna(v.y - ih);
    }
    for (int e = tid; e < TN * TK; e += NTH) {
      const int col = e % TN, k = e / TN;
      const int j = n0 + col, kk = k0 + k;
      cplx<float> v = mk<float>(0.f, 0.f);
      if (j < g.N && kk < g.K) {
        v = B[view_row(g.vb, kk) + view_col(g.vb, j)];
        if (g.vb.conj) v.y = -v.y;
      }
      const float rh = tf32_rna(v.x), ih = tf32_rna(v.y);
      const int o = tile_off(col, k);
      *reinterpret_cast<float*>(st + 4 * TILE_BYTES + o) = rh;
      *reinterpret_cast<float*>(st + 5 * TILE_BYTES + o) = tf32_rna(v.x - rh);
      *reinterpret_cast<float*>(st + 6 * TILE_BYTES + o) = ih;
      *reinterpret_cast<float*>(st + 7 * TILE_BYTES + o) = tf32_rna(v.y - ih);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy stores -> MMA reads
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(st);
      const uint64_t arh = smem_desc(base + 0 * TILE_BYTES), arl = smem_desc(base + 1 * TILE_BYTES);
      const uint64_t aih = smem_desc(base + 2 * TILE_BYTES), ail = smem_desc(base + 3 * TILE_BYTES);
      const uint64_t brh = smem_desc(base + 4 * TILE_BYTES), brl = smem_desc(base + 5 * TILE_BYTES);
      const uint64_t bih = smem_desc(base + 6 * TILE_BYTES), bil = smem_desc(base + 7 * TILE_BYTES);
      const uint32_t pos = instr_desc(0), neg = instr_desc(1);
      const uint32_t dre = tmem, dim = tmem + TN;
      const int acc = kt > 0 ? 1 : 0;
      // Re += Ar Br - Ai Bi
      mma_tf32(dre, arh, brh, pos, acc);
      mma_tf32(dre, arh, brl, pos, 1);
      mma_tf32(dre, arl, brh, pos, 1);
      mma_tf32(dre, aih, bih, neg, 1);
      mma_tf32(dre, aih, bil, neg, 1);
      mma_tf32(dre, ail, bih, neg, 1);
      // Im += Ar Bi + Ai Br
      mma_tf32(dim, arh, bih, pos, acc);
      mma_tf32(dim, arh, bil, pos, 1);
      mma_tf32(dim, arl, bih, pos, 1);
      mma_tf32(dim, aih, brh, pos, 1);
      mma_tf32(dim, aih, brl, pos, 1);
      mma_tf32(dim, ail, brh, pos, 1);
      mma_commit(smem_u32(&mbar[s]));
    }
    __syncthreads();
  }
  // every stage has exactly one commit not yet waited for (the last one made on it)
  for (int s = 0; s < STAGES && s < KT; ++s) {
    if (!mbar_wait(smem_u32(&mbar[s]), phase[s])) *s_fail = 1;
    phase[s] ^= 1;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  const bool ok = (*s_fail == 0);
  if (!ok && tid == 0) atomicExch(err_flag, 1);

  // epilogue: warp w reads TMEM lanes 32w..32w+31 (tile rows), 16 columns at a time
  const int row = warp * 32 + lane;
  const int i = m0 + row;
  const bool use_beta = (g.beta.x != 0.f || g.beta.y != 0.f);
  const int64_t ro = (i < g.M) ? view_row(g.vc, i) : 0;
  for (int c0 = 0; c0 < TN; c0 += 16) {
    uint32_t re[16], im[16];
    const uint32_t lane_addr = ((uint32_t)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]), "=r"(re[6]), "=r"(re[7]),
          "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]), "=r"(re[12]), "=r"(re[13]), "=r"(re[14]),
          "=r"(re[15])
        : "r"(tmem + lane_addr + c0));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]), "=r"(im[6]), "=r"(im[7]),
          "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]), "=r"(im[12]), "=r"(im[13]), "=r"(im[14]),
          "=r"(im[15])
        : "r"(tmem + lane_addr + TN + c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (!ok || i >= g.M) continue;
    for (int c = 0; c < 16; ++c) {
      const int j = n0 + c0 + c;
      if (j >= g.N) break;
      const int64_t o = ro + view_col(g.vc, j);
      cplx<float> v = g.alpha * mk<float>(__uint_as_float(re[c]), __uint_as_float(im[c]));
      if (use_beta) {
        cplx<float> old = C[o];
        if (g.vc.conj) old.y = -old.y;
        v = v + g.beta * old;
      }
      if (g.vc.conj) v.y = -v.y;
      C[o] = v;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

int* g_err = nullptr;
}  // namespace

bool tc_gemm_applicable(const GemmArgs<float>& g) { return !g.herm && g.M >= TM && g.N >= 64 && g.K >= TK; }

cudaError_t tc_gemm(cudaStream_t s, int batch, const GemmArgs<float>& g) {
  if (batch <= 0 || g.M <= 0 || g.N <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    // at most two CTAs per SM (TMEM: 2 x 256 columns of 512), so no allocation ever waits
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    if (e != cudaSuccess) return e;
    if (!g_err) {
      e = cudaMalloc(&g_err, sizeof(int));
      if (e != cudaSuccess) return e;
      e = cudaMemset(g_err, 0, sizeof(int));
      if (e != cudaSuccess) return e;
    }
    attr = true;
  }
  dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, batch);
  tc_gemm_kernel<<<grid, NTH, 100 * 1024, s>>>(g, g_err);
  return cudaGetLastError();
}

int tc_gemm_error_flag() {
  if (!g_err) return 0;
  int h = 0;
  cudaMemcpy(&h, g_err, sizeof(int), cudaMemcpyDeviceToHost);
  return h;
}

}  // namespace mpdo

// ---------------------------------------------------------------------------------------------
// Self-test: random complex64 operands, the tensor-core product against the CUDA-core GEMM.
extern "C" mpdo_status mpdo_tc_selftest(int M, int N, int K, double* max_rel_err, int* err_flag) {
  using namespace mpdo;
  if (M < 1 || N < 1 || K < 1 || !max_rel_err || !err_flag) return MPDO_EINVAL;
  std::vector<cplx<float>> ha((size_t)M * K), hb((size_t)K * N);
  uint64_t st = 12345;
  auto rnd = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (float)((int64_t)(st >> 40) - (1ll << 23)) / (float)(1 << 23);
  };
  for (auto& v : ha) v = mk<float>(rnd(), rnd());
  for (auto& v : hb) v = mk<float>(rnd(), rnd());
  cplx<float>*da = nullptr, *db = nullptr, *dc = nullptr, *dr = nullptr;
  mpdo_status ret = MPDO_OK;
  if (cudaMalloc(&da, sizeof(cplx<float>) * ha.size()) != cudaSuccess ||
      cudaMalloc(&db, sizeof(cplx<float>) * hb.size()) != cudaSuccess ||
      cudaMalloc(&dc, sizeof(cplx<float>) * (size_t)M * N) != cudaSuccess ||
      cudaMalloc(&dr, sizeof(cplx<float>) * (size_t)M * N) != cudaSuccess) {
    ret = MPDO_ENOMEM;
  } else {
    cudaMemcpy(da, ha.data(), sizeof(cplx<float>) * ha.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(db, hb.data(), sizeof(cplx<float>) * hb.size(), cudaMemcpyHostToDevice);
    GemmArgs<float> g;
    g.M = M;
    g.N = N;
    g.K = K;
    g.alpha = mk<float>(1, 0);
    g.beta = mk<float>(0, 0);
    g.A = da;
    g.va = row_major(K, 0);
    g.B = db;
    g.vb = row_major(N, 0);
    g.C = dc;
    g.vc = row_major(N, 0);
    g.herm = 0;
    if (tc_gemm(nullptr, 1, g) != cudaSuccess) ret = MPDO_ECUDA;
    g.C = dr;
    if (!ret && gemm<float>(nullptr, 1, g) != cudaSuccess) ret = MPDO_ECUDA;
    if (!ret && cudaDeviceSynchronize() != cudaSuccess) ret = MPDO_ECUDA;
    if (!ret) {
      std::vector<cplx<float>> hc((size_t)M * N), hr((size_t)M * N);
      cudaMemcpy(hc.data(), dc, sizeof(cplx<float>) * hc.size(), cudaMemcpyDeviceToHost);
      cudaMemcpy(hr.data(), dr, sizeof(cplx<float>) * hr.size(), cudaMemcpyDeviceToHost);
      double num = 0, den = 0;
      for (size_t e = 0; e < hc.size(); ++e) {
        double dx = (double)hc[e].x - hr[e].x, dy = (double)hc[e].y - hr[e].y;
        num = std::max(num, std::sqrt(dx * dx + dy * dy));
        den = std::max(den, std::sqrt((double)hr[e].x * hr[e].x + (double)hr[e].y * hr[e].y));
      }
      *max_rel_err = den > 0 ? num / den : num;
      *err_flag = tc_gemm_error_flag();
    }
  }
  cudaFree(da);
  cudaFree(db);
  cudaFree(dc);
  cudaFree(dr);
  return ret;
}
