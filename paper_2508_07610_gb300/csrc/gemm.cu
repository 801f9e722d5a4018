// Batched complex GEMM over strided tensor views (CUDA cores, FP32 or FP64 complex).
//   C[z](i, j) = alpha * sum_k opA[z](i, k) * opB[z](k, j) + beta * C[z](i, j)
// Every operand is addressed through a View, so site tensors are multiplied in place in whatever
// index grouping a contraction needs (no permute copies).
//
// Tiling: 256 threads per CTA on a 16 x 16 thread grid.  Thread (ty, tx) owns rows ty*TMR .. +TMR-1
// and columns tx, tx+16, ..., tx+16(TNC-1) of the CTA tile (16 TMR x 16 TNC), so the B fragment
// reads of a warp hit consecutive shared-memory words and the C stores of a warp are contiguous.
// Operands move global -> shared memory with element-wise cp.async (8 or 16 bytes, zero-filled
// outside the matrix) through a STAGES-deep ring of k-tiles of 16, so loads for later k-tiles are in
// flight while the current one is multiplied, without staging registers.  The per-row (A) and
// per-column (B) view offsets of the tile are computed once into shared memory.
// FP32 reductions sum each k-tile into a fresh partial and add it to the running value with Knuth's
// TwoSum, so their rounding error does not grow with K.
// Long reductions whose output has too few tiles to fill the GPU (the Kraus-leg Grams: 128 x 128
// or 32 x 32 per chain over 8192 rows) are split along K over several CTAs; each writes its partial
// tile to a workspace and a second kernel adds the partials in FP64 and applies alpha and beta.
#include "device_once.cuh"
#include "kernels.h"

namespace mpdo {

namespace {
constexpr int BK = 16, NT = 256;
constexpr int PAD = 1;  // one element of padding per k-row: k-fast copies of a warp land in distinct banks

// s + c += x with Knuth's TwoSum: s takes the rounded sum, c collects the exact rounding error
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  float t = __fadd_rn(s, x);
  float bp = __fsub_rn(t, s);
  float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  s = t;
  c = __fadd_rn(c, err);
}
__device__ __forceinline__ void two_sum_acc(double& s, double& c, double x) { s += x; }

// one complex element global -> shared, zero-filled when !valid (src must still be a valid address)
template <typename R>
__device__ __forceinline__ void cp_elem(cplx<R>* dst, const cplx<R>* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? (int)sizeof(cplx<R>) : 0;
  if constexpr (sizeof(cplx<R>) == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename R, int TMR, int TNC, int STAGES>
constexpr size_t smem_bytes() {
  return sizeof(cplx<R>) * (size_t)STAGES * BK * (16 * TMR + 16 * TNC + 2 * PAD) +
         sizeof(int64_t) * (16 * TMR + 16 * TNC);
}

template <typename R, bool COMP, int TMR, int TNC, int STAGES>
__global__ void __launch_bounds__(NT, 2) gemm_kernel(GemmArgs<R> g, int a_m_fast, int b_n_fast, int sk, int kc,
                                                     int ty0) {
  constexpr int BM = 16 * TMR, BN = 16 * TNC, SA = BM + PAD, SB = BN + PAD;
  constexpr int LA = BM * BK / NT, LB = BN * BK / NT;  // elements each thread copies per k-tile
  static_assert(LA >= 1 && LB >= 1, "tile too small for the thread count");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* As = reinterpret_cast<cplx<R>*>(smem_raw);  // [STAGES][BK][SA]
  cplx<R>* Bs = As + STAGES * BK * SA;                  // [STAGES][BK][SB]
  int64_t* rowA = reinterpret_cast<int64_t*>(Bs + STAGES * BK * SB);  // [BM], -1 outside
  int64_t* colB = rowA + BM;                                          // [BN], -1 outside

  const int z = blockIdx.z / sk, kz = blockIdx.z % sk;  // batch item, K chunk
  const int kb = kz * kc, ke = (g.K - kb < kc) ? g.K : kb + kc;
  const int m0 = (blockIdx.y + ty0) * BM, n0 = blockIdx.x * BN;  // ty0: row-tile offset of this launch
  if (g.herm && n0 > m0 + BM - 1) return;  // tile strictly above the diagonal of a Hermitian result
  const cplx<R>* A = g.A + view_batch(g.va, z);
  const cplx<R>* B = g.B + view_batch(g.vb, z);
  cplx<R>* C = g.C + view_batch(g.vc, z);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;

  for (int i = tid; i < BM; i += NT) rowA[i] = (m0 + i < g.M) ? view_row(g.va, m0 + i) : -1;
  for (int j = tid; j < BN; j += NT) colB[j] = (n0 + j < g.N) ? view_col(g.vb, n0 + j) : -1;
  __syncthreads();

  // element e = tid + t * NT of a k-tile is (row, k) = (e % BM, e / BM) when A is row-fast, else
  // (e / BK, e % BK); likewise for B (tile sizes are powers of two: shifts and masks)
  auto load_tile = [&](int stage, int k0) {
    cplx<R>* as = As + stage * BK * SA;
    cplx<R>* bs = Bs + stage * BK * SB;
#pragma unroll
    for (int t = 0; t < LA; ++t) {
      const int e = tid + t * NT;
      const int ai = a_m_fast ? e % BM : e / BK, ak = a_m_fast ? e / BM : e % BK;
      const int k = k0 + ak;
      const int64_t ro = rowA[ai];
      const bool ok = ro >= 0 && k < ke;
      cp_elem(as + ak * SA + ai, ok ? GP(A + ro + view_col(g.va, k)) : A, ok);
    }
#pragma unroll
    for (int t = 0; t < LB; ++t) {
      const int e = tid + t * NT;
      const int bj = b_n_fast ? e % BN : e / BK, bk = b_n_fast ? e / BN : e % BK;
      const int k = k0 + bk;
      const int64_t co = colB[bj];
      const bool ok = co >= 0 && k < ke;
      cp_elem(bs + bk * SB + bj, ok ? GP(B + co + view_row(g.vb, k)) : B, ok);
    }
  };

  cplx<R> acc[TMR][TNC], comp[COMP ? TMR : 1][COMP ? TNC : 1];
#pragma unroll
  for (int r = 0; r < TMR; ++r)
#pragma unroll
    for (int c = 0; c < TNC; ++c) acc[r][c] = mk<R>(0, 0);
  if constexpr (COMP) {
#pragma unroll
    for (int r = 0; r < TMR; ++r)
#pragma unroll
      for (int c = 0; c < TNC; ++c) comp[r][c] = mk<R>(0, 0);
  }
  const bool conjA = g.va.conj != 0, conjB = g.vb.conj != 0;

  const int nk = (ke - kb + BK - 1) / BK;
#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < nk) load_tile(s, kb + s * BK);
    cp_commit();
  }
  for (int kt = 0; kt < nk; ++kt) {
    cp_wait<STAGES - 2>();
    __syncthreads();  // tile kt is in shared memory for every thread; stage (kt - 1) is free
    {
      const int pf = kt + STAGES - 1;
      if (pf < nk) load_tile(pf % STAGES, kb + pf * BK);
      cp_commit();
    }
    const cplx<R>* as = As + (kt % STAGES) * BK * SA;
    const cplx<R>* bs = Bs + (kt % STAGES) * BK * SB;
    cplx<R> part[COMP ? TMR : 1][COMP ? TNC : 1];
    if constexpr (COMP) {
#pragma unroll
      for (int r = 0; r < TMR; ++r)
#pragma unroll
        for (int c = 0; c < TNC; ++c) part[r][c] = mk<R>(0, 0);
    }
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      cplx<R> a[TMR], b[TNC];
#pragma unroll
      for (int r = 0; r < TMR; ++r) {
        a[r] = as[kk * SA + ty * TMR + r];
        if (conjA) a[r].y = -a[r].y;
      }
#pragma unroll
      for (int c = 0; c < TNC; ++c) {
        b[c] = bs[kk * SB + tx + 16 * c];
        if (conjB) b[c].y = -b[c].y;
      }
#pragma unroll
      for (int r = 0; r < TMR; ++r)
#pragma unroll
        for (int c = 0; c < TNC; ++c) {
          if constexpr (COMP) cfma(part[r][c], a[r], b[c]);
          else cfma(acc[r][c], a[r], b[c]);
        }
    }
    if constexpr (COMP) {
#pragma unroll
      for (int r = 0; r < TMR; ++r)
#pragma unroll
        for (int c = 0; c < TNC; ++c) {
          two_sum_acc(acc[r][c].x, comp[r][c].x, part[r][c].x);
          two_sum_acc(acc[r][c].y, comp[r][c].y, part[r][c].y);
        }
    }
  }
  cp_wait<0>();

  if (sk > 1) {  // partial tile of K chunk kz -> workspace [z][kz][M][N]
    cplx<R>* P = g.ws + ((int64_t)z * sk + kz) * g.M * g.N;
#pragma unroll
    for (int r = 0; r < TMR; ++r) {
      const int i = m0 + ty * TMR + r;
      if (i >= g.M) continue;
#pragma unroll
      for (int c = 0; c < TNC; ++c) {
        const int j = n0 + tx + 16 * c;
        if (j >= g.N) continue;
        cplx<R> sum = acc[r][c];
        if constexpr (COMP) sum = sum + comp[r][c];
        GX(P, (int64_t)i * g.N + j) = sum;
      }
    }
    return;
  }
  const bool use_beta = (g.beta.x != R(0) || g.beta.y != R(0));
#pragma unroll
  for (int r = 0; r < TMR; ++r) {
    const int i = m0 + ty * TMR + r;
    if (i >= g.M) continue;
    const int64_t ro = view_row(g.vc, i);
#pragma unroll
    for (int c = 0; c < TNC; ++c) {
      const int j = n0 + tx + 16 * c;
      if (j >= g.N) continue;
      const int64_t o = ro + view_col(g.vc, j);
      cplx<R> sum = acc[r][c];
      if constexpr (COMP) sum = sum + comp[r][c];
      cplx<R> v = g.alpha * sum;
      if (use_beta) {
        cplx<R> old = GX(C, o);
        if (g.vc.conj) old.y = -old.y;
        v = v + g.beta * old;
      }
      if (g.vc.conj) v.y = -v.y;
      GX(C, o) = v;
    }
  }
}

// C = alpha * (sum of the sk partials, in FP64) + beta * C; Hermitian results only on and below the
// diagonal (the caller mirrors the strict upper triangle)
template <typename R>
__global__ void splitk_reduce_kernel(GemmArgs<R> g, int sk) {
  const int z = blockIdx.y;
  const int64_t MN = (int64_t)g.M * g.N;
  const cplx<R>* P = g.ws + (int64_t)z * sk * MN;
  cplx<R>* C = g.C + view_batch(g.vc, z);
  const bool use_beta = (g.beta.x != R(0) || g.beta.y != R(0));
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / g.N), j = (int)(e % g.N);
    if (g.herm && j > i) continue;
    double sx = 0, sy = 0;
    for (int t = 0; t < sk; ++t) {
      const cplx<R> p = GX(P, t * MN + e);
      sx += (double)p.x;
      sy += (double)p.y;
    }
    cplx<R> v = g.alpha * mk<R>((R)sx, (R)sy);
    const int64_t o = view_row(g.vc, i) + view_col(g.vc, j);
    if (use_beta) {
      cplx<R> old = GX(C, o);
      if (g.vc.conj) old.y = -old.y;
      v = v + g.beta * old;
    }
    if (g.vc.conj) v.y = -v.y;
    GX(C, o) = v;
  }
}

template <typename R, bool COMP, int TMR, int TNC>
cudaError_t launch(cudaStream_t s, int batch, const GemmArgs<R>& g) {
  constexpr int BM = 16 * TMR, BN = 16 * TNC;
  // three stages for complex64, two for complex128 (twice the bytes per element)
  constexpr int STAGES = sizeof(R) == 4 ? 3 : 2;
  constexpr size_t bytes = smem_bytes<R, TMR, TNC, STAGES>();
  static PerDevice setup;
  {
    cudaError_t e = setup.once([](int) {
      return cudaFuncSetAttribute(gemm_kernel<R, COMP, TMR, TNC, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)bytes);
    });
    if (e != cudaSuccess) return e;
  }
  const int n_sm = sm_count();
  const int a_m_fast = (g.va.rdiv == 0 && g.va.rlo == 1) ? 1 : 0;
  const int b_n_fast = (g.vb.cdiv == 0 && g.vb.clo == 1) ? 1 : 0;
  const int tm = (g.M + BM - 1) / BM, tn = (g.N + BN - 1) / BN;
  // split K when the output tiles (on and below the diagonal for a Hermitian result) cannot keep
  // two CTAs on every SM busy for four waves and each chunk still spans at least 64 k-tiles
  int sk = 1;
  if (g.ws && g.K >= 1024) {
    const int64_t tiles = (int64_t)(g.herm ? tm * (tm + 1) / 2 : tm * tn) * batch;
    const int64_t want = (8 * (int64_t)n_sm + tiles - 1) / tiles;
    const int64_t most = g.K / (64 * BK);
    sk = (int)(want < most ? want : most);
    if (sk > 8) sk = 8;
    while (sk > 1 && ((int64_t)sk * g.M * g.N * batch > g.ws_elems || (int64_t)sk * batch > 65535)) --sk;
    if (sk < 1) sk = 1;
  }
  const int kc = (sk > 1) ? ((g.K + sk - 1) / sk + BK - 1) / BK * BK : (g.K > 0 ? g.K : 1);
  if (sk > 1) sk = (g.K + kc - 1) / kc;
  // grid.y is limited to 65535 row tiles per launch: taller outputs (the purity contraction) take
  // several launches over consecutive row-tile ranges
  constexpr int kMaxY = 65535;
  cudaError_t e = cudaSuccess;
  for (int ty0 = 0; ty0 < tm; ty0 += kMaxY) {
    dim3 grid(tn, (tm - ty0 < kMaxY) ? tm - ty0 : kMaxY, batch * sk);
    gemm_kernel<R, COMP, TMR, TNC, STAGES><<<grid, NT, bytes, s>>>(g, a_m_fast, b_n_fast, sk, kc, ty0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (sk == 1) return e;
  const int64_t mn = (int64_t)g.M * g.N;
  dim3 rgrid((unsigned)((mn + 255) / 256 < 1024 ? (mn + 255) / 256 : 1024), batch);
  splitk_reduce_kernel<R><<<rgrid, 256, 0, s>>>(g, sk);
  return cudaGetLastError();
}
}  // namespace

template <typename R>
cudaError_t gemm(cudaStream_t s, int batch, const GemmArgs<R>& g) {
  if (batch <= 0 || g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.herm && g.M != g.N) return cudaErrorInvalidValue;
  // small outputs (<= 32 x 32 per batch item: the Kraus-leg Gram of a 1q gate, the rank-kappa
  // projection) take 32 x 32 tiles so that no tile is mostly padding
  // outputs of at most 16 rows and many columns (the rank-kappa projections, kappa x 8192) take
  // 16 x 128 tiles
  const bool small = g.M <= 32 && g.N <= 32;
  const bool wide = g.M <= 16 && g.N > 32 && !g.herm;
  if constexpr (sizeof(R) == 4) {
    if (g.allow_tc && tc_gemm_applicable(g, batch)) return tc_gemm(s, batch, g);
    // every FP32 product sums its k-tiles with TwoSum: the stored complex64 state is rounded at
    // every step anyway, and uncompensated sums of even 64 terms added measurably to it
    if (wide) return launch<R, true, 1, 8>(s, batch, g);
    return small ? launch<R, true, 2, 2>(s, batch, g) : launch<R, true, 4, 4>(s, batch, g);
  } else {
    if (wide) return launch<R, false, 1, 8>(s, batch, g);
    return small ? launch<R, false, 2, 2>(s, batch, g) : launch<R, false, 4, 4>(s, batch, g);
  }
}

template cudaError_t gemm<float>(cudaStream_t, int, const GemmArgs<float>&);
template cudaError_t gemm<double>(cudaStream_t, int, const GemmArgs<double>&);

}  // namespace mpdo
