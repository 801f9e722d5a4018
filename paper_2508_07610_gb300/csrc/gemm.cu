// Batched complex GEMM over strided tensor views (CUDA cores, FP32 or FP64 complex).
//   C[z](i, j) = alpha * sum_k opA[z](i, k) * opB[z](k, j) + beta * C[z](i, j)
// Every operand is addressed through a View, so site tensors are multiplied in place in whatever
// index grouping a contraction needs (no permute copies).
//
// Tiling: 256 threads per CTA on a 16 x 16 thread grid; each thread owns a TMR x TNC block of
// contiguous rows and columns of the CTA tile (16 TMR x 16 TNC), operands are staged through shared
// memory in k-tiles of 16 with the next tile's global loads issued before the current tile is used.
// Long FP32 reductions (K >= 1024, the Gram matrices of the truncations) sum each k-tile into a fresh
// partial and add it to the running value with Knuth's TwoSum, so their rounding error does not grow
// with K; the other products accumulate directly.
#include "kernels.h"

namespace mpdo {

namespace {
constexpr int BK = 16, NT = 256;

// s + c += x with Knuth's TwoSum: s takes the rounded sum, c collects the exact rounding error
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  float t = __fadd_rn(s, x);
  float bp = __fsub_rn(t, s);
  float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  s = t;
  c = __fadd_rn(c, err);
}
__device__ __forceinline__ void two_sum_acc(double& s, double& c, double x) { s += x; }

template <typename R, bool COMP, int TMR, int TNC>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs<R> g, int a_m_fast, int b_n_fast) {
  constexpr int BM = 16 * TMR, BN = 16 * TNC;
  constexpr int LA = BM * BK / NT, LB = BN * BK / NT;  // elements each thread stages per k-tile
  __shared__ cplx<R> As[BK][BM];
  __shared__ cplx<R> Bs[BK][BN];
  const int z = blockIdx.z;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (g.herm && n0 > m0 + BM - 1) return;  // tile strictly above the diagonal of a Hermitian result
  const cplx<R>* A = g.A + view_batch(g.va, z);
  const cplx<R>* B = g.B + view_batch(g.vb, z);
  cplx<R>* C = g.C + view_batch(g.vc, z);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;

  int64_t aoff[LA];
  int ai[LA], ak[LA];
#pragma unroll
  for (int t = 0; t < LA; ++t) {
    int e = tid + t * NT;
    if (a_m_fast) { ai[t] = e % BM; ak[t] = e / BM; } else { ak[t] = e % BK; ai[t] = e / BK; }
    int i = m0 + ai[t];
    aoff[t] = (i < g.M) ? view_row(g.va, i) : -1;
  }
  int64_t boff[LB];
  int bj[LB], bk[LB];
#pragma unroll
  for (int t = 0; t < LB; ++t) {
    int e = tid + t * NT;
    if (b_n_fast) { bj[t] = e % BN; bk[t] = e / BN; } else { bk[t] = e % BK; bj[t] = e / BK; }
    int j = n0 + bj[t];
    boff[t] = (j < g.N) ? view_col(g.vb, j) : -1;
  }
  cplx<R> ra[LA], rb[LB];
  auto load_tile = [&](int k0) {
#pragma unroll
    for (int t = 0; t < LA; ++t) {
      int k = k0 + ak[t];
      cplx<R> v = mk<R>(0, 0);
      if (aoff[t] >= 0 && k < g.K) {
        v = A[aoff[t] + view_col(g.va, k)];
        if (g.va.conj) v.y = -v.y;
      }
      ra[t] = v;
    }
#pragma unroll
    for (int t = 0; t < LB; ++t) {
      int k = k0 + bk[t];
      cplx<R> v = mk<R>(0, 0);
      if (boff[t] >= 0 && k < g.K) {
        v = B[boff[t] + view_row(g.vb, k)];
        if (g.vb.conj) v.y = -v.y;
      }
      rb[t] = v;
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

  load_tile(0);
  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int t = 0; t < LA; ++t) As[ak[t]][ai[t]] = ra[t];
#pragma unroll
    for (int t = 0; t < LB; ++t) Bs[bk[t]][bj[t]] = rb[t];
    __syncthreads();
    if (k0 + BK < g.K) load_tile(k0 + BK);  // next tile's loads in flight during the products
    if constexpr (COMP) {
      cplx<R> part[TMR][TNC];
#pragma unroll
      for (int r = 0; r < TMR; ++r)
#pragma unroll
        for (int c = 0; c < TNC; ++c) part[r][c] = mk<R>(0, 0);
#pragma unroll 4
      for (int kk = 0; kk < BK; ++kk) {
        cplx<R> a[TMR], b[TNC];
#pragma unroll
        for (int r = 0; r < TMR; ++r) a[r] = As[kk][ty * TMR + r];
#pragma unroll
        for (int c = 0; c < TNC; ++c) b[c] = Bs[kk][tx * TNC + c];
#pragma unroll
        for (int r = 0; r < TMR; ++r)
#pragma unroll
          for (int c = 0; c < TNC; ++c) cfma(part[r][c], a[r], b[c]);
      }
#pragma unroll
      for (int r = 0; r < TMR; ++r)
#pragma unroll
        for (int c = 0; c < TNC; ++c) {
          two_sum_acc(acc[r][c].x, comp[r][c].x, part[r][c].x);
          two_sum_acc(acc[r][c].y, comp[r][c].y, part[r][c].y);
        }
    } else {
#pragma unroll 4
      for (int kk = 0; kk < BK; ++kk) {
        cplx<R> a[TMR], b[TNC];
#pragma unroll
        for (int r = 0; r < TMR; ++r) a[r] = As[kk][ty * TMR + r];
#pragma unroll
        for (int c = 0; c < TNC; ++c) b[c] = Bs[kk][tx * TNC + c];
#pragma unroll
        for (int r = 0; r < TMR; ++r)
#pragma unroll
          for (int c = 0; c < TNC; ++c) cfma(acc[r][c], a[r], b[c]);
      }
    }
    __syncthreads();
  }

  const bool use_beta = (g.beta.x != R(0) || g.beta.y != R(0));
#pragma unroll
  for (int r = 0; r < TMR; ++r) {
    int i = m0 + ty * TMR + r;
    if (i >= g.M) continue;
    int64_t ro = view_row(g.vc, i);
#pragma unroll
    for (int c = 0; c < TNC; ++c) {
      int j = n0 + tx * TNC + c;
      if (j >= g.N) continue;
      int64_t o = ro + view_col(g.vc, j);
      cplx<R> sum = acc[r][c];
      if constexpr (COMP) sum = sum + comp[r][c];
      cplx<R> v = g.alpha * sum;
      if (use_beta) {
        cplx<R> old = C[o];
        if (g.vc.conj) old.y = -old.y;
        v = v + g.beta * old;
      }
      if (g.vc.conj) v.y = -v.y;
      C[o] = v;
    }
  }
}

template <typename R, bool COMP, int TMR, int TNC>
cudaError_t launch(cudaStream_t s, int batch, const GemmArgs<R>& g) {
  constexpr int BM = 16 * TMR, BN = 16 * TNC;
  int a_m_fast = (g.va.rdiv == 0 && g.va.rlo == 1) ? 1 : 0;
  int b_n_fast = (g.vb.cdiv == 0 && g.vb.clo == 1) ? 1 : 0;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, batch);
  gemm_kernel<R, COMP, TMR, TNC><<<grid, NT, 0, s>>>(g, a_m_fast, b_n_fast);
  return cudaGetLastError();
}
}  // namespace

template <typename R>
cudaError_t gemm(cudaStream_t s, int batch, const GemmArgs<R>& g) {
  if (batch <= 0 || g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.herm && g.M != g.N) return cudaErrorInvalidValue;
  // small outputs (<= 32 x 32 per batch item: the Kraus-leg Gram of a 1q gate, the rank-kappa
  // projection) take 32 x 32 tiles so that no tile is mostly padding
  const bool small = g.M <= 32 && g.N <= 32;
  if constexpr (sizeof(R) == 4) {
    if (g.allow_tc && g.K <= 2048 && tc_gemm_applicable(g)) return tc_gemm(s, batch, g);
    if (g.K >= 1024) return small ? launch<R, true, 2, 2>(s, batch, g) : launch<R, true, 4, 4>(s, batch, g);
    if (g.M > 64 && !g.herm) return launch<R, false, 8, 4>(s, batch, g);
    return small ? launch<R, false, 2, 2>(s, batch, g) : launch<R, false, 4, 4>(s, batch, g);
  } else {
    return small ? launch<R, false, 2, 2>(s, batch, g) : launch<R, false, 4, 4>(s, batch, g);
  }
}

template cudaError_t gemm<float>(cudaStream_t, int, const GemmArgs<float>&);
template cudaError_t gemm<double>(cudaStream_t, int, const GemmArgs<double>&);

}  // namespace mpdo
