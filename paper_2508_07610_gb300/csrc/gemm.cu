// Batched complex GEMM over strided tensor views (CUDA cores, FP32 or FP64 complex).
//   C[z](i, j) = alpha * sum_k opA[z](i, k) * opB[z](k, j) + beta * C[z](i, j)
// Every operand is addressed through a View, so site tensors are multiplied in place
// in whatever index grouping a contraction needs (no permute copies).
#include "kernels.h"

namespace mpdo {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename R>
struct kCompensated {
  static constexpr bool value = false;
};
template <>
struct kCompensated<float> {
  static constexpr bool value = true;
};
// s + c += x with Knuth's TwoSum: s takes the rounded sum, c collects the exact rounding error
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  float t = __fadd_rn(s, x);
  float bp = __fsub_rn(t, s);
  float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  s = t;
  c = __fadd_rn(c, err);
}

template <typename R>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs<R> g, int a_m_fast, int b_n_fast) {
  __shared__ cplx<R> As[BK][BM];
  __shared__ cplx<R> Bs[BK][BN];
  const int z = blockIdx.z;
  const cplx<R>* A = g.A + view_batch(g.va, z);
  const cplx<R>* B = g.B + view_batch(g.vb, z);
  cplx<R>* C = g.C + view_batch(g.vc, z);
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;

  // Per-thread load coordinates that stay fixed over the K loop.
  int64_t aoff[4];
  int ai[4], ak[4];
  for (int t = 0; t < 4; ++t) {
    int e = tid + t * NT;
    if (a_m_fast) { ai[t] = e % BM; ak[t] = e / BM; } else { ak[t] = e % BK; ai[t] = e / BK; }
    int i = m0 + ai[t];
    aoff[t] = (i < g.M) ? view_row(g.va, i) : -1;
  }
  int64_t boff[4];
  int bj[4], bk[4];
  for (int t = 0; t < 4; ++t) {
    int e = tid + t * NT;
    if (b_n_fast) { bj[t] = e % BN; bk[t] = e / BN; } else { bk[t] = e % BK; bj[t] = e / BK; }
    int j = n0 + bj[t];
    boff[t] = (j < g.N) ? view_col(g.vb, j) : -1;
  }

  // acc holds the running sum; for FP32 each k-tile is summed into `part` first and added to
  // (acc, comp) with an error-free TwoSum, so the rounding error no longer grows with K.
  cplx<R> acc[4][4], comp[4][4];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      acc[r][c] = mk<R>(0, 0);
      comp[r][c] = mk<R>(0, 0);
    }

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int t = 0; t < 4; ++t) {
      int k = k0 + ak[t];
      cplx<R> v = mk<R>(0, 0);
      if (aoff[t] >= 0 && k < g.K) {
        v = A[aoff[t] + view_col(g.va, k)];
        if (g.va.conj) v.y = -v.y;
      }
      As[ak[t]][ai[t]] = v;
    }
    for (int t = 0; t < 4; ++t) {
      int k = k0 + bk[t];
      cplx<R> v = mk<R>(0, 0);
      if (boff[t] >= 0 && k < g.K) {
        v = B[boff[t] + view_row(g.vb, k)];
        if (g.vb.conj) v.y = -v.y;
      }
      Bs[bk[t]][bj[t]] = v;
    }
    __syncthreads();
    if constexpr (kCompensated<R>::value) {
      cplx<R> part[4][4];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) part[r][c] = mk<R>(0, 0);
#pragma unroll 4
      for (int kk = 0; kk < BK; ++kk) {
        cplx<R> a[4], b[4];
        for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
        for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < 4; ++c) cfma(part[r][c], a[r], b[c]);
      }
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          two_sum_acc(acc[r][c].x, comp[r][c].x, part[r][c].x);
          two_sum_acc(acc[r][c].y, comp[r][c].y, part[r][c].y);
        }
    } else {
#pragma unroll 4
      for (int kk = 0; kk < BK; ++kk) {
        cplx<R> a[4], b[4];
        for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
        for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < 4; ++c) cfma(acc[r][c], a[r], b[c]);
      }
    }
    __syncthreads();
  }

  const bool use_beta = (g.beta.x != R(0) || g.beta.y != R(0));
  for (int r = 0; r < 4; ++r) {
    int i = m0 + ty + 16 * r;
    if (i >= g.M) continue;
    int64_t ro = view_row(g.vc, i);
    for (int c = 0; c < 4; ++c) {
      int j = n0 + tx + 16 * c;
      if (j >= g.N) continue;
      int64_t o = ro + view_col(g.vc, j);
      cplx<R> v = g.alpha * (acc[r][c] + comp[r][c]);
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
}  // namespace

template <typename R>
cudaError_t gemm(cudaStream_t s, int batch, const GemmArgs<R>& g) {
  if (batch <= 0 || g.M <= 0 || g.N <= 0) return cudaSuccess;
  int a_m_fast = (g.va.rdiv == 0 && g.va.rlo == 1) ? 1 : 0;
  int b_n_fast = (g.vb.cdiv == 0 && g.vb.clo == 1) ? 1 : 0;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, batch);
  gemm_kernel<R><<<grid, NT, 0, s>>>(g, a_m_fast, b_n_fast);
  return cudaGetLastError();
}

template cudaError_t gemm<float>(cudaStream_t, int, const GemmArgs<float>&);
template cudaError_t gemm<double>(cudaStream_t, int, const GemmArgs<double>&);

}  // namespace mpdo
