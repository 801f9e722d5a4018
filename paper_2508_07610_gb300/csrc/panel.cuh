// Block-reflector helpers shared by the blocked Householder QR and the eigensolver's
// back-transformation (256-thread CTAs).  A panel of pb <= NB Householder vectors sits in shared
// memory (vector i at Vs + i * ldv); the product H_0 ... H_{pb-1} = I - V T V^H (compact WY form,
// T upper triangular) is applied to a block of columns as two small matrix products.  The block of
// columns A is in global memory (its accesses are checked in the address-checked build); the panel,
// T and the products are in shared memory.
#pragma once
#include "kernels.h"

namespace mpdo {
namespace panel {
constexpr int NT = 256;

template <typename R>
__device__ __forceinline__ cplx<R> warp_csum(cplx<R> v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Ws[i * ldw + c] = (V^H A)[i][c] over a block of columns, A column-major (ld lda, rows 0..M-1 of
// the block), V = the panel's pb reflectors in shared memory (column i at Vs + i * ldv).
template <typename R, int NB>
__device__ void panel_vh_times(const cplx<R>* A, int64_t lda, int M, int nc, const cplx<R>* Vs, int ldv, int pb,
                               cplx<R>* Ws, int ldw) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c0 = 2 * wid; c0 < nc; c0 += 2 * (NT / 32)) {
    const bool two = c0 + 1 < nc;
    cplx<R> acc0[NB], acc1[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) acc0[i] = acc1[i] = mk<R>(0, 0);
    const cplx<R>* a0p = A + (int64_t)c0 * lda;
    const cplx<R>* a1p = a0p + lda;
#pragma unroll 4
    for (int r = lane; r < M; r += 32) {
      const cplx<R> a0 = GX(a0p, r);
      const cplx<R> a1 = two ? GX(a1p, r) : mk<R>(0, 0);
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        if (i < pb) {
          const cplx<R> v = Vs[i * ldv + r];
          cfma_cj(acc0[i], v, a0);
          cfma_cj(acc1[i], v, a1);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      if (i < pb) {
        const cplx<R> s0 = warp_csum(acc0[i]);
        const cplx<R> s1 = warp_csum(acc1[i]);
        if (lane == 0) {
          Ws[i * ldw + c0] = s0;
          if (two) Ws[i * ldw + c0 + 1] = s1;
        }
      }
    }
  }
}

// A -= V Y over a block of columns, Y[i][c] = Ws[i * ldw + c].
template <typename R, int NB>
__device__ void panel_minus_v_times(cplx<R>* A, int64_t lda, int M, int nc, const cplx<R>* Vs, int ldv, int pb,
                                    const cplx<R>* Ws, int ldw) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c0 = 2 * wid; c0 < nc; c0 += 2 * (NT / 32)) {
    const bool two = c0 + 1 < nc;
    cplx<R> y0[NB], y1[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      y0[i] = (i < pb) ? Ws[i * ldw + c0] : mk<R>(0, 0);
      y1[i] = (i < pb && two) ? Ws[i * ldw + c0 + 1] : mk<R>(0, 0);
    }
    cplx<R>* a0p = A + (int64_t)c0 * lda;
    cplx<R>* a1p = a0p + lda;
    // RU rows per lane per pass: their loads are issued together before any update is stored
    constexpr int RU = 4;
    for (int r0 = lane; r0 < M; r0 += 32 * RU) {
      cplx<R> x0[RU], x1[RU];
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int r = r0 + 32 * u;
        if (r < M) {
          x0[u] = GX(a0p, r);
          x1[u] = two ? GX(a1p, r) : mk<R>(0, 0);
        }
      }
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int r = r0 + 32 * u;
        if (r >= M) continue;
        cplx<R> s0 = mk<R>(0, 0), s1 = mk<R>(0, 0);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          if (i < pb) {
            const cplx<R> v = Vs[i * ldv + r];
            cfma(s0, v, y0[i]);
            cfma(s1, v, y1[i]);
          }
        }
        GX(a0p, r) = x0[u] - s0;
        if (two) GX(a1p, r) = x1[u] - s1;
      }
    }
  }
}

// Ws[., c] <- T^H Ws[., c] (herm) or T Ws[., c]; T upper triangular pb x pb, column-major, ld NB
template <typename R, int NB>
__device__ void panel_apply_t(const cplx<R>* T, int pb, bool herm, cplx<R>* Ws, int ldw, int nc) {
  for (int c = threadIdx.x; c < nc; c += NT) {
    cplx<R> w[NB], y[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) w[i] = (i < pb) ? Ws[i * ldw + c] : mk<R>(0, 0);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      cplx<R> acc = mk<R>(0, 0);
      if (herm) {
#pragma unroll
        for (int k = 0; k <= i; ++k) cfma_cj(acc, T[k + i * NB], w[k]);  // (T^H)[i][k] = conj(T[k][i])
      } else {
#pragma unroll
        for (int k = i; k < NB; ++k) cfma(acc, T[i + k * NB], w[k]);
      }
      y[i] = acc;
    }
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i < pb) Ws[i * ldw + c] = y[i];
  }
}

}  // namespace panel
}  // namespace mpdo
