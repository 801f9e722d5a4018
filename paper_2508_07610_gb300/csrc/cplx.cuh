// Complex arithmetic, strided tensor views and launch helpers shared by the sm_103a kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bounds.cuh"

namespace mpdo {

template <typename R>
struct cplx {
  R x, y;
};

template <typename R>
__host__ __device__ __forceinline__ cplx<R> mk(R a, R b) {
  cplx<R> c;
  c.x = a;
  c.y = b;
  return c;
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator*(R s, cplx<R> a) { return mk(s * a.x, s * a.y); }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> conjg(cplx<R> a) { return mk(a.x, -a.y); }
template <typename R>
__host__ __device__ __forceinline__ R norm2(cplx<R> a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void cfma(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ void cfma_cj(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// acc -= a * b and acc -= a * conj(b), four fused multiply-adds each (the operator form costs two
// multiplications, two fused multiply-adds and two additions)
template <typename R>
__host__ __device__ __forceinline__ void cfms(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
template <typename R>
__host__ __device__ __forceinline__ void cfms_cj(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(-a.y, b.x, acc.y);
  acc.y = fma(a.x, b.y, acc.y);
}

// Norms below this are treated as exact zeros by the Householder steps, so that 1 / (|x| (|x| + |a|))
// cannot overflow (its square stays far above the smallest normal number).
template <typename R>
__host__ __device__ __forceinline__ R tiny_norm();
template <>
__host__ __device__ __forceinline__ float tiny_norm<float>() { return 1e-17f; }
template <>
__host__ __device__ __forceinline__ double tiny_norm<double>() { return 1e-140; }

// A 2-D view of a strided tensor.  Logical (row i, col j) of batch item z lives at
//   off(z) + (i / rdiv) * rhi + (i % rdiv) * rlo + (j / cdiv) * chi + (j % cdiv) * clo
// where off(z) = (z / bdiv) * bhi + (z % bdiv) * blo.  A divisor of 0 means "no split"
// (the index uses the lo stride only), which keeps plain row/column-major views cheap.
struct View {
  int64_t bhi, blo;
  int64_t rhi, rlo, chi, clo;
  int32_t bdiv, rdiv, cdiv;
  int32_t conj;
};

__host__ __device__ __forceinline__ int64_t split_off(int64_t i, int32_t d, int64_t hi, int64_t lo) {
  if (d == 0) return i * lo;
  int64_t q = i / d;
  return q * hi + (i - q * d) * lo;
}
__host__ __device__ __forceinline__ int64_t view_batch(const View& v, int64_t z) { return split_off(z, v.bdiv, v.bhi, v.blo); }
__host__ __device__ __forceinline__ int64_t view_row(const View& v, int64_t i) { return split_off(i, v.rdiv, v.rhi, v.rlo); }
__host__ __device__ __forceinline__ int64_t view_col(const View& v, int64_t j) { return split_off(j, v.cdiv, v.chi, v.clo); }

// Plain views.
inline View row_major(int64_t ld, int64_t bstride) {
  View v{};
  v.blo = bstride;
  v.rlo = ld;
  v.clo = 1;
  return v;
}
inline View col_major(int64_t ld, int64_t bstride) {
  View v{};
  v.blo = bstride;
  v.rlo = 1;
  v.clo = ld;
  return v;
}
inline View conj_of(View v) {
  v.conj ^= 1;
  return v;
}
// transpose: swap the row and column maps
inline View transpose(View v) {
  View t = v;
  t.rhi = v.chi; t.rlo = v.clo; t.rdiv = v.cdiv;
  t.chi = v.rhi; t.clo = v.rlo; t.cdiv = v.rdiv;
  return t;
}

}  // namespace mpdo
