// Batched complex Householder QR, one CTA per matrix (CUDA cores, FP32 or FP64 complex).
//
// Used to keep the chain in canonical form (QR sweeps, Sec. II.D / Fig. 3b) and to reduce the
// left site of a two-site update to its (p, bond) block.  For an m x n input (read through a
// View, optionally conjugated) it leaves R (x x n, x = min(m, n), upper trapezoidal, zeros below)
// in the column-major work matrix W (ld = m) and writes the thin Q (m x x, orthonormal columns)
// both to the column-major buffer Qw (ld = m) and, when given, through an output View.
// Reflectors are H = I - beta v v^H with v = y + e^{i arg y0} |y| e_0, so H y = -e^{i arg y0} |y| e_0.
#include "kernels.h"

namespace mpdo {

namespace {
constexpr int NT = 256;
constexpr int MAXX = 1024;

template <typename R>
__device__ R block_sum(R v, R* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  R s = 0;
  for (int w = 0; w < NT / 32; ++w) s += red[w];
  return s;
}

template <typename R>
__device__ cplx<R> warp_csum(cplx<R> v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

template <typename R>
__global__ void __launch_bounds__(NT) qr_kernel(QrArgs<R> g) {
  __shared__ R red[NT / 32];
  __shared__ R s_beta[MAXX];
  __shared__ cplx<R> s_v0[MAXX];
  const int z = blockIdx.x;
  const int m = g.m, n = g.n, x = (m < n) ? m : n;
  cplx<R>* W = g.W + (int64_t)z * g.wstride;
  cplx<R>* Q = g.Qw + (int64_t)z * g.qstride;
  const cplx<R>* in = g.in + view_batch(g.vin, z);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  for (int64_t e = tid; e < (int64_t)m * n; e += NT) {
    int i = (int)(e % m), j = (int)(e / m);
    cplx<R> v = in[view_row(g.vin, i) + view_col(g.vin, j)];
    if (g.vin.conj) v.y = -v.y;
    W[e] = v;
  }
  __syncthreads();

  for (int j = 0; j < x; ++j) {
    cplx<R>* col = W + (int64_t)j * m;
    R s = 0;
    for (int i = j + 1 + tid; i < m; i += NT) s += norm2(col[i]);
    s = block_sum(s, red);
    const cplx<R> a = col[j];
    const R aa = sqrt(norm2(a));
    const R nrm = sqrt(aa * aa + s);
    cplx<R> ph = (aa > R(0)) ? mk<R>(a.x / aa, a.y / aa) : mk<R>(1, 0);
    const R beta = (nrm > tiny_norm<R>()) ? R(1) / (nrm * (nrm + aa)) : R(0);
    const cplx<R> v0 = a + nrm * ph;
    if (tid == 0) {
      s_beta[j] = beta;
      s_v0[j] = v0;
    }
    // trailing columns: y <- y - beta v (v^H y); one warp per column
    if (beta != R(0)) {
      for (int c = j + 1 + wid; c < n; c += NT / 32) {
        cplx<R>* y = W + (int64_t)c * m;
        cplx<R> acc = mk<R>(0, 0);
        if (lane == 0) cfma_cj(acc, v0, y[j]);
        for (int i = j + 1 + lane; i < m; i += 32) cfma_cj(acc, col[i], y[i]);
        acc = warp_csum(acc);
        acc = beta * acc;
        if (lane == 0) y[j] = y[j] - v0 * acc;
        for (int i = j + 1 + lane; i < m; i += 32) y[i] = y[i] - col[i] * acc;
      }
    }
    __syncthreads();
    if (tid == 0) col[j] = (beta != R(0)) ? mk<R>(-nrm * ph.x, -nrm * ph.y) : a;
    __syncthreads();
  }

  // Q = H_0 H_1 ... H_{x-1} [I; 0]: apply the reflectors to the identity columns, last first.
  for (int64_t e = tid; e < (int64_t)m * x; e += NT) {
    int i = (int)(e % m), c = (int)(e / m);
    Q[e] = mk<R>(i == c ? R(1) : R(0), R(0));
  }
  __syncthreads();
  for (int j = x - 1; j >= 0; --j) {
    const R beta = s_beta[j];
    if (beta == R(0)) continue;
    const cplx<R> v0 = s_v0[j];
    const cplx<R>* col = W + (int64_t)j * m;
    for (int c = j + wid; c < x; c += NT / 32) {
      cplx<R>* y = Q + (int64_t)c * m;
      cplx<R> acc = mk<R>(0, 0);
      if (lane == 0) cfma_cj(acc, v0, y[j]);
      for (int i = j + 1 + lane; i < m; i += 32) cfma_cj(acc, col[i], y[i]);
      acc = warp_csum(acc);
      acc = beta * acc;
      if (lane == 0) y[j] = y[j] - v0 * acc;
      for (int i = j + 1 + lane; i < m; i += 32) y[i] = y[i] - col[i] * acc;
    }
    __syncthreads();
  }
  // R: clear the reflectors below the diagonal of the leading x rows.
  for (int64_t e = tid; e < (int64_t)x * x; e += NT) {
    int i = (int)(e % x), j = (int)(e / x);
    if (i > j) W[(int64_t)j * m + i] = mk<R>(0, 0);
  }
  if (g.qout) {
    cplx<R>* out = g.qout + view_batch(g.vq, z);
    for (int64_t e = tid; e < (int64_t)m * x; e += NT) {
      int i = (int)(e % m), c = (int)(e / m);
      cplx<R> v = Q[e];
      if (g.vq.conj) v.y = -v.y;
      out[view_row(g.vq, i) + view_col(g.vq, c)] = v;
    }
  }
}
}  // namespace

template <typename R>
cudaError_t qr(cudaStream_t s, int batch, const QrArgs<R>& g) {
  if (batch <= 0 || g.m <= 0 || g.n <= 0) return cudaSuccess;
  int x = g.m < g.n ? g.m : g.n;
  if (x > MAXX) return cudaErrorInvalidValue;
  qr_kernel<R><<<batch, NT, 0, s>>>(g);
  return cudaGetLastError();
}

template cudaError_t qr<float>(cudaStream_t, int, const QrArgs<float>&);
template cudaError_t qr<double>(cudaStream_t, int, const QrArgs<double>&);

}  // namespace mpdo
