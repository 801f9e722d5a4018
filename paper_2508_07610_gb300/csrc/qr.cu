// Batched complex Householder QR (CUDA cores, FP32 or FP64 complex) in three variants chosen per
// launch: a blocked one-CTA-per-matrix kernel (compact-WY panels in shared memory) for batches that
// fill the GPU, a thread-block-cluster kernel that spreads one matrix over 2-8 CTAs for small batches,
// and a plain one-CTA-per-matrix kernel when neither fits.
//
// Used to keep the chain in canonical form (QR sweeps, Sec. II.D / Fig. 3b) and to reduce the
// left site of a two-site update to its (p, bond) block.  For an m x n input (read through a
// View, optionally conjugated) it leaves R (x x n, x = min(m, n), upper trapezoidal, zeros below)
// in the column-major work matrix W (ld = m) and writes the thin Q (m x x, orthonormal columns)
// both to the column-major buffer Qw (ld = m) and, when given, through an output View.
// Reflectors are H = I - beta v v^H with v = y + e^{i arg y0} |y| e_0, so H y = -e^{i arg y0} |y| e_0.
#include <cooperative_groups.h>

#include "device_once.cuh"
#include "kernels.h"
#include "panel.cuh"

namespace cg = cooperative_groups;

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
    cplx<R> v = GX(in, view_row(g.vin, i) + view_col(g.vin, j));
    if (g.vin.conj) v.y = -v.y;
    GX(W, e) = v;
  }
  __syncthreads();

  for (int j = 0; j < x; ++j) {
    cplx<R>* col = W + (int64_t)j * m;
    R s = 0;
    for (int i = j + 1 + tid; i < m; i += NT) s += norm2(GX(col, i));
    s = block_sum(s, red);
    const cplx<R> a = GX(col, j);
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
        if (lane == 0) cfma_cj(acc, v0, GX(y, j));
        for (int i = j + 1 + lane; i < m; i += 32) cfma_cj(acc, GX(col, i), GX(y, i));
        acc = warp_csum(acc);
        acc = beta * acc;
        if (lane == 0) GX(y, j) = GX(y, j) - v0 * acc;
        for (int i = j + 1 + lane; i < m; i += 32) GX(y, i) = GX(y, i) - GX(col, i) * acc;
      }
    }
    __syncthreads();
    if (tid == 0) GX(col, j) = (beta != R(0)) ? mk<R>(-nrm * ph.x, -nrm * ph.y) : a;
    __syncthreads();
  }

  // Q = H_0 H_1 ... H_{x-1} [I; 0]: apply the reflectors to the identity columns, last first.
  for (int64_t e = tid; e < (int64_t)m * x; e += NT) {
    int i = (int)(e % m), c = (int)(e / m);
    GX(Q, e) = mk<R>(i == c ? R(1) : R(0), R(0));
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
      if (lane == 0) cfma_cj(acc, v0, GX(y, j));
      for (int i = j + 1 + lane; i < m; i += 32) cfma_cj(acc, GX(col, i), GX(y, i));
      acc = warp_csum(acc);
      acc = beta * acc;
      if (lane == 0) GX(y, j) = GX(y, j) - v0 * acc;
      for (int i = j + 1 + lane; i < m; i += 32) GX(y, i) = GX(y, i) - GX(col, i) * acc;
    }
    __syncthreads();
  }
  // R: clear the reflectors below the diagonal of the leading x rows.
  for (int64_t e = tid; e < (int64_t)x * x; e += NT) {
    int i = (int)(e % x), j = (int)(e / x);
    if (i > j) GX(W, (int64_t)j * m + i) = mk<R>(0, 0);
  }
  if (g.qout) {
    cplx<R>* out = g.qout + view_batch(g.vq, z);
    for (int64_t e = tid; e < (int64_t)m * x; e += NT) {
      int i = (int)(e % m), c = (int)(e / m);
      cplx<R> v = GX(Q, e);
      if (g.vq.conj) v.y = -v.y;
      GX(out, view_row(g.vq, i) + view_col(g.vq, c)) = v;
    }
  }
}
// ---------------------------------------------------------------------------------------------
// Cluster variant: the C CTAs of a thread-block cluster hold the m x n matrix in their shared memory,
// ceil(m / C) rows each, so every pass over the trailing matrix runs from on-chip memory.  Column
// norms and the reflector-column dot products are reduced across the cluster through distributed
// shared memory (two alternating partial buffers, one cluster barrier per reduction).  Q is formed in
// place after R has been written out.  Every loop has a fixed trip count shared by the whole cluster.
template <typename R>
__global__ void __launch_bounds__(NT) qr_cluster_kernel(QrArgs<R> g, int C, int mloc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int z = blockIdx.x / C;
  const int m = g.m, n = g.n, x = (m < n) ? m : n;
  const int r0 = rank * mloc;
  const int r1 = (r0 + mloc < m) ? r0 + mloc : m;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  cplx<R>* Wl = reinterpret_cast<cplx<R>*>(smem_raw);        // [n][mloc] column-major
  cplx<R>* red = Wl + (int64_t)mloc * n;                       // 2 x (n + 2) partials
  cplx<R>* wv = red + 2 * (n + 2);                              // n gathered values
  cplx<R>* s_v0 = wv + n;                                       // n
  R* s_beta = reinterpret_cast<R*>(s_v0 + n);                   // n
  R* bred = s_beta + n;                                         // NT / 32
  cplx<R>* W = g.W + (int64_t)z * g.wstride;
  cplx<R>* Qg = g.Qw + (int64_t)z * g.qstride;
  const cplx<R>* in = g.in + view_batch(g.vin, z);

  for (int64_t e = tid; e < (int64_t)mloc * n; e += NT) {
    int il = (int)(e % mloc), j = (int)(e / mloc);
    int i = r0 + il;
    cplx<R> v = mk<R>(0, 0);
    if (i < r1) {
      v = GX(in, view_row(g.vin, i) + view_col(g.vin, j));
      if (g.vin.conj) v.y = -v.y;
    }
    Wl[e] = v;
  }
  __syncthreads();

  int buf = 0;
  // gather slot `slot` (count values) of buffer `b` from every CTA into wv, summed in rank order
  auto gather = [&](int b, int count) {
    for (int c = tid; c < count; c += NT) {
      cplx<R> acc = mk<R>(0, 0);
      for (int r = 0; r < C; ++r) {
        cplx<R>* rem = cluster.map_shared_rank(red + b * (n + 2), r);
        acc = acc + rem[c];
      }
      wv[c] = acc;
    }
    __syncthreads();
  };

  for (int j = 0; j < x; ++j) {
    const cplx<R>* col = Wl + (int64_t)j * mloc;
    // partial |column j below j|^2 and the diagonal entry (from its owner)
    R s = 0;
    for (int i = (j + 1 > r0 ? j + 1 : r0) + tid; i < r1; i += NT) s += norm2(col[i - r0]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) bred[wid] = s;
    __syncthreads();
    if (tid == 0) {
      R t = 0;
      for (int w = 0; w < NT / 32; ++w) t += bred[w];
      red[buf * (n + 2) + 0] = mk<R>(t, 0);
      red[buf * (n + 2) + 1] = (j >= r0 && j < r1) ? col[j - r0] : mk<R>(0, 0);
    }
    cluster.sync();
    gather(buf, 2);
    buf ^= 1;
    const cplx<R> a = wv[1];
    const R aa = sqrt(norm2(a));
    const R nrm = sqrt(aa * aa + wv[0].x);
    const cplx<R> ph = (aa > R(0)) ? mk<R>(a.x / aa, a.y / aa) : mk<R>(1, 0);
    const R beta = (nrm > tiny_norm<R>()) ? R(1) / (nrm * (nrm + aa)) : R(0);
    const cplx<R> v0 = a + nrm * ph;
    if (beta != R(0)) {
      // partial w_c = v^H W[:, c] over my rows, one warp per column
      for (int c = j + 1 + wid; c < n; c += NT / 32) {
        const cplx<R>* y = Wl + (int64_t)c * mloc;
        cplx<R> acc = mk<R>(0, 0);
        if (lane == 0 && j >= r0 && j < r1) cfma_cj(acc, v0, y[j - r0]);
        for (int i = (j + 1 > r0 ? j + 1 : r0) + lane; i < r1; i += 32) cfma_cj(acc, col[i - r0], y[i - r0]);
        acc = warp_csum(acc);
        if (lane == 0) red[buf * (n + 2) + c] = acc;
      }
    }
    cluster.sync();  // taken whether or not beta vanished, so every CTA passes the same barriers
    if (beta != R(0)) {
      for (int c = tid; c < n; c += NT) {
        cplx<R> acc = mk<R>(0, 0);
        if (c > j)
          for (int r = 0; r < C; ++r) acc = acc + cluster.map_shared_rank(red + buf * (n + 2), r)[c];
        wv[c] = beta * acc;
      }
      __syncthreads();
      for (int64_t e = tid; e < (int64_t)(n - j - 1) * mloc; e += NT) {
        int il = (int)(e % mloc), c = j + 1 + (int)(e / mloc);
        int i = r0 + il;
        if (i < j || i >= r1) continue;
        cplx<R> vi = (i == j) ? v0 : col[il];
        Wl[(int64_t)c * mloc + il] = Wl[(int64_t)c * mloc + il] - vi * wv[c];
      }
    }
    buf ^= 1;
    __syncthreads();
    if (tid == 0) {
      s_beta[j] = beta;
      s_v0[j] = v0;
      if (j >= r0 && j < r1) Wl[(int64_t)j * mloc + (j - r0)] = (beta != R(0)) ? mk<R>(-nrm * ph.x, -nrm * ph.y) : a;
    }
    __syncthreads();
  }

  // R (leading x rows, zeros below the diagonal) to the global work matrix
  for (int64_t e = tid; e < (int64_t)mloc * n; e += NT) {
    int il = (int)(e % mloc), c = (int)(e / mloc);
    int i = r0 + il;
    if (i < r1 && i < x) GX(W, (int64_t)c * m + i) = (c >= i) ? Wl[e] : mk<R>(0, 0);
  }
  __syncthreads();
  // Q in place: clear the strict upper triangle of the leading x columns, then apply the reflectors
  for (int64_t e = tid; e < (int64_t)mloc * x; e += NT) {
    int il = (int)(e % mloc), c = (int)(e / mloc);
    if (r0 + il < c) Wl[e] = mk<R>(0, 0);
  }
  __syncthreads();
  for (int j = x - 1; j >= 0; --j) {
    const R beta = s_beta[j];
    const cplx<R> v0 = s_v0[j];
    const cplx<R>* col = Wl + (int64_t)j * mloc;
    if (beta != R(0)) {
      for (int c = j + 1 + wid; c < x; c += NT / 32) {
        const cplx<R>* y = Wl + (int64_t)c * mloc;
        cplx<R> acc = mk<R>(0, 0);
        if (lane == 0 && j >= r0 && j < r1) cfma_cj(acc, v0, y[j - r0]);
        for (int i = (j + 1 > r0 ? j + 1 : r0) + lane; i < r1; i += 32) cfma_cj(acc, col[i - r0], y[i - r0]);
        acc = warp_csum(acc);
        if (lane == 0) red[buf * (n + 2) + c] = acc;
      }
    }
    cluster.sync();
    if (beta != R(0)) {
      for (int c = tid; c < x; c += NT) {
        cplx<R> acc = mk<R>(0, 0);
        if (c > j)
          for (int r = 0; r < C; ++r) acc = acc + cluster.map_shared_rank(red + buf * (n + 2), r)[c];
        wv[c] = beta * acc;
      }
      __syncthreads();
      for (int64_t e = tid; e < (int64_t)(x - j - 1) * mloc; e += NT) {
        int il = (int)(e % mloc), c = j + 1 + (int)(e / mloc);
        int i = r0 + il;
        if (i < j || i >= r1) continue;
        cplx<R> vi = (i == j) ? v0 : col[il];
        Wl[(int64_t)c * mloc + il] = Wl[(int64_t)c * mloc + il] - vi * wv[c];
      }
      __syncthreads();
    }
    // column j of Q: e_j - beta v conj(v0) on rows >= j, zero above
    for (int il = tid; il < mloc; il += NT) {
      int i = r0 + il;
      if (i >= r1) continue;
      cplx<R> q = mk<R>(0, 0);
      if (i >= j) {
        cplx<R> vi = (i == j) ? v0 : Wl[(int64_t)j * mloc + il];
        q = mk<R>(i == j ? R(1) : R(0), R(0)) - beta * (vi * conjg(v0));
      }
      Wl[(int64_t)j * mloc + il] = q;
    }
    buf ^= 1;
    __syncthreads();
  }
  // Q out: the column-major work buffer and, when given, the output view
  cplx<R>* out = g.qout ? g.qout + view_batch(g.vq, z) : nullptr;
  for (int64_t e = tid; e < (int64_t)mloc * x; e += NT) {
    int il = (int)(e % mloc), c = (int)(e / mloc);
    int i = r0 + il;
    if (i >= r1) continue;
    cplx<R> v = Wl[e];
    GX(Qg, (int64_t)c * m + i) = v;
    if (out) {
      if (g.vq.conj) v.y = -v.y;
      GX(out, view_row(g.vq, i) + view_col(g.vq, c)) = v;
    }
  }
  cluster.sync();  // no CTA leaves while a peer may still read its shared memory
}

// ---------------------------------------------------------------------------------------------
// Blocked variant (throughput path for many matrices): reflectors are generated NB columns at a
// time on a panel held in shared memory and applied to the rest of the matrix as one block reflector
// I - V T V^H (compact WY form: T upper triangular with T_jj = beta_j and
// T[0:j, j] = -beta_j T[0:j, 0:j] V[:, 0:j]^H v_j), so every pass over the trailing columns serves NB
// reflectors instead of one and runs as two small matrix products with V in shared memory.  Q is
// accumulated the same way, panels last to first.
//
template <typename R, int NB>
size_t blocked_smem_bytes(int m, int n) {
  const int x = m < n ? m : n;
  const int npan = (x + NB - 1) / NB;
  return sizeof(cplx<R>) * ((size_t)NB * m + (size_t)npan * NB * NB + (size_t)NB * n + x) +
         sizeof(R) * ((size_t)x + NT / 32);
}

template <typename R, int NB>
__global__ void __launch_bounds__(NT) qr_blocked_kernel(QrArgs<R> g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int z = blockIdx.x;
  const int m = g.m, n = g.n, x = (m < n) ? m : n;
  const int npan = (x + NB - 1) / NB;
  cplx<R>* Vs = reinterpret_cast<cplx<R>*>(smem_raw);  // NB panel columns, ld m (rows relative to p0)
  cplx<R>* Ts = Vs + (size_t)NB * m;                    // T of every panel, NB x NB column-major
  cplx<R>* Ws = Ts + (size_t)npan * NB * NB;            // NB x n products (row i at Ws + i * n)
  cplx<R>* s_v0 = Ws + (size_t)NB * n;                  // x reflector heads
  R* s_beta = reinterpret_cast<R*>(s_v0 + x);           // x
  R* red = s_beta + x;                                  // NT / 32
  cplx<R>* W = g.W + (int64_t)z * g.wstride;
  cplx<R>* Q = g.Qw + (int64_t)z * g.qstride;
  const cplx<R>* in = g.in + view_batch(g.vin, z);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  for (int64_t e = tid; e < (int64_t)m * n; e += NT) {
    int i = (int)(e % m), j = (int)(e / m);
    cplx<R> v = GX(in, view_row(g.vin, i) + view_col(g.vin, j));
    if (g.vin.conj) v.y = -v.y;
    GX(W, e) = v;
  }
  __syncthreads();

  for (int P = 0; P < npan; ++P) {
    const int p0 = P * NB, pb = (x - p0 < NB) ? x - p0 : NB, M = m - p0;
    for (int e = tid; e < pb * M; e += NT) {
      int i = e / M, r = e % M;
      Vs[i * m + r] = GX(W, (int64_t)(p0 + i) * m + p0 + r);
    }
    __syncthreads();
    // factor the panel in shared memory
    for (int jj = 0; jj < pb; ++jj) {
      cplx<R>* col = Vs + jj * m;
      R s = 0;
      for (int r = jj + 1 + tid; r < M; r += NT) s += norm2(col[r]);
      s = block_sum(s, red);
      const cplx<R> a = col[jj];
      const R aa = sqrt(norm2(a));
      const R nrm = sqrt(aa * aa + s);
      const cplx<R> ph = (aa > R(0)) ? mk<R>(a.x / aa, a.y / aa) : mk<R>(1, 0);
      const R beta = (nrm > tiny_norm<R>()) ? R(1) / (nrm * (nrm + aa)) : R(0);
      const cplx<R> v0 = a + nrm * ph;
      if (beta != R(0)) {
        for (int c = jj + 1 + wid; c < pb; c += NT / 32) {
          cplx<R>* y = Vs + c * m;
          cplx<R> acc = mk<R>(0, 0);
          if (lane == 0) cfma_cj(acc, v0, y[jj]);
          for (int r = jj + 1 + lane; r < M; r += 32) cfma_cj(acc, col[r], y[r]);
          acc = warp_csum(acc);
          acc = beta * acc;
          if (lane == 0) y[jj] = y[jj] - v0 * acc;
          for (int r = jj + 1 + lane; r < M; r += 32) y[r] = y[r] - col[r] * acc;
        }
      }
      __syncthreads();
      // column p0 + jj: R entries (rows p0 .. p0 + jj) and the reflector below go back to W; the
      // shared copy becomes the full reflector (zeros above, v0 on the diagonal)
      cplx<R>* wc = W + (int64_t)(p0 + jj) * m + p0;
      for (int r = tid; r < M; r += NT) {
        if (r < jj) {
          GX(wc, r) = col[r];
          col[r] = mk<R>(0, 0);
        } else if (r > jj) {
          GX(wc, r) = col[r];
        }
      }
      if (tid == 0) {
        GX(wc, jj) = (beta != R(0)) ? mk<R>(-nrm * ph.x, -nrm * ph.y) : a;
        col[jj] = v0;
        s_beta[p0 + jj] = beta;
        s_v0[p0 + jj] = v0;
      }
      __syncthreads();
    }
    // T of the panel: S[i][k] = v_i^H v_k (i < k; v_k vanishes above row k), then the recurrence
    cplx<R>* T = Ts + (size_t)P * NB * NB;
    cplx<R>* S = Ws;  // NB x NB scratch, S[i * NB + k]
    for (int pr = wid; pr < pb * pb; pr += NT / 32) {
      const int i = pr / pb, k = pr % pb;
      if (i >= k) continue;
      cplx<R> acc = mk<R>(0, 0);
      for (int r = k + lane; r < M; r += 32) cfma_cj(acc, Vs[i * m + r], Vs[k * m + r]);
      acc = warp_csum(acc);
      if (lane == 0) S[i * NB + k] = acc;
    }
    __syncthreads();
    for (int k = 0; k < NB; ++k) {
      if (tid < NB) {
        const int i = tid;
        cplx<R> t = mk<R>(0, 0);
        if (k < pb && i < k) {
          cplx<R> acc = mk<R>(0, 0);
          for (int l = i; l < k; ++l) cfma(acc, T[i + l * NB], S[l * NB + k]);
          t = -s_beta[p0 + k] * acc;
        } else if (k < pb && i == k) {
          t = mk<R>(s_beta[p0 + k], 0);
        }
        T[i + k * NB] = t;
      }
      __syncthreads();
    }
    // trailing columns: A <- (I - V T^H V^H) A on rows p0.., columns p0 + pb ..
    const int nc = n - p0 - pb;
    if (nc > 0) {
      cplx<R>* A = W + (int64_t)(p0 + pb) * m + p0;
      panel::panel_vh_times<R, NB>(A, m, M, nc, Vs, m, pb, Ws, n);
      __syncthreads();
      panel::panel_apply_t<R, NB>(T, pb, true, Ws, n, nc);
      __syncthreads();
      panel::panel_minus_v_times<R, NB>(A, m, M, nc, Vs, m, pb, Ws, n);
      __syncthreads();
    }
  }

  // Q = H_0 H_1 ... H_{x-1} [I; 0], one block reflector I - V T V^H per panel, last panel first
  for (int64_t e = tid; e < (int64_t)m * x; e += NT) {
    int i = (int)(e % m), c = (int)(e / m);
    GX(Q, e) = mk<R>(i == c ? R(1) : R(0), R(0));
  }
  __syncthreads();
  for (int P = npan - 1; P >= 0; --P) {
    const int p0 = P * NB, pb = (x - p0 < NB) ? x - p0 : NB, M = m - p0;
    for (int e = tid; e < pb * M; e += NT) {
      int i = e / M, r = e % M;
      cplx<R> v = mk<R>(0, 0);
      if (r == i) v = s_v0[p0 + i];
      else if (r > i) v = GX(W, (int64_t)(p0 + i) * m + p0 + r);
      Vs[i * m + r] = v;
    }
    __syncthreads();
    const int nc = x - p0;
    cplx<R>* A = Q + (int64_t)p0 * m + p0;
    panel::panel_vh_times<R, NB>(A, m, M, nc, Vs, m, pb, Ws, n);
    __syncthreads();
    panel::panel_apply_t<R, NB>(Ts + (size_t)P * NB * NB, pb, false, Ws, n, nc);
    __syncthreads();
    panel::panel_minus_v_times<R, NB>(A, m, M, nc, Vs, m, pb, Ws, n);
    __syncthreads();
  }
  // R: clear the reflectors below the diagonal of the leading x rows.
  for (int64_t e = tid; e < (int64_t)x * x; e += NT) {
    int i = (int)(e % x), j = (int)(e / x);
    if (i > j) GX(W, (int64_t)j * m + i) = mk<R>(0, 0);
  }
  if (g.qout) {
    cplx<R>* out = g.qout + view_batch(g.vq, z);
    for (int64_t e = tid; e < (int64_t)m * x; e += NT) {
      int i = (int)(e % m), c = (int)(e / m);
      cplx<R> v = GX(Q, e);
      if (g.vq.conj) v.y = -v.y;
      GX(out, view_row(g.vq, i) + view_col(g.vq, c)) = v;
    }
  }
}

template <typename R, int NB>
cudaError_t launch_blocked(cudaStream_t s, int batch, const QrArgs<R>& g, size_t bytes) {
  static PerDevice setup;
  cudaError_t e = setup.once([](int) {
    return cudaFuncSetAttribute(qr_blocked_kernel<R, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (e != cudaSuccess) return e;
  qr_blocked_kernel<R, NB><<<batch, NT, bytes, s>>>(g);
  return cudaGetLastError();
}

template <typename R>
size_t cluster_smem_bytes(int mloc, int n) {
  return sizeof(cplx<R>) * ((size_t)mloc * n + 2 * (n + 2) + 2 * (size_t)n) + sizeof(R) * ((size_t)n + NT / 32) + 64;
}
constexpr size_t kClusterSmemBudget = 200 * 1024;
}  // namespace

template <typename R>
cudaError_t qr(cudaStream_t s, int batch, const QrArgs<R>& g) {
  if (batch <= 0 || g.m <= 0 || g.n <= 0) return cudaSuccess;
  int x = g.m < g.n ? g.m : g.n;
  if (x > MAXX) return cudaErrorInvalidValue;
  // Few matrices (latency-bound): the smallest cluster (2, 4 or 8 CTAs) whose shared memory holds the
  // matrix.  Many matrices (throughput-bound): one CTA per matrix, which keeps every SM busy with
  // several small-footprint CTAs and spends fewer SM-cycles per factorisation.
  const int n_sm = sm_count();
  for (int C = 2; C <= 8; C *= 2) {
    int mloc = (g.m + C - 1) / C;
    size_t bytes = cluster_smem_bytes<R>(mloc, g.n);
    if (bytes > kClusterSmemBudget || g.m < 2 * C) continue;
    if ((int64_t)batch * C > n_sm) break;
    static PerDevice setup;
    cudaError_t ea = setup.once([](int) {
      return cudaFuncSetAttribute(qr_cluster_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kClusterSmemBudget);
    });
    if (ea != cudaSuccess) return ea;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(batch * C));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, qr_cluster_kernel<R>, g, C, mloc);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  // many matrices: the blocked kernel with the widest panel that still lets two CTAs share an SM,
  // else the widest panel that fits at all
  constexpr size_t kBlockedBudget = 200 * 1024, kTwoPerSm = 110 * 1024;
  constexpr int NB1 = 8, NB2 = 4;  // measured: 8-column panels beat 16 for both QR shapes of the update
  const size_t b1 = blocked_smem_bytes<R, NB1>(g.m, g.n), b2 = blocked_smem_bytes<R, NB2>(g.m, g.n);
  if (b1 <= kTwoPerSm) return launch_blocked<R, NB1>(s, batch, g, b1);
  if (b2 <= kTwoPerSm) return launch_blocked<R, NB2>(s, batch, g, b2);
  if (b1 <= kBlockedBudget) return launch_blocked<R, NB1>(s, batch, g, b1);
  if (b2 <= kBlockedBudget) return launch_blocked<R, NB2>(s, batch, g, b2);
  qr_kernel<R><<<batch, NT, 0, s>>>(g);
  return cudaGetLastError();
}

template cudaError_t qr<float>(cudaStream_t, int, const QrArgs<float>&);
template cudaError_t qr<double>(cudaStream_t, int, const QrArgs<double>&);

}  // namespace mpdo
