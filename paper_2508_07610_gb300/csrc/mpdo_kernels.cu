// MPDO-specific kernels: chi -> Choi -> Kraus (Sec. III), noisy-gate fusion K_i = N_i U (Sec. II.C),
// the single-qubit noisy-gate contraction with its new Kraus leg (Fig. 2c), the small tensors of the
// two-site split, and helpers for readouts.  All batched over independent instances.
#include "kernels.h"

namespace mpdo {

namespace {
constexpr int NT = 256;

__device__ __forceinline__ cplx<double> pauli1(int m, int i, int j) {
  // I, X, Y, Z
  if (m == 0) return mk<double>(i == j ? 1.0 : 0.0, 0.0);
  if (m == 1) return mk<double>(i != j ? 1.0 : 0.0, 0.0);
  if (m == 2) {
    if (i == j) return mk<double>(0.0, 0.0);
    return mk<double>(0.0, i == 0 ? -1.0 : 1.0);  // [[0, -i], [i, 0]]
  }
  return mk<double>(i == j ? (i == 0 ? 1.0 : -1.0) : 0.0, 0.0);
}
// element (i, j) of the Pauli string with index m (first qubit most significant)
__device__ cplx<double> pauli_elem(int nq, int m, int i, int j) {
  cplx<double> v = mk<double>(1.0, 0.0);
  for (int q = 0; q < nq; ++q) {
    int sh = nq - 1 - q;
    v = v * pauli1((m >> (2 * sh)) & 3, (i >> sh) & 1, (j >> sh) & 1);
  }
  return v;
}

__global__ void chi_to_choi_kernel(int count, int nq, const cplx<double>* chi, cplx<double>* choi) {
  const int d = 1 << nq, d2 = d * d;
  const int c = blockIdx.x;
  if (c >= count) return;
  const cplx<double>* X = chi + (int64_t)c * d2 * d2;
  cplx<double>* L = choi + (int64_t)c * d2 * d2;
  for (int e = threadIdx.x; e < d2 * d2; e += blockDim.x) {
    int a = e % d2, b = e / d2;  // column-major L[a + b d2]
    int ai = a / d, aj = a % d, bi = b / d, bj = b % d;
    cplx<double> acc = mk<double>(0, 0);
    for (int m = 0; m < d2; ++m) {
      cplx<double> sm = pauli_elem(nq, m, ai, aj);
      if (sm.x == 0.0 && sm.y == 0.0) continue;
      for (int n = 0; n < d2; ++n) {
        cplx<double> sn = pauli_elem(nq, n, bi, bj);
        if (sn.x == 0.0 && sn.y == 0.0) continue;
        acc = acc + GX(X, m * d2 + n) * sm * conjg(sn);
      }
    }
    GX(L, e) = acc;
  }
}

__global__ void choi_to_kraus_kernel(int count, int nq, int rmax, const int* r_dev, const double* eta,
                                     const cplx<double>* vecs, cplx<double>* kraus) {
  const int d = 1 << nq, d2 = d * d;
  const int c = blockIdx.x;
  if (c >= count) return;
  const int r = GX(r_dev, c);
  for (int e = threadIdx.x; e < rmax * d2; e += blockDim.x) {
    int i = e / d2, a = e % d2;  // K_i[row][col] with a = row * d + col (row-major vec)
    cplx<double> v = mk<double>(0, 0);
    if (i < r) {
      double s = sqrt(fmax(GX(eta, (int64_t)c * d2 + i), 0.0));
      v = s * GX(vecs, (int64_t)c * d2 * d2 + a + (int64_t)i * d2);
    }
    GX(kraus, (int64_t)c * rmax * d2 + e) = v;
  }
}

__global__ void kraus_tp_kernel(int count, int nq, int rmax, const cplx<double>* kraus, double* err) {
  const int d = 1 << nq, d2 = d * d;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= count) return;
  const cplx<double>* K = kraus + (int64_t)c * rmax * d2;
  double e = 0;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      cplx<double> s = mk<double>(a == b ? -1.0 : 0.0, 0.0);
      for (int i = 0; i < rmax; ++i)
        for (int t = 0; t < d; ++t) cfma_cj(s, GX(K, i * d2 + t * d + a), GX(K, i * d2 + t * d + b));
      e = fmax(e, sqrt(norm2(s)));
    }
  GX(err, c) = e;
}

template <typename R>
__global__ void fuse_kernel(FuseArgs<R> a) {
  const int z = blockIdx.x;
  const int d = 1 << a.nq, dd = d * d;
  __shared__ cplx<double> Kh[16 * 16];
  const cplx<double>* U = a.Udev ? a.Udev + (int64_t)z * dd : a.U;
  const int ch = a.chan_idx ? GX(a.chan_idx, z) : 0;
  const cplx<double>* N = a.kraus + (int64_t)ch * a.chan_stride;
  for (int e = threadIdx.x; e < a.rk * dd; e += blockDim.x) {
    int k = e / dd, i = (e % dd) / d, j = e % d;
    cplx<double> acc = mk<double>(0, 0);
    for (int t = 0; t < d; ++t) cfma(acc, GX(N, k * dd + i * d + t), a.Udev ? GX(U, t * d + j) : U[t * d + j]);
    if (a.nq == 2) Kh[e] = acc;  // the reduced superoperator below needs the 2q operators only
    GX(a.Khat, (int64_t)z * a.rk * dd + e) = mk<R>((R)acc.x, (R)acc.y);
  }
  __syncthreads();
  if (a.nq == 2 && a.Rt) {
    // Rt[(a,b)][(p1 p2)][(q1 q2)] = sum_{p2', k} Khat_k[(a p2'), (p1 p2)] conj(Khat_k[(b p2'), (q1 q2)])
    for (int e = threadIdx.x; e < 64; e += blockDim.x) {
      int ab = e / 16, pp = (e / 4) % 4, qq = e % 4;
      int ra = ab / 2, rb = ab % 2;
      cplx<double> acc = mk<double>(0, 0);
      for (int k = 0; k < a.rk; ++k)
        for (int p2 = 0; p2 < 2; ++p2)
          cfma_cj(acc, Kh[k * 16 + (rb * 2 + p2) * 4 + qq], Kh[k * 16 + (ra * 2 + p2) * 4 + pp]);
      GX(a.Rt, (int64_t)z * 64 + e) = mk<R>((R)acc.x, (R)acc.y);
    }
  }
}

template <typename R>
__global__ void build_T_kernel(int dm, const cplx<R>* Rt, const cplx<R>* E, int64_t estride, cplx<R>* T,
                               int64_t tstride) {
  const int z = blockIdx.y;
  const int C2 = 2 * dm;
  const int64_t total = (int64_t)C2 * 2 * C2 * 2;
  const cplx<R>* Rz = Rt + (int64_t)z * 64;
  const cplx<R>* Ez = E + (int64_t)z * estride;
  cplx<R>* Tz = T + (int64_t)z * tstride;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int b = (int)(e % 2);
    int cp = (int)((e / 2) % C2);
    int a = (int)((e / (2 * C2)) % 2);
    int c = (int)(e / (4 * C2));
    int p1 = c / dm, bb = c % dm, q1 = cp / dm, bbp = cp % dm;
    cplx<R> acc = mk<R>(0, 0);
    for (int p2 = 0; p2 < 2; ++p2)
      for (int q2 = 0; q2 < 2; ++q2)
        cfma(acc, GX(Rz, (a * 2 + b) * 16 + (p1 * 2 + p2) * 4 + (q1 * 2 + q2)),
             GX(Ez, (int64_t)(bb * 2 + p2) * C2 + (bbp * 2 + q2)));
    GX(Tz, e) = acc;
  }
}

template <typename R>
__global__ void build_Y_kernel(int kchi, int dm, int rk, const cplx<R>* Khat, const cplx<R>* H, int64_t hstride,
                               cplx<R>* Y, int64_t ystride) {
  const int z = blockIdx.y;
  const int C2 = 2 * dm;
  const int64_t total = (int64_t)kchi * 2 * rk * C2;
  const cplx<R>* K = Khat + (int64_t)z * rk * 16;
  const cplx<R>* Hz = H + (int64_t)z * hstride;
  cplx<R>* Yz = Y + (int64_t)z * ystride;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int col = (int)(e % C2);
    int64_t row = e / C2;
    int k = (int)(row % rk);
    int p2p = (int)((row / rk) % 2);
    int bp = (int)(row / (2 * rk));
    int bb = col / 2, p2 = col % 2;
    cplx<R> acc = mk<R>(0, 0);
    for (int p1p = 0; p1p < 2; ++p1p)
      for (int p1 = 0; p1 < 2; ++p1)
        cfma(acc, GX(K, k * 16 + (p1p * 2 + p2p) * 4 + (p1 * 2 + p2)), GX(Hz, (int64_t)(bp * 2 + p1p) * C2 + (p1 * dm + bb)));
    GX(Yz, e) = acc;
  }
}

template <typename R>
__global__ void gate3_kernel(int X, int dn2, int dn3, int dr, int rk, const cplx<R>* Khat, const cplx<R>* T0,
                             int64_t t0stride, cplx<R>* T, int64_t tstride) {
  const int z = blockIdx.y;
  const cplx<R>* K = Khat + (int64_t)z * rk * 64;
  const cplx<R>* Tz0 = T0 + (int64_t)z * t0stride;
  cplx<R>* Tz = T + (int64_t)z * tstride;
  const int64_t total = (int64_t)X * 4 * dn2 * rk * dn3 * 2 * dr;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = e;
    const int r = (int)(t % dr);
    t /= dr;
    const int a3 = (int)(t % 2);
    t /= 2;
    const int n3 = (int)(t % dn3);
    t /= dn3;
    const int k = (int)(t % rk);
    t /= rk;
    const int n2 = (int)(t % dn2);
    t /= dn2;
    const int a2 = (int)(t % 2);
    t /= 2;
    const int a1 = (int)(t % 2);
    const int64_t x = t / 2;
    const cplx<R>* Kk = K + k * 64 + (a1 * 4 + a2 * 2 + a3) * 8;
    cplx<R> acc = mk<R>(0, 0);
    for (int b = 0; b < 8; ++b) {
      const int b1 = b >> 2, b2 = (b >> 1) & 1, b3 = b & 1;
      const int64_t src = (((((x * 2 + b1) * 2 + b2) * dn2 + n2) * 2 + b3) * dn3 + n3) * dr + r;
      cfma(acc, GX(Kk, b), GX(Tz0, src));
    }
    GX(Tz, e) = acc;
  }
}

// Keeps a site near unit scale: per chain, the binary exponent ex of the largest |Re|, |Im| of the
// site's `elems` entries; when |ex| > 24 the site is multiplied by 2^-ex (exact) and 2 ex is added to
// the chain's trace exponent exp2 (the stored state times 2^exp2 is the represented one).
template <typename R>
__global__ void renorm_kernel(int64_t elems, cplx<R>* site, int64_t stride, int* exp2) {
  const int z = blockIdx.x;
  cplx<R>* S = site + (int64_t)z * stride;
  __shared__ R red[NT / 32];
  __shared__ int s_ex;
  R m = 0;
  for (int64_t e = threadIdx.x; e < elems; e += NT) {
    const cplx<R> v = GX(S, e);
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    R mm = 0;
    for (int w = 0; w < NT / 32; ++w) mm = fmax(mm, red[w]);
    int ex = 0;
    if (mm > R(0) && isfinite((double)mm)) frexp(mm, &ex);
    if (ex > 24 || ex < -24) GX(exp2, z) += 2 * ex;
    else ex = 0;
    s_ex = ex;
  }
  __syncthreads();
  if (s_ex != 0) {
    const R f = ldexp(R(1), -s_ex);
    for (int64_t e = threadIdx.x; e < elems; e += NT) {
      cplx<R>& v = GX(S, e);
      v.x *= f;
      v.y *= f;
    }
  }
}

// Kraus-leg Gram of a site (or merged pair) with a new Kraus leg, X = (Khat (x) I) A, from the Gram H
// of A over its bond indices:  G[(k, n), (k', n')] = sum_{p, p''} M_kk'[p, p''] H[(p, n), (p'', n')]
// with M_kk' = Khat_k^H Khat_k' (d x d, d = 2 for one qubit, 4 for a pair); G column-major (ld rk dn),
// H row-major (d dn x d dn).
template <typename R>
__global__ void kraus_gram_kernel(int d, int rk, int dn, const cplx<R>* Khat, const cplx<R>* H, int64_t hstride,
                                  cplx<R>* G, int64_t gstride) {
  const int z = blockIdx.y;
  const int NK = rk * dn, NH = d * dn, dd = d * d;
  const cplx<R>* K = Khat + (int64_t)z * rk * dd;
  const cplx<R>* Hz = H + (int64_t)z * hstride;
  cplx<R>* Gz = G + (int64_t)z * gstride;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)NK * NK;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % NK), b = (int)(e / NK);
    const int k = a / dn, n = a % dn, k2 = b / dn, n2 = b % dn;
    cplx<R> acc = mk<R>(0, 0);
    for (int p = 0; p < d; ++p)
      for (int pp = 0; pp < d; ++pp) {
        cplx<R> m = mk<R>(0, 0);
        for (int t = 0; t < d; ++t) cfma_cj(m, GX(K, k * dd + t * d + p), GX(K, k2 * dd + t * d + pp));
        cfma(acc, m, GX(Hz, (int64_t)(p * dn + n) * NH + pp * dn + n2));
      }
    GX(Gz, e) = acc;
  }
}

// The kept Kraus directions folded into the fused gate:
//   W[(p', nu), (p, n)] = sum_k Khat_k[p', p] V[(k, n), nu]   (row-major d kap x d dn; V column-major, ld vld)
template <typename R>
__global__ void kraus_fold_kernel(int d, int rk, int dn, int kap, const cplx<R>* Khat, const cplx<R>* V,
                                  int64_t vstride, int vld, cplx<R>* W, int64_t wstride) {
  const int z = blockIdx.y;
  const int rows = d * kap, cols = d * dn, dd = d * d;
  const cplx<R>* K = Khat + (int64_t)z * rk * dd;
  const cplx<R>* Vz = V + (int64_t)z * vstride;
  cplx<R>* Wz = W + (int64_t)z * wstride;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols; e += gridDim.x * blockDim.x) {
    const int i = e / cols, j = e % cols;
    const int pq = i / kap, nu = i % kap, p = j / dn, n = j % dn;
    cplx<R> acc = mk<R>(0, 0);
    for (int k = 0; k < rk; ++k) cfma(acc, GX(K, k * dd + pq * d + p), GX(Vz, (int64_t)(k * dn + n) + (int64_t)nu * vld));
    GX(Wz, e) = acc;
  }
}

// V[:, j] *= s[j] for a column-major n x n matrix (FP64)
__global__ void scale_cols_kernel(int n, cplx<double>* V, const double* s) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const double f = GX(s, e / n);
    cplx<double>& v = GX(V, e);
    v.x *= f;
    v.y *= f;
  }
}

template <typename R>
__global__ void copy_view_kernel(int M, int N, const cplx<R>* in, View vin, cplx<R>* out, View vout) {
  const int z = blockIdx.y;
  const cplx<R>* I = in + view_batch(vin, z);
  cplx<R>* O = out + view_batch(vout, z);
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / N), j = (int)(e % N);
    cplx<R> v = GX(I, view_row(vin, i) + view_col(vin, j));
    if (vin.conj) v.y = -v.y;
    if (vout.conj) v.y = -v.y;
    GX(O, view_row(vout, i) + view_col(vout, j)) = v;
  }
}

template <typename R>
__global__ void scale_odd_kernel(int64_t len, int64_t div, R sgn, cplx<R>* x, int64_t stride) {
  cplx<R>* X = x + (int64_t)blockIdx.y * stride;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
    if ((e / div) % 2 == 1) GX(X, e) = sgn * GX(X, e);
}

template <typename A, typename B>
__global__ void convert_kernel(int64_t count, const cplx<A>* in, cplx<B>* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const cplx<A> v = GX(in, e);
    GX(out, e) = mk<B>((B)v.x, (B)v.y);
  }
}

template <typename R>
__global__ void init_zero_kernel(int count, cplx<R>* base, int64_t stride) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= count) return;
  GX(base, (int64_t)c * stride) = mk<R>(1, 0);
  GX(base, (int64_t)c * stride + 1) = mk<R>(0, 0);
}

template <typename R>
__global__ void dot_kernel(int64_t len, const cplx<R>* a, int64_t astride, const cplx<R>* b, int64_t bstride,
                           cplx<double>* out) {
  __shared__ double rx[NT / 32], ry[NT / 32];
  const int z = blockIdx.x;
  const cplx<R>* A = a + (int64_t)z * astride;
  const cplx<R>* B = b + (int64_t)z * bstride;
  double sx = 0, sy = 0;
  for (int64_t e = threadIdx.x; e < len; e += NT) {
    cplx<R> u = GX(A, e), v = GX(B, e);
    sx += (double)u.x * v.x + (double)u.y * v.y;
    sy += (double)u.x * v.y - (double)u.y * v.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  if ((threadIdx.x & 31) == 0) {
    rx[threadIdx.x >> 5] = sx;
    ry[threadIdx.x >> 5] = sy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tx = 0, ty = 0;
    for (int w = 0; w < NT / 32; ++w) {
      tx += rx[w];
      ty += ry[w];
    }
    GX(out, z) = mk<double>(tx, ty);
  }
}

template <typename R>
__global__ void fill_kernel(int64_t count, cplx<R>* x, cplx<R> v) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    GX(x, e) = v;
}

template <typename R>
__global__ void herm_fill_kernel(int n, cplx<R>* A, int64_t stride) {
  cplx<R>* M = A + (int64_t)blockIdx.y * stride;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e % n), j = (int)(e / n);
    if (i < j) GX(M, e) = conjg(GX(M, (int64_t)i * n + j));
  }
}

__global__ void init_disc_kernel(int batch, double* d) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  GX(d, 3 * b) = 0.0;
  GX(d, 3 * b + 1) = 0.0;
  GX(d, 3 * b + 2) = 1e300;
}

struct PermDesc {
  int nd;
  int dims[6];     // input dims (row-major)
  int64_t ostr[6]; // output stride of each input dim
};

template <typename R>
__global__ void permute_kernel(PermDesc p, int64_t total, const cplx<R>* in, int64_t istride, cplx<R>* out,
                               int64_t ostride) {
  const cplx<R>* I = in + (int64_t)blockIdx.y * istride;
  cplx<R>* O = out + (int64_t)blockIdx.y * ostride;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = e, o = 0;
    for (int q = p.nd - 1; q >= 0; --q) {
      int64_t idx = t % p.dims[q];
      t /= p.dims[q];
      o += idx * p.ostr[q];
    }
    GX(O, o) = GX(I, e);
  }
}

inline int grid_for(int64_t total) {
  int64_t b = (total + NT - 1) / NT;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (int)b;
}
}  // namespace

cudaError_t chi_to_choi(cudaStream_t s, int count, int nq, const cplx<double>* chi, cplx<double>* choi) {
  if (count <= 0) return cudaSuccess;
  chi_to_choi_kernel<<<count, NT, 0, s>>>(count, nq, chi, choi);
  return cudaGetLastError();
}
cudaError_t choi_to_kraus(cudaStream_t s, int count, int nq, int rmax, const int* r_dev, const double* eta,
                          const cplx<double>* vecs, cplx<double>* kraus) {
  if (count <= 0) return cudaSuccess;
  choi_to_kraus_kernel<<<count, NT, 0, s>>>(count, nq, rmax, r_dev, eta, vecs, kraus);
  return cudaGetLastError();
}
template <typename R>
cudaError_t herm_fill_upper(cudaStream_t s, int batch, int n, cplx<R>* A, int64_t stride) {
  if (batch <= 0 || n <= 1) return cudaSuccess;
  dim3 grid(grid_for((int64_t)n * n), batch);
  herm_fill_kernel<R><<<grid, NT, 0, s>>>(n, A, stride);
  return cudaGetLastError();
}
template cudaError_t herm_fill_upper<float>(cudaStream_t, int, int, cplx<float>*, int64_t);
template cudaError_t herm_fill_upper<double>(cudaStream_t, int, int, cplx<double>*, int64_t);

cudaError_t init_discarded(cudaStream_t s, int batch, double* d) {
  if (batch <= 0) return cudaSuccess;
  init_disc_kernel<<<(batch + 127) / 128, 128, 0, s>>>(batch, d);
  return cudaGetLastError();
}
cudaError_t kraus_tp_error(cudaStream_t s, int count, int nq, int rmax, const cplx<double>* kraus, double* err) {
  if (count <= 0) return cudaSuccess;
  kraus_tp_kernel<<<(count + 63) / 64, 64, 0, s>>>(count, nq, rmax, kraus, err);
  return cudaGetLastError();
}
template <typename R>
cudaError_t fuse_gate(cudaStream_t s, int batch, const FuseArgs<R>& a) {
  if (batch <= 0) return cudaSuccess;
  if (a.nq < 1 || a.nq > 3 || a.rk < 1 || a.rk > (a.nq == 3 ? 64 : 16)) return cudaErrorInvalidValue;
  fuse_kernel<R><<<batch, 128, 0, s>>>(a);
  return cudaGetLastError();
}
template <typename R>
cudaError_t renorm_sites(cudaStream_t s, int batch, int64_t elems, cplx<R>* site, int64_t stride, int* exp2) {
  if (batch <= 0 || elems <= 0) return cudaSuccess;
  renorm_kernel<R><<<batch, NT, 0, s>>>(elems, site, stride, exp2);
  return cudaGetLastError();
}
template <typename R>
cudaError_t gate3(cudaStream_t s, int batch, int X, int dn2, int dn3, int dr, int rk, const cplx<R>* Khat,
                  const cplx<R>* T0, int64_t t0stride, cplx<R>* T, int64_t tstride) {
  if (batch <= 0) return cudaSuccess;
  if (rk < 1 || rk > 64) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)X * 4 * dn2 * rk * dn3 * 2 * dr;
  dim3 grid(grid_for(total), batch);
  gate3_kernel<R><<<grid, NT, 0, s>>>(X, dn2, dn3, dr, rk, Khat, T0, t0stride, T, tstride);
  return cudaGetLastError();
}
template <typename R>
cudaError_t build_T(cudaStream_t s, int batch, int dm, const cplx<R>* Rt, const cplx<R>* E, int64_t estride,
                    cplx<R>* T, int64_t tstride) {
  if (batch <= 0) return cudaSuccess;
  int64_t total = (int64_t)16 * dm * dm;
  dim3 grid(grid_for(total), batch);
  build_T_kernel<R><<<grid, NT, 0, s>>>(dm, Rt, E, estride, T, tstride);
  return cudaGetLastError();
}
template <typename R>
cudaError_t build_Y(cudaStream_t s, int batch, int kchi, int dm, int rk, const cplx<R>* Khat, const cplx<R>* H,
                    int64_t hstride, cplx<R>* Y, int64_t ystride) {
  if (batch <= 0) return cudaSuccess;
  int64_t total = (int64_t)kchi * 2 * rk * 2 * dm;
  dim3 grid(grid_for(total), batch);
  build_Y_kernel<R><<<grid, NT, 0, s>>>(kchi, dm, rk, Khat, H, hstride, Y, ystride);
  return cudaGetLastError();
}
cudaError_t scale_cols(cudaStream_t s, int n, cplx<double>* V, const double* f) {
  scale_cols_kernel<<<grid_for((int64_t)n * n), NT, 0, s>>>(n, V, f);
  return cudaGetLastError();
}

template <typename R>
cudaError_t kraus_gram(cudaStream_t s, int batch, int d, int rk, int dn, const cplx<R>* Khat, const cplx<R>* H,
                       int64_t hstride, cplx<R>* G, int64_t gstride) {
  if (batch <= 0) return cudaSuccess;
  if (rk > 16 || (d != 2 && d != 4)) return cudaErrorInvalidValue;
  dim3 grid(grid_for((int64_t)rk * dn * rk * dn), batch);
  kraus_gram_kernel<R><<<grid, NT, 0, s>>>(d, rk, dn, Khat, H, hstride, G, gstride);
  return cudaGetLastError();
}
template <typename R>
cudaError_t kraus_fold(cudaStream_t s, int batch, int d, int rk, int dn, int kap, const cplx<R>* Khat,
                       const cplx<R>* V, int64_t vstride, int vld, cplx<R>* W, int64_t wstride) {
  if (batch <= 0) return cudaSuccess;
  if (rk > 16 || (d != 2 && d != 4)) return cudaErrorInvalidValue;
  dim3 grid(grid_for((int64_t)d * d * kap * dn), batch);
  kraus_fold_kernel<R><<<grid, NT, 0, s>>>(d, rk, dn, kap, Khat, V, vstride, vld, W, wstride);
  return cudaGetLastError();
}
template <typename R>
cudaError_t copy_view(cudaStream_t s, int batch, int M, int N, const cplx<R>* in, View vin, cplx<R>* out, View vout) {
  if (batch <= 0 || M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid(grid_for((int64_t)M * N), batch);
  copy_view_kernel<R><<<grid, NT, 0, s>>>(M, N, in, vin, out, vout);
  return cudaGetLastError();
}
template <typename R>
cudaError_t scale_odd(cudaStream_t s, int batch, int64_t len, int64_t div, R sgn, cplx<R>* x, int64_t stride) {
  if (batch <= 0 || len <= 0) return cudaSuccess;
  dim3 grid(grid_for(len), batch);
  scale_odd_kernel<R><<<grid, NT, 0, s>>>(len, div, sgn, x, stride);
  return cudaGetLastError();
}
template <typename A, typename B>
cudaError_t convert(cudaStream_t s, int64_t count, const cplx<A>* in, cplx<B>* out) {
  if (count <= 0) return cudaSuccess;
  convert_kernel<A, B><<<grid_for(count), NT, 0, s>>>(count, in, out);
  return cudaGetLastError();
}
template <typename R>
cudaError_t init_zero_sites(cudaStream_t s, int count, cplx<R>* base, int64_t stride) {
  if (count <= 0) return cudaSuccess;
  init_zero_kernel<R><<<(count + 127) / 128, 128, 0, s>>>(count, base, stride);
  return cudaGetLastError();
}
template <typename R>
cudaError_t dot_batch(cudaStream_t s, int batch, int64_t len, const cplx<R>* a, int64_t astride, const cplx<R>* b,
                      int64_t bstride, cplx<double>* out) {
  if (batch <= 0) return cudaSuccess;
  dot_kernel<R><<<batch, NT, 0, s>>>(len, a, astride, b, bstride, out);
  return cudaGetLastError();
}
template <typename R>
cudaError_t fill(cudaStream_t s, int64_t count, cplx<R>* x, cplx<R> v) {
  if (count <= 0) return cudaSuccess;
  fill_kernel<R><<<grid_for(count), NT, 0, s>>>(count, x, v);
  return cudaGetLastError();
}
template <typename R>
cudaError_t permute(cudaStream_t s, int batch, int nd, const int* dims, const int* perm, const cplx<R>* in,
                    int64_t istride, cplx<R>* out, int64_t ostride) {
  if (batch <= 0 || nd < 1 || nd > 6) return nd > 6 ? cudaErrorInvalidValue : cudaSuccess;
  PermDesc p{};
  p.nd = nd;
  int64_t total = 1;
  for (int q = 0; q < nd; ++q) {
    p.dims[q] = dims[q];
    total *= dims[q];
  }
  // output dim j is input dim perm[j]; output is row-major over the permuted dims
  int64_t st = 1;
  for (int j = nd - 1; j >= 0; --j) {
    p.ostr[perm[j]] = st;
    st *= dims[perm[j]];
  }
  if (total == 0) return cudaSuccess;
  dim3 grid(grid_for(total), batch);
  permute_kernel<R><<<grid, NT, 0, s>>>(p, total, in, istride, out, ostride);
  return cudaGetLastError();
}

#define INST(R)                                                                                                  \
  template cudaError_t fuse_gate<R>(cudaStream_t, int, const FuseArgs<R>&);                                      \
  template cudaError_t renorm_sites<R>(cudaStream_t, int, int64_t, cplx<R>*, int64_t, int*);                  \
  template cudaError_t gate3<R>(cudaStream_t, int, int, int, int, int, int, const cplx<R>*, const cplx<R>*,      \
                                int64_t, cplx<R>*, int64_t);                                                     \
  template cudaError_t build_T<R>(cudaStream_t, int, int, const cplx<R>*, const cplx<R>*, int64_t, cplx<R>*,     \
                                  int64_t);                                                                      \
  template cudaError_t build_Y<R>(cudaStream_t, int, int, int, int, const cplx<R>*, const cplx<R>*, int64_t,     \
                                  cplx<R>*, int64_t);                                                            \
  template cudaError_t copy_view<R>(cudaStream_t, int, int, int, const cplx<R>*, View, cplx<R>*, View);          \
  template cudaError_t kraus_gram<R>(cudaStream_t, int, int, int, int, const cplx<R>*, const cplx<R>*, int64_t,  \
                                     cplx<R>*, int64_t);                                                         \
  template cudaError_t kraus_fold<R>(cudaStream_t, int, int, int, int, int, const cplx<R>*, const cplx<R>*,      \
                                     int64_t, int, cplx<R>*, int64_t);                                           \
  template cudaError_t scale_odd<R>(cudaStream_t, int, int64_t, int64_t, R, cplx<R>*, int64_t);                  \
  template cudaError_t init_zero_sites<R>(cudaStream_t, int, cplx<R>*, int64_t);                                 \
  template cudaError_t dot_batch<R>(cudaStream_t, int, int64_t, const cplx<R>*, int64_t, const cplx<R>*,         \
                                    int64_t, cplx<double>*);                                                     \
  template cudaError_t fill<R>(cudaStream_t, int64_t, cplx<R>*, cplx<R>);                                        \
  template cudaError_t permute<R>(cudaStream_t, int, int, const int*, const int*, const cplx<R>*, int64_t,       \
                                  cplx<R>*, int64_t);
INST(float)
INST(double)
template cudaError_t convert<float, double>(cudaStream_t, int64_t, const cplx<float>*, cplx<double>*);
template cudaError_t convert<double, float>(cudaStream_t, int64_t, const cplx<double>*, cplx<float>*);
template cudaError_t convert<double, double>(cudaStream_t, int64_t, const cplx<double>*, cplx<double>*);
template cudaError_t convert<float, float>(cudaStream_t, int64_t, const cplx<float>*, cplx<float>*);

}  // namespace mpdo
