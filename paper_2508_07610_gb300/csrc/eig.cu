// Batched Hermitian eigensolver for the truncation steps: the top-k eigenpairs of an n x n
// Hermitian matrix, one CTA per matrix (CUDA cores, FP32 or FP64).
//
// The SVD truncations of Sec. II.D (Eq. svdNoise for the Kraus leg, Fig. 3b for the bond) only
// need the leading singular subspace of a tall or wide matrix X, i.e. the top eigenpairs of its
// Gram matrix X X^H; this kernel supplies them.  The Choi-matrix eigendecomposition of Sec. III
// (chi -> Kraus) uses it with k = n in FP64.
//
// Steps: (1) Householder reduction to a complex Hermitian tridiagonal (matrix kept in global
// memory, which the L2 holds), blocked in panels of NB reflectors whose (v, w) pairs stay in shared
// memory, followed by a diagonal phase change that makes it real symmetric; (2) bisection with Sturm
// counts for the top k eigenvalues, one thread per eigenvalue; (3) inverse iteration on the
// tridiagonal (LU with partial pivoting) from distinct pseudo-random starts, one thread per vector;
// (4) classical Gram-Schmidt applied twice, in descending eigenvalue order and in blocks of GB
// vectors, which also separates vectors of (near-)degenerate eigenvalues; (5) back-transformation of
// all k vectors through the phases and the Householder reflectors, NB reflectors at a time as one
// block reflector.  Every loop is bounded; the input matrix is overwritten.
//
// FP64 on this GPU has 1/64 of the FP32 issue rate, so the FP64 instantiation saves FP64 operations
// where it can without losing accuracy: the reduction updates only the lower triangle of the
// trailing block with fused complex multiply-adds, the off-diagonal magnitudes are taken once, the
// substitutions of the inverse iteration multiply by reciprocal pivots instead of dividing, and the
// bisection starts from an FP32 bracket confirmed by FP64 Sturm counts.  (Taking the FP32 values as
// the final shifts was tried and rejected: they cannot separate eigenvalues closer than about
// u32 ||T||, and cuts with relative gaps between 1e-9 and 1e-6 then lost FP64 accuracy.)
#include "device_once.cuh"
#include "kernels.h"
#include "panel.cuh"

namespace mpdo {

namespace {
constexpr int NT = 256;
constexpr int MAXN = 512;
constexpr int GB = 8;  // vectors per block of the Gram-Schmidt step

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
__device__ R block_max(R v, R* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  R s = 0;
  for (int w = 0; w < NT / 32; ++w) s = fmax(s, red[w]);
  return s;
}

template <typename R>
__device__ cplx<R> block_csum(cplx<R> v, R* red) {
  R a = block_sum(v.x, red);
  R b = block_sum(v.y, red);
  return mk(a, b);
}

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

template <typename R>
__device__ __forceinline__ R eps_of();
template <>
__device__ __forceinline__ float eps_of<float>() { return 1.1920929e-07f; }
template <>
__device__ __forceinline__ double eps_of<double>() { return 2.220446049250313e-16; }

// FP64 runs on a pipe 64 times narrower than FP32 on this GPU, so in FP64 the reduction keeps only the
// lower triangle of the trailing block up to date (a third fewer FP64 operations); in FP32, where
// the kernel is bound by latency rather than arithmetic, the full square is cheaper to address.
template <typename R>
__host__ __device__ constexpr bool kLowerOnly() {
  return sizeof(R) == 8;
}

// number of eigenvalues of the real symmetric tridiagonal (d, e2 = e^2) below sigma
template <typename R>
__device__ int sturm_count(const R* d, const R* e2, int n, R sigma, R pivmin) {
  int cnt = 0;
  R q = d[0] - sigma;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < R(0)) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = d[i] - sigma - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < R(0)) ++cnt;
  }
  return cnt;
}

template <typename R, int NB>
__global__ void __launch_bounds__(NT, 2) heevk_kernel(EigArgs<R> g) {
  __shared__ R red[NT / 32];
  __shared__ R s_d[MAXN], s_e2[MAXN], s_beta[MAXN], s_eabs[MAXN];
  __shared__ float s_d32[sizeof(R) == 8 ? MAXN : 1], s_e232[sizeof(R) == 8 ? MAXN : 1];
  __shared__ cplx<R> s_p[MAXN], s_v[MAXN];
  __shared__ R s_w[MAXN];
  __shared__ cplx<R> s_v0[MAXN];
  __shared__ int s_flag, s_bad;
  const int z = blockIdx.x;
  const int n = g.n, k = g.k;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_bad = 0;
  GPTR(cplx<R>, A, g.A + (int64_t)z * g.astride);
  R* const S = g.scratch + (int64_t)z * g.sstride;
  const int64_t nk = (int64_t)n * k;
  // scratch layout (R units, vector t element i at [i * k + t] so threads walk it coalesced)
  GPTR(R, Ldl, S);
  GPTR(R, Ldd, S + nk);
  GPTR(R, Ldu, S + 2 * nk);
  GPTR(R, Ldu2, S + 3 * nk);
  GPTR(R, Lpiv, S + 4 * nk);
  GPTR(R, Zr, S + 5 * nk);
  GPTR(cplx<R>, U, reinterpret_cast<cplx<R>*>(S + 6 * nk));        // complex, vector t column at [t * n]
  GPTR(cplx<R>, PH, reinterpret_cast<cplx<R>*>(S + 6 * nk) + nk);  // phases, n

  // ---- (0) scale.  The safeguards below (pivot minimum, the zero test of Householder norms, the FP32
  // bracket) are absolute, so the matrix is first multiplied by the power of two that brings its
  // largest entry into [1/2, 1): Gram matrices of states whose norm has decayed by many orders of
  // magnitude then behave like unit-scale ones.  The scaling is exact; eigenvalues are scaled back on
  // output, and the discarded weight and the gap are ratios.
  __shared__ int s_exp;
  {
    R amax = 0;
    for (int64_t e = tid; e < (int64_t)n * n; e += NT) amax = fmax(amax, fmax(fabs(A[e].x), fabs(A[e].y)));
    amax = block_max(amax, red);
    if (tid == 0) {
      int ex = 0;
      if (amax > R(0) && isfinite((double)amax)) frexp(amax, &ex);
      s_exp = ex;
    }
    __syncthreads();
    if (s_exp != 0) {
      const R f = ldexp(R(1), -s_exp);
      for (int64_t e = tid; e < (int64_t)n * n; e += NT) {
        A[e].x *= f;
        A[e].y *= f;
      }
    }
    __syncthreads();
  }

  // ---- (1) tridiagonalisation: A <- H A H on the trailing block, H = I - beta v v^H, in panels of
  // NB reflectors.  Inside a panel the trailing block is not updated: column j is brought up to date
  // from the panel's earlier pairs (v_l, w_l) when it is reached, and the product with the block uses
  // A v - V (W^H v) - W (V^H v).  At the end of the panel the whole rank-2 NB update is applied in one
  // pass (the blocked reduction of LAPACK's Hermitian tridiagonalisation).
  extern __shared__ __align__(16) unsigned char eig_dyn[];
  cplx<R>* Vb = reinterpret_cast<cplx<R>*>(eig_dyn);  // NB x n, reflector l at Vb + l * n
  cplx<R>* Wb = Vb + (size_t)NB * n;                  // NB x n
  __shared__ cplx<R> s_x[2 * NB];
  for (int j0 = 0; j0 + 2 < n; j0 += NB) {
    const int pb = (n - 2 - j0 < NB) ? n - 2 - j0 : NB;
    for (int jj = 0; jj < pb; ++jj) {
      const int j = j0 + jj;
      auto col = A + (int64_t)j * n;
      // column j (rows j..n-1) brought up to date and written back
      for (int i = j + tid; i < n; i += NT) {
        cplx<R> c = col[i];
        for (int l = 0; l < jj; ++l) {
          cfms_cj(c, Vb[l * n + i], Wb[l * n + j]);
          cfms_cj(c, Wb[l * n + i], Vb[l * n + j]);
        }
        col[i] = c;
      }
      __syncthreads();
      R s = 0;
      for (int i = j + 2 + tid; i < n; i += NT) s += norm2(col[i]);
      s = block_sum(s, red);
      const cplx<R> a = col[j + 1];
      const R aa = sqrt(norm2(a));
      const R nrm = sqrt(aa * aa + s);
      const cplx<R> ph = (aa > R(0)) ? mk<R>(a.x / aa, a.y / aa) : mk<R>(1, 0);
      const R beta = (nrm > tiny_norm<R>()) ? R(1) / (nrm * (nrm + aa)) : R(0);
      const cplx<R> v0 = a + nrm * ph;
      for (int i = tid; i < n; i += NT) {
        const cplx<R> v = (i > j + 1) ? col[i] : (i == j + 1 ? v0 : mk<R>(0, 0));
        s_v[i] = v;
        Vb[jj * n + i] = v;
      }
      if (tid == 0) s_beta[j] = beta;
      __syncthreads();
      if (beta != R(0)) {
        // x1_l = w_l^H v, x2_l = v_l^H v for the panel's earlier reflectors
        for (int d = wid; d < 2 * jj; d += NT / 32) {
          const cplx<R>* u = (d < jj) ? Wb + d * n : Vb + (d - jj) * n;
          cplx<R> acc = mk<R>(0, 0);
          for (int i = j + 1 + lane; i < n; i += 32) cfma_cj(acc, u[i], s_v[i]);
          for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
          }
          if (lane == 0) s_x[d] = acc;
        }
        __syncthreads();
        // p = beta (A_sub v - V x1 - W x2) on rows j+1..
        if constexpr (kLowerOnly<R>()) {
          // only the lower triangle of the trailing block is current: rows i take sum_{c <= i}
          // A(i, c) v_c from the columns (coalesced over i), then one warp per column i adds
          // sum_{c > i} conj(A(c, i)) v_c, the stored column read downwards
          for (int i = j + 1 + tid; i < n; i += NT) {
            constexpr int MV = 8;
            cplx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
            int c = j + 1;
            for (; c + MV <= i + 1; c += MV) {
              cplx<R> a[MV];
#pragma unroll
              for (int u = 0; u < MV; ++u) a[u] = A[(int64_t)(c + u) * n + i];
#pragma unroll
              for (int u = 0; u < MV; u += 2) {
                cfma(acc0, a[u], s_v[c + u]);
                cfma(acc1, a[u + 1], s_v[c + u + 1]);
              }
            }
            for (; c <= i; ++c) cfma(acc0, A[(int64_t)c * n + i], s_v[c]);
            s_p[i] = acc0 + acc1;
          }
          __syncthreads();
          for (int i = j + 1 + wid; i + 1 < n; i += NT / 32) {
            const auto coli = A + (int64_t)i * n;
            cplx<R> dot = mk<R>(0, 0);
            for (int c = i + 1 + lane; c < n; c += 32) cfma_cj(dot, coli[c], s_v[c]);
            dot = panel::warp_csum(dot);
            if (lane == 0) s_p[i] = s_p[i] + dot;
          }
          __syncthreads();
          for (int i = j + 1 + tid; i < n; i += NT) {
            cplx<R> acc = s_p[i];
            for (int l = 0; l < jj; ++l) {
              cfms(acc, Vb[l * n + i], s_x[l]);
              cfms(acc, Wb[l * n + i], s_x[jj + l]);
            }
            s_p[i] = beta * acc;
          }
        } else
        for (int i = j + 1 + tid; i < n; i += NT) {
          // the column loads of a block of MV columns are all issued before any is used, so a
          // thread has MV L2 requests in flight instead of one
          constexpr int MV = sizeof(R) == 8 ? 8 : 16;
          cplx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0), acc2 = mk<R>(0, 0), acc3 = mk<R>(0, 0);
          int c = j + 1;
          for (; c + MV <= n; c += MV) {
            cplx<R> a[MV];
#pragma unroll
            for (int u = 0; u < MV; ++u) a[u] = A[(int64_t)(c + u) * n + i];
#pragma unroll
            for (int u = 0; u < MV; u += 4) {
              cfma(acc0, a[u], s_v[c + u]);
              cfma(acc1, a[u + 1], s_v[c + u + 1]);
              cfma(acc2, a[u + 2], s_v[c + u + 2]);
              cfma(acc3, a[u + 3], s_v[c + u + 3]);
            }
          }
          for (; c < n; ++c) cfma(acc0, A[(int64_t)c * n + i], s_v[c]);
          cplx<R> acc = (acc0 + acc1) + (acc2 + acc3);
          for (int l = 0; l < jj; ++l) {
            cfms(acc, Vb[l * n + i], s_x[l]);
            cfms(acc, Wb[l * n + i], s_x[jj + l]);
          }
          s_p[i] = beta * acc;
        }
        __syncthreads();
        // K = (beta / 2) v^H p ; w = p - K v
        cplx<R> part = mk<R>(0, 0);
        for (int i = j + 1 + tid; i < n; i += NT) cfma_cj(part, s_v[i], s_p[i]);
        cplx<R> K = block_csum(part, red);
        K = (beta * R(0.5)) * K;
        for (int i = tid; i < n; i += NT) Wb[jj * n + i] = (i > j) ? s_p[i] - K * s_v[i] : mk<R>(0, 0);
      } else {
        for (int i = tid; i < n; i += NT) Wb[jj * n + i] = mk<R>(0, 0);
      }
      __syncthreads();
      if (tid == 0) {
        col[j + 1] = (beta != R(0)) ? mk<R>(-nrm * ph.x, -nrm * ph.y) : a;  // the new subdiagonal e_j
        s_v0[j] = v0;  // v_{j+1}; v_i for i >= j + 2 stay in col[i]
      }
      __syncthreads();
    }
    // trailing block (rows and columns from t0 on): A -= V W^H + W V^H over the panel
    const int t0 = j0 + pb, nt = n - t0;
    // four elements per thread per pass, loaded together before any is updated
    constexpr int EU = 4;
    const int64_t nn = (int64_t)nt * nt;
    for (int64_t e0 = tid; e0 < nn; e0 += (int64_t)NT * EU) {
      cplx<R> v[EU];
#pragma unroll
      for (int u = 0; u < EU; ++u) {
        const int64_t e = e0 + (int64_t)u * NT;
        const bool need = e < nn && !(kLowerOnly<R>() && (int)(e % nt) < (int)(e / nt));
        if (need) v[u] = A[(int64_t)(t0 + (int)(e / nt)) * n + t0 + (int)(e % nt)];
      }
#pragma unroll
      for (int u = 0; u < EU; ++u) {
        const int64_t e = e0 + (int64_t)u * NT;
        if (e >= nn) continue;
        const int i = t0 + (int)(e % nt), c = t0 + (int)(e / nt);
        if (kLowerOnly<R>() && i < c) continue;  // the upper triangle is never read again
        cplx<R> w = v[u];
        for (int l = 0; l < pb; ++l) {
          cfms_cj(w, Vb[l * n + i], Wb[l * n + c]);
          cfms_cj(w, Wb[l * n + i], Vb[l * n + c]);
        }
        A[(int64_t)c * n + i] = w;
      }
    }
    __syncthreads();
  }
  // diagonal, |off-diagonal|^2 and the phases Phi that make the tridiagonal real:
  // T_real = Phi^H T Phi with phi_0 = 1, phi_{j+1} = phi_j e_j / |e_j|
  for (int i = tid; i < n; i += NT) s_d[i] = A[(int64_t)i * n + i].x;
  if (tid == 0) {
    cplx<R> phi = mk<R>(1, 0);
    PH[0] = phi;
    for (int j = 0; j + 1 < n; ++j) {
      cplx<R> e = A[(int64_t)j * n + j + 1];
      R ae = sqrt(norm2(e));
      s_e2[j] = ae * ae;
      if (ae > R(0)) phi = phi * mk<R>(e.x / ae, e.y / ae);
      PH[j + 1] = phi;
    }
  }
  __syncthreads();

  // ---- (2) bisection for the top kk = min(k + 1, n) eigenvalues (descending)
  const int kk = (k < n) ? k + 1 : n;
  R gl = s_d[0], gu = s_d[0], emax2 = 0, trace = 0;
  for (int i = 0; i < n; ++i) {
    R r = 0;
    if (i > 0) r += sqrt(s_e2[i - 1]);
    if (i + 1 < n) r += sqrt(s_e2[i]);
    gl = fmin(gl, s_d[i] - r);
    gu = fmax(gu, s_d[i] + r);
    if (i + 1 < n) emax2 = fmax(emax2, s_e2[i]);
    trace += s_d[i];
  }
  const R eps = eps_of<R>();
  const R tnorm = fmax(fabs(gl), fabs(gu));
  const R pivmin = R(1e-30) * fmax(R(1), emax2);
  const R abstol = eps * tnorm + pivmin;
  gl -= R(2) * eps * tnorm * n + pivmin;
  gu += R(2) * eps * tnorm * n + pivmin;
  for (int i = tid; i < n; i += NT) s_eabs[i] = (i + 1 < n) ? sqrt(s_e2[i]) : R(0);
  if constexpr (sizeof(R) == 8) {
    for (int i = tid; i < n; i += NT) {
      s_d32[i] = (float)s_d[i];
      s_e232[i] = (float)s_e2[i];
    }
    __syncthreads();
  }
  for (int t = tid; t < kk; t += NT) {
    const int target = n - 1 - t;  // ascending index of the t-th largest eigenvalue
    R lo = gl, hi = gu;
    if constexpr (sizeof(R) == 8) {
      // FP64 Sturm counts divide on a pipe 64 times narrower than FP32: bracket the eigenvalue in
      // FP32 first, widen the bracket by the FP32 counts' error, keep it if two FP64 counts confirm
      // it, and let the FP64 bisection below finish from there (same result, fewer FP64 counts)
      const float e32 = eps_of<float>(), tn32 = (float)tnorm;
      const float piv32 = fmaxf(1e-30f * fmaxf(1.f, (float)emax2), 1e-36f);
      float l32 = (float)gl, h32 = (float)gu;
      for (int it = 0; it < 128; ++it) {
        const float mid = 0.5f * (l32 + h32);
        if (h32 - l32 <= 2.f * e32 * fmaxf(fabsf(l32), fabsf(h32)) + e32 * tn32 + piv32 || mid == l32 || mid == h32)
          break;
        if (sturm_count(s_d32, s_e232, n, mid, piv32) > target) h32 = mid; else l32 = mid;
      }
      const R pad = R(16) * R(e32) * tnorm + pivmin;
      const R blo = R(l32) - pad, bhi = R(h32) + pad;
      if (sturm_count(s_d, s_e2, n, blo, pivmin) <= target && sturm_count(s_d, s_e2, n, bhi, pivmin) > target) {
        lo = blo;
        hi = bhi;
      }
    }
    for (int it = 0; it < 256; ++it) {
      R mid = R(0.5) * (lo + hi);
      if (hi - lo <= R(2) * eps * fmax(fabs(lo), fabs(hi)) + abstol || mid == lo || mid == hi) break;
      if (sturm_count(s_d, s_e2, n, mid, pivmin) > target) hi = mid; else lo = mid;
    }
    s_w[t] = R(0.5) * (lo + hi);
  }
  __syncthreads();

  // ---- (3) inverse iteration, one thread per vector t < k.  The recurrences carry the running row
  // (LU) or the running solution entries (substitutions) in registers, so the only memory traffic
  // inside a recurrence is independent loads of the factors and stores of the results.
  const R pert = eps * fmax(tnorm, R(1e-30));
  for (int t = tid; t < k; t += NT) {
    const R lam = s_w[t];
    // LU with partial pivoting of T - lam I: factors dd (diagonal of U), du, du2 (its two upper
    // diagonals), dl (multipliers) and the row interchanges, row by row; (d, u) is the current row
    R d = s_d[0] - lam;
    R u = (n > 1) ? s_eabs[0] : R(0);
    for (int i = 0; i + 1 < n; ++i) {
      const R l = s_eabs[i];
      const R dn = s_d[i + 1] - lam;
      const R un = (i + 2 < n) ? s_eabs[i + 1] : R(0);
      const int64_t o = (int64_t)i * k + t;
      if (fabs(d) >= fabs(l)) {
        if (fabs(d) < pert) d = (d < R(0)) ? -pert : pert;
        const R f = l / d;
        Ldd[o] = R(1) / d;  // reciprocal pivots: the substitutions multiply
        Ldu[o] = u;
        Ldu2[o] = 0;
        Ldl[o] = f;
        Lpiv[o] = 0;
        d = dn - f * u;
        u = un;
      } else {
        const R f = d / l;
        Ldd[o] = R(1) / l;
        Ldu[o] = dn;
        Ldu2[o] = un;
        Ldl[o] = f;
        Lpiv[o] = 1;
        d = u - f * dn;
        u = -f * un;
      }
    }
    if (fabs(d) < pert) d = (d < R(0)) ? -pert : pert;
    Ldd[(int64_t)(n - 1) * k + t] = R(1) / d;
    // start vector
    for (int i = 0; i < n; ++i) {
      uint32_t h = hash32((uint32_t)(t * 7919 + 1) * 2654435761u ^ (uint32_t)(i * 40503 + 17));
      Zr[(int64_t)i * k + t] = R((int)(h >> 8) - (1 << 23)) / R(1 << 23);
    }
    // the substitutions work through the vector in chunks of CH entries: the chunk's factors and
    // inputs are loaded together (independent loads), then the recurrence runs on registers
    constexpr int CH = 8;
    for (int it = 0; it < 3; ++it) {
      // forward: apply L^-1 with the row interchanges; zi is the running entry i
      R zi = Zr[t];
      for (int i0 = 0; i0 + 1 < n; i0 += CH) {
        const int cnt = (n - 1 - i0 < CH) ? n - 1 - i0 : CH;
        R zn[CH], f[CH], pv[CH], out[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          if (c < cnt) {
            const int64_t o = (int64_t)(i0 + c) * k + t;
            zn[c] = Zr[o + k];
            f[c] = Ldl[o];
            pv[c] = Lpiv[o];
          }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          if (c < cnt) {
            if (pv[c] != R(0)) {
              out[c] = zn[c];
              zi = zi - f[c] * zn[c];
            } else {
              out[c] = zi;
              zi = zn[c] - f[c] * zi;
            }
          }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (c < cnt) Zr[(int64_t)(i0 + c) * k + t] = out[c];
      }
      Zr[(int64_t)(n - 1) * k + t] = zi;
      // backward: U z = y; z1, z2 are the solution entries i + 1, i + 2
      R zmax = 0, z1 = 0, z2 = 0;
      for (int i1 = n - 1; i1 >= 0; i1 -= CH) {
        const int cnt = (i1 + 1 < CH) ? i1 + 1 : CH;
        R y[CH], du[CH], du2[CH], dd[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          if (c < cnt) {
            const int64_t o = (int64_t)(i1 - c) * k + t;
            y[c] = Zr[o];
            du[c] = Ldu[o];
            du2[c] = Ldu2[o];
            dd[c] = Ldd[o];
          }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          if (c < cnt) {
            const int i = i1 - c;
            R v = y[c];
            if (i + 1 < n) v -= du[c] * z1;
            if (i + 2 < n) v -= du2[c] * z2;
            v *= dd[c];
            if (!(fabs(v) < R(1e30))) v = (v > 0) ? R(1e30) : R(-1e30);
            y[c] = v;
            zmax = fmax(zmax, fabs(v));
            z2 = z1;
            z1 = v;
          }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (c < cnt) Zr[(int64_t)(i1 - c) * k + t] = y[c];
      }
      const R sc = (zmax > R(0)) ? R(1) / zmax : R(1);
      R nn = 0;
      for (int i0 = 0; i0 < n; i0 += CH) {
        R y[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (i0 + c < n) y[c] = Zr[(int64_t)(i0 + c) * k + t] * sc;
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (i0 + c < n) nn += y[c] * y[c];
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (i0 + c < n) Zr[(int64_t)(i0 + c) * k + t] = y[c];
      }
      const R inv = (nn > R(0)) ? R(1) / sqrt(nn) : R(0);
      for (int i0 = 0; i0 < n; i0 += CH) {
        R y[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (i0 + c < n) y[c] = Zr[(int64_t)(i0 + c) * k + t];
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (i0 + c < n) Zr[(int64_t)(i0 + c) * k + t] = y[c] * inv;
      }
    }
  }
  __syncthreads();

  // ---- (4) Gram-Schmidt (twice) in descending order, in blocks of GB vectors: each block is first
  // projected against every earlier vector as a block (twice), then orthogonalised within itself
  // vector by vector; a vector that collapses is redone from a fresh start against all earlier ones
  R* s_G = reinterpret_cast<R*>(Wb + (size_t)NB * n);  // GB x k: the block's projections (dynamic)
  for (int t0 = 0; t0 < k; t0 += GB) {
  const int nb = (k - t0 < GB) ? k - t0 : GB;
  if (t0 > 0) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int e = tid; e < t0 * nb; e += NT) {
        const int u = e % t0, c = e / t0;
        R acc0 = 0, acc1 = 0;
        int i = 0;
        for (; i + 1 < n; i += 2) {
          acc0 += Zr[(int64_t)i * k + u] * Zr[(int64_t)i * k + t0 + c];
          acc1 += Zr[(int64_t)(i + 1) * k + u] * Zr[(int64_t)(i + 1) * k + t0 + c];
        }
        if (i < n) acc0 += Zr[(int64_t)i * k + u] * Zr[(int64_t)i * k + t0 + c];
        s_G[c * k + u] = acc0 + acc1;
      }
      __syncthreads();
      for (int e = tid; e < n * nb; e += NT) {
        const int c = e % nb, i = e / nb;
        R v = Zr[(int64_t)i * k + t0 + c];
        for (int u = 0; u < t0; ++u) v -= s_G[c * k + u] * Zr[(int64_t)i * k + u];
        Zr[(int64_t)i * k + t0 + c] = v;
      }
      __syncthreads();
    }
  }
  for (int t = t0; t < t0 + nb; ++t) {
    for (int attempt = 0; attempt < 3; ++attempt) {
      const int ub = (attempt == 0) ? t0 : 0;  // earlier blocks were projected out already
      for (int pass = 0; pass < 2; ++pass) {
        // dots with the previous vectors: warp w handles u = ub + w, ub + w + 8, ...
        for (int u = ub + wid; u < t; u += NT / 32) {
          R acc = 0;
          for (int i = lane; i < n; i += 32) acc += Zr[(int64_t)i * k + u] * Zr[(int64_t)i * k + t];
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) s_w[MAXN - 1 - u] = acc;  // dots parked at the tail of s_w (k + 1 <= MAXN / 2)
        }
        __syncthreads();
        for (int i = tid; i < n; i += NT) {
          R v = Zr[(int64_t)i * k + t];
          for (int u = ub; u < t; ++u) v -= s_w[MAXN - 1 - u] * Zr[(int64_t)i * k + u];
          Zr[(int64_t)i * k + t] = v;
        }
        __syncthreads();
      }
      R nn = 0;
      for (int i = tid; i < n; i += NT) nn += Zr[(int64_t)i * k + t] * Zr[(int64_t)i * k + t];
      nn = block_sum(nn, red);
      if (tid == 0) s_flag = (nn > R(0.01)) ? 1 : 0;
      __syncthreads();
      const R inv = (nn > R(0)) ? R(1) / sqrt(nn) : R(0);
      for (int i = tid; i < n; i += NT) Zr[(int64_t)i * k + t] *= inv;
      __syncthreads();
      if (s_flag || attempt == 2) break;
      // collapsed: one more inverse-iteration step from a fresh start, then orthogonalise again
      if (tid == 0) {
        for (int i = 0; i < n; ++i) {
          uint32_t h = hash32((uint32_t)(t * 104729 + attempt * 7 + 3) ^ (uint32_t)(i * 92821 + 5));
          Zr[(int64_t)i * k + t] = R((int)(h >> 8) - (1 << 23)) / R(1 << 23);
        }
        for (int i = 0; i + 1 < n; ++i) {
          R zi = Zr[(int64_t)i * k + t], zn = Zr[(int64_t)(i + 1) * k + t], f = Ldl[(int64_t)i * k + t];
          if (Lpiv[(int64_t)i * k + t] != R(0)) {
            Zr[(int64_t)i * k + t] = zn;
            Zr[(int64_t)(i + 1) * k + t] = zi - f * zn;
          } else {
            Zr[(int64_t)(i + 1) * k + t] = zn - f * zi;
          }
        }
        R zmax = 0;
        for (int i = n - 1; i >= 0; --i) {
          R v = Zr[(int64_t)i * k + t];
          if (i + 1 < n) v -= Ldu[(int64_t)i * k + t] * Zr[(int64_t)(i + 1) * k + t];
          if (i + 2 < n) v -= Ldu2[(int64_t)i * k + t] * Zr[(int64_t)(i + 2) * k + t];
          v *= Ldd[(int64_t)i * k + t];
          if (!(fabs(v) < R(1e30))) v = (v > 0) ? R(1e30) : R(-1e30);
          Zr[(int64_t)i * k + t] = v;
          zmax = fmax(zmax, fabs(v));
        }
        R sc = (zmax > R(0)) ? R(1) / zmax : R(1);
        for (int i = 0; i < n; ++i) Zr[(int64_t)i * k + t] *= sc;
      }
      __syncthreads();
    }
  }
  }

  // ---- (5) back-transformation u = H_0 ... H_{n-3} Phi z for all k vectors at once, NB reflectors
  // per panel (last panel first), each panel applied as one block reflector I - V T V^H
  __shared__ cplx<R> s_T[NB * NB], s_S[NB * NB];
  for (int64_t e = tid; e < (int64_t)n * k; e += NT) {
    const int i = (int)(e % n), t = (int)(e / n);
    U[e] = Zr[(int64_t)i * k + t] * PH[i];
  }
  __syncthreads();
  const int nref = n - 2;  // reflectors H_0 .. H_{n-3}
  for (int j0 = ((nref - 1) / NB) * NB; nref > 0 && j0 >= 0; j0 -= NB) {
    const int pb = (nref - j0 < NB) ? nref - j0 : NB;
    const int r0 = j0 + 1, M = n - r0;  // rows touched by the panel
    // V panel: reflector j0 + l as column l (rows relative to r0): v_{j+1} = v0, v_i = A[j][i] below
    for (int e = tid; e < pb * M; e += NT) {
      const int l = e / M, r = e % M, i = r0 + r, j = j0 + l;
      cplx<R> v = mk<R>(0, 0);
      if (i == j + 1) v = s_v0[j];
      else if (i > j + 1) v = A[(int64_t)j * n + i];
      Vb[l * n + r] = v;
    }
    __syncthreads();
    // T: S[l][m] = v_l^H v_m (l < m), T_mm = beta_m, T[0:m, m] = -beta_m T[0:m, 0:m] S[0:m, m]
    for (int pr = wid; pr < pb * pb; pr += NT / 32) {
      const int l = pr / pb, m = pr % pb;
      if (l >= m) continue;
      cplx<R> acc = mk<R>(0, 0);
      for (int r = m + lane; r < M; r += 32) cfma_cj(acc, Vb[l * n + r], Vb[m * n + r]);
      acc = panel::warp_csum(acc);
      if (lane == 0) s_S[l * NB + m] = acc;
    }
    __syncthreads();
    for (int m = 0; m < NB; ++m) {
      if (tid < NB) {
        const int l = tid;
        cplx<R> tv = mk<R>(0, 0);
        if (m < pb && l < m) {
          cplx<R> acc = mk<R>(0, 0);
          for (int q = l; q < m; ++q) cfma(acc, s_T[l + q * NB], s_S[q * NB + m]);
          tv = -s_beta[j0 + m] * acc;
        } else if (m < pb && l == m) {
          tv = mk<R>(s_beta[j0 + m], 0);
        }
        s_T[l + m * NB] = tv;
      }
      __syncthreads();
    }
    // U[r0:, :] <- (I - V T V^H) U[r0:, :]
    panel::panel_vh_times<R, NB>(U + r0, n, M, k, Vb, n, pb, Wb, n);
    __syncthreads();
    panel::panel_apply_t<R, NB>(s_T, pb, false, Wb, n, k);
    __syncthreads();
    panel::panel_minus_v_times<R, NB>(U + r0, n, M, k, Vb, n, pb, Wb, n);
    __syncthreads();
  }

  // ---- outputs
  GPTR(cplx<R>, V, g.V + view_batch(g.vv, z));
  for (int64_t e = tid; e < (int64_t)n * k; e += NT) {
    int i = (int)(e % n), t = (int)(e / n);
    cplx<R> v = U[(int64_t)t * n + i];
    if (g.vv.conj) v.y = -v.y;
    V[view_row(g.vv, i) + view_col(g.vv, t)] = v;
  }
  if (g.w) {
    GPTR(R, w, g.w + (int64_t)z * g.wstride);
    for (int t = tid; t < k; t += NT) w[t] = ldexp(s_w[t], s_exp);
  }
  // non-finite eigenvalues, trace or eigenvector entries (from non-finite input: the inverse
  // iteration's growth guard keeps finite inputs finite) are reported as non-convergence
  for (int64_t e = tid; e < (int64_t)n * k; e += NT) {
    const cplx<R> v = U[e];
    if (!isfinite((double)v.x) || !isfinite((double)v.y)) s_bad = 1;
  }
  __syncthreads();
  if (tid == 0) {
    double kept = 0;
    for (int t = 0; t < k; ++t) kept += (double)s_w[t];
    if (g.status && (s_bad || !isfinite(kept) || !isfinite((double)trace))) atomicOr(GP(g.status), kStatusNoConv);
    double tr = (double)trace;
    if (g.disc && tr > 0) {
      double w = (tr - kept) / tr;
      if (w < 0) w = 0;
      GX(g.disc, (int64_t)z * g.disc_stride) += w;
    }
    if (g.gap && k < n && s_w[0] > R(0)) {
      double gp = ((double)s_w[k - 1] - (double)s_w[k]) / (double)s_w[0];
      double* gz = GP(g.gap + (int64_t)z * g.disc_stride);
      if (gp < *gz) *gz = gp;
    }
  }
}
}  // namespace

int64_t eig_scratch_elems(int n, int k) { return 8 * (int64_t)n * k + 2 * (int64_t)n + 64; }

template <typename R>
cudaError_t heevk(cudaStream_t s, int batch, const EigArgs<R>& g) {
  if (batch <= 0 || g.n <= 0 || g.k <= 0) return cudaSuccess;
  if (g.n > MAXN || g.k > g.n || g.k + 1 > MAXN / 2) return cudaErrorInvalidValue;
  // reflectors per panel (tridiagonalisation and back-transformation); FP64 takes 4 so that two
  // matrices share an SM and fill each other's barrier waits on the narrow FP64 pipe
  constexpr int NB = sizeof(R) == 8 ? 4 : 8;
  const size_t bytes = 2 * sizeof(cplx<R>) * (size_t)NB * g.n + sizeof(R) * (size_t)GB * g.k;
  static PerDevice setup;
  static size_t dyn_max[kMaxDevices];
  int dev = 0;
  cudaError_t e = setup.once([](int d) {
    cudaFuncAttributes fa;
    cudaError_t r = cudaFuncGetAttributes(&fa, heevk_kernel<R, NB>);
    if (r != cudaSuccess) return r;
    const size_t want = 2 * sizeof(cplx<R>) * NB * MAXN + sizeof(R) * GB * (MAXN / 2);
    const size_t cap = 227 * 1024 - fa.sharedSizeBytes;
    dyn_max[d] = want < cap ? want : cap;
    return cudaFuncSetAttribute(heevk_kernel<R, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max[d]);
  });
  if (e != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (bytes > dyn_max[dev]) return cudaErrorInvalidValue;
  heevk_kernel<R, NB><<<batch, NT, bytes, s>>>(g);
  return cudaGetLastError();
}

template cudaError_t heevk<float>(cudaStream_t, int, const EigArgs<float>&);
template cudaError_t heevk<double>(cudaStream_t, int, const EigArgs<double>&);

}  // namespace mpdo
