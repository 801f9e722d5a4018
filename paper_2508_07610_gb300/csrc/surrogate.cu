// Learned surrogate for the variational loop: an MLP (in -> H -> ... -> H -> out, GELU) trained with
// mean-squared error and AdamW.  Weights and activations are stored in BF16; every product is
// accumulated in FP32; FP32 master weights and AdamW moments are kept for the update.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include <cmath>
#include <new>
#include <vector>

#include "surrogate.h"
#include "surrogate_tc.h"

namespace {
constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

// C[i][j] (+)= sum_k A(i, k) B(k, j); A(i, k) = A[i*as0 + k*as1], B(k, j) = B[k*bs0 + j*bs1].
template <typename TA, typename TB>
__global__ void __launch_bounds__(NT) gemm_f32acc(int M, int N, int K, const TA* A, int64_t as0, int64_t as1,
                                                  const TB* B, int64_t bs0, int64_t bs1, float* C, int64_t ldc,
                                                  int accumulate, int kc, float* ws) {
  __shared__ float As[TK][TM + 1];
  __shared__ float Bs[TK][TN + 1];
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  // K chunk of this CTA (split-K: blockIdx.z chunks of kc, partial tiles to ws)
  const int kb = blockIdx.z * kc, ke = (K - kb < kc) ? K : kb + kc;
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += NT) {
      int i = e / TK, kk = e % TK;
      int gi = m0 + i, gk = k0 + kk;
      As[kk][i] = (gi < M && gk < ke) ? to_f(A[gi * as0 + gk * as1]) : 0.f;
    }
    for (int e = threadIdx.x; e < TN * TK; e += NT) {
      int j = e % TN, kk = e / TN;
      int gj = n0 + j, gk = k0 + kk;
      Bs[kk][j] = (gj < N && gk < ke) ? to_f(B[gk * bs0 + gj * bs1]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  for (int r = 0; r < 4; ++r) {
    int i = m0 + ty + 16 * r;
    if (i >= M) continue;
    for (int c = 0; c < 4; ++c) {
      int j = n0 + tx + 16 * c;
      if (j >= N) continue;
      float v = acc[r][c];
      if (ws) {
        ws[((int64_t)blockIdx.z * M + i) * N + j] = v;
        continue;
      }
      if (accumulate) v += C[(int64_t)i * ldc + j];
      C[(int64_t)i * ldc + j] = v;
    }
  }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  // d/dz [z Phi(z)] = Phi(z) + z phi(z)
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Z[b][o] += bias[o]; H = GELU(Z) (BF16) or, for the output layer, Z itself
__global__ void bias_act(int Bn, int O, float* Z, const float* bias, __nv_bfloat16* H, int act) {
  int64_t total = (int64_t)Bn * O;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int o = (int)(e % O);
    float z = Z[e] + bias[o];
    Z[e] = z;
    if (act) H[e] = __float2bfloat16(gelu(z));
  }
}

// dZ = dH * GELU'(Z)
__global__ void act_back(int64_t total, const float* Z, float* dH) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    dH[e] *= gelu_grad(Z[e]);
}

// mean-squared error over Bn x O: loss partial sums and dY = 2 (Y - T) / (Bn * O)
__global__ void mse(int Bn, int O, const float* Y, const float* T, float* dY, double* loss) {
  __shared__ double red[NT / 32];
  int64_t total = (int64_t)Bn * O;
  double s = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float d = Y[e] - T[e];
    dY[e] = 2.f * d / (float)total;
    s += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    atomicAdd(loss, t / (double)total);
  }
}

// db[o] = sum_b dZ[b][o]
__global__ void bias_grad(int Bn, int O, const float* dZ, float* db) {
  int o = blockIdx.x;
  float s = 0;
  for (int b = threadIdx.x; b < Bn; b += blockDim.x) s += dZ[(int64_t)b * O + o];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    db[o] = t;
  }
}

// AdamW (decoupled weight decay): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * (mhat / (sqrt(vhat) + eps) + wd * p)
__global__ void adamw(int64_t count, float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, float lr,
                      float b1, float b2, float eps, float wd, float c1, float c2, int decay) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    float gi = g[e];
    float mi = b1 * m[e] + (1.f - b1) * gi;
    float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    float mh = mi / c1, vh = vi / c2;
    float pi = p[e];
    pi -= lr * (mh / (sqrtf(vh) + eps) + (decay ? wd * pi : 0.f));
    p[e] = pi;
    if (pb) pb[e] = __float2bfloat16(pi);
  }
}

__global__ void to_bf16(int64_t count, const float* x, __nv_bfloat16* y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = __float2bfloat16(x[e]);
}

inline int grid_for(int64_t n) {
  int64_t b = (n + NT - 1) / NT;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

// C (+)= the sum of the sk partial tiles, added in a fixed order (deterministic)
__global__ void splitk_sum(int M, int N, int sk, const float* ws, float* C, int64_t ldc, int accumulate) {
  const int64_t MN = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int t = 0; t < sk; ++t) v += ws[t * MN + e];
    const int64_t o = (e / N) * ldc + e % N;
    C[o] = accumulate ? C[o] + v : v;
  }
}

// ws (nullable, ws_elems floats): workspace for split-K, used when the output has too few tiles for
// the GPU and K is long (the weight gradients: 256 x 256 over the batch)
template <typename TA, typename TB>
cudaError_t gemm(cudaStream_t s, int M, int N, int K, const TA* A, int64_t as0, int64_t as1, const TB* B, int64_t bs0,
                 int64_t bs1, float* C, int64_t ldc, int accumulate, float* ws = nullptr, int64_t ws_elems = 0) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int tiles = ((N + TN - 1) / TN) * ((M + TM - 1) / TM);
  int sk = 1;
  if (ws && K >= 1024 && tiles < 304) {
    sk = (304 + tiles - 1) / tiles;
    if (sk > K / 256) sk = K / 256;
    if (sk > 16) sk = 16;
    while (sk > 1 && (int64_t)sk * M * N > ws_elems) --sk;
    if (sk < 1) sk = 1;
  }
  const int kc = (sk > 1) ? ((K + sk - 1) / sk + TK - 1) / TK * TK : (K > 0 ? K : 1);
  if (sk > 1) sk = (K + kc - 1) / kc;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, sk);
  gemm_f32acc<TA, TB><<<grid, NT, 0, s>>>(M, N, K, A, as0, as1, B, bs0, bs1, C, ldc, accumulate, kc,
                                          sk > 1 ? ws : nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || sk == 1) return e;
  const int64_t mn = (int64_t)M * N;
  splitk_sum<<<(unsigned)((mn + NT - 1) / NT < 1024 ? (mn + NT - 1) / NT : 1024), NT, 0, s>>>(M, N, sk, ws, C, ldc,
                                                                                               accumulate);
  return cudaGetLastError();
}
}  // namespace

struct surr_ctx {
  int in = 0, hid = 0, layers = 0, out = 0, cap = 0;
  cudaStream_t stream = nullptr;
  std::vector<int> dims;                     // layers + 1 entries
  std::vector<int64_t> woff, boff;           // offsets of W_l and b_l in the parameter vector
  int64_t nparam = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master params, grads, moments
  __nv_bfloat16* pb = nullptr;                                   // BF16 copy of the parameters
  __nv_bfloat16* xb = nullptr;                                   // BF16 input batch
  std::vector<float*> Z;                                         // pre-activations per layer (FP32)
  std::vector<__nv_bfloat16*> H;                                 // activations per layer (BF16)
  float *d0 = nullptr, *d1 = nullptr;                            // gradient ping-pong buffers
  float* ws = nullptr;                                           // split-K partials of the weight gradients
  int64_t ws_elems = 0;
  double* dloss = nullptr;
  long long step = 0;
  ~surr_ctx() {
    void* ptrs[] = {p, g, m, v, pb, xb, d0, d1, ws, dloss};
    for (void* q : ptrs)
      if (q) cudaFree(q);
    for (auto* q : Z) cudaFree(q);
    for (auto* q : H) cudaFree(q);
  }
};

namespace {
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

surr_status forward(surr_ctx* c, const float* X, int Bn) {
  cudaStream_t s = c->stream;
  to_bf16<<<grid_for((int64_t)Bn * c->in), NT, 0, s>>>((int64_t)Bn * c->in, X, c->xb);
  if (cudaGetLastError() != cudaSuccess) return SURR_ECUDA;
  const __nv_bfloat16* act = c->xb;
  for (int l = 0; l < c->layers; ++l) {
    int I = c->dims[l], O = c->dims[l + 1];
    const __nv_bfloat16* W = c->pb + c->woff[l];
    // Z = act W^T  (act: Bn x I, W: O x I): on the tensor cores where the shape allows (the hidden
    // layers), else on CUDA cores (the 2-wide output layer)
    if (surr_tc::applicable(O, I, act, W)) {
      if (surr_tc::linear(s, Bn, O, I, act, W, c->Z[l]) != cudaSuccess) return SURR_ECUDA;
    } else if (gemm(s, Bn, O, I, act, (int64_t)I, (int64_t)1, W, (int64_t)1, (int64_t)I, c->Z[l], (int64_t)O, 0) !=
               cudaSuccess) {
      return SURR_ECUDA;
    }
    int last = (l == c->layers - 1);
    bias_act<<<grid_for((int64_t)Bn * O), NT, 0, s>>>(Bn, O, c->Z[l], c->p + c->boff[l], c->H[l], last ? 0 : 1);
    if (cudaGetLastError() != cudaSuccess) return SURR_ECUDA;
    act = c->H[l];
  }
  return SURR_OK;
}
}  // namespace

extern "C" {

surr_status surr_create(int in_dim, int hidden, int n_hidden, int out_dim, int max_batch, unsigned long long seed,
                        void* stream, surr_t* out) {
  if (!out || in_dim < 1 || hidden < 1 || n_hidden < 1 || out_dim < 1 || max_batch < 1) return SURR_EINVAL;
  surr_ctx* c = new (std::nothrow) surr_ctx();
  if (!c) return SURR_ENOMEM;
  c->in = in_dim;
  c->hid = hidden;
  c->layers = n_hidden + 1;
  c->out = out_dim;
  c->cap = max_batch;
  c->stream = (cudaStream_t)stream;
  c->dims.push_back(in_dim);
  for (int l = 0; l < n_hidden; ++l) c->dims.push_back(hidden);
  c->dims.push_back(out_dim);
  for (int l = 0; l < c->layers; ++l) {
    c->woff.push_back(c->nparam);
    c->nparam += (int64_t)c->dims[l] * c->dims[l + 1];
    c->boff.push_back(c->nparam);
    c->nparam += c->dims[l + 1];
  }
  // He-style uniform initialisation from a counter-based generator; biases zero
  std::vector<float> h((size_t)c->nparam, 0.f);
  uint64_t st = seed;
  for (int l = 0; l < c->layers; ++l) {
    float a = std::sqrt(6.f / (float)c->dims[l]) * (l == c->layers - 1 ? 0.5f : 1.f);
    for (int64_t e = 0; e < (int64_t)c->dims[l] * c->dims[l + 1]; ++e) {
      double u = (double)(splitmix(st) >> 11) / 9007199254740992.0;
      h[c->woff[l] + e] = (float)((2 * u - 1) * a);
    }
  }
  bool ok = cudaMalloc(&c->p, sizeof(float) * c->nparam) == cudaSuccess &&
            cudaMalloc(&c->g, sizeof(float) * c->nparam) == cudaSuccess &&
            cudaMalloc(&c->m, sizeof(float) * c->nparam) == cudaSuccess &&
            cudaMalloc(&c->v, sizeof(float) * c->nparam) == cudaSuccess &&
            cudaMalloc(&c->pb, sizeof(__nv_bfloat16) * c->nparam) == cudaSuccess &&
            cudaMalloc(&c->xb, sizeof(__nv_bfloat16) * (size_t)max_batch * in_dim) == cudaSuccess &&
            cudaMalloc(&c->d0, sizeof(float) * (size_t)max_batch * std::max(hidden, out_dim)) == cudaSuccess &&
            cudaMalloc(&c->d1, sizeof(float) * (size_t)max_batch * std::max(hidden, out_dim)) == cudaSuccess &&
            cudaMalloc(&c->dloss, sizeof(double)) == cudaSuccess;
  {
    int64_t wmax = 0;
    for (int l = 0; l < c->layers; ++l) wmax = std::max<int64_t>(wmax, (int64_t)c->dims[l] * c->dims[l + 1]);
    c->ws_elems = 16 * wmax;
    ok = ok && cudaMalloc(&c->ws, sizeof(float) * c->ws_elems) == cudaSuccess;
  }
  for (int l = 0; ok && l < c->layers; ++l) {
    float* z = nullptr;
    __nv_bfloat16* a = nullptr;
    ok = cudaMalloc(&z, sizeof(float) * (size_t)max_batch * c->dims[l + 1]) == cudaSuccess &&
         cudaMalloc(&a, sizeof(__nv_bfloat16) * (size_t)max_batch * c->dims[l + 1]) == cudaSuccess;
    c->Z.push_back(z);
    c->H.push_back(a);
  }
  if (!ok) {
    delete c;
    return SURR_ENOMEM;
  }
  if (cudaMemcpy(c->p, h.data(), sizeof(float) * c->nparam, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->m, 0, sizeof(float) * c->nparam) != cudaSuccess ||
      cudaMemset(c->v, 0, sizeof(float) * c->nparam) != cudaSuccess) {
    delete c;
    return SURR_ECUDA;
  }
  to_bf16<<<grid_for(c->nparam), NT, 0, c->stream>>>(c->nparam, c->p, c->pb);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) {
    delete c;
    return SURR_ECUDA;
  }
  *out = c;
  return SURR_OK;
}

surr_status surr_free(surr_t c) {
  if (!c) return SURR_EINVAL;
  cudaStreamSynchronize(c->stream);
  delete c;
  return SURR_OK;
}

long long surr_num_params(surr_t c) { return c ? c->nparam : -1; }

surr_status surr_get_params(surr_t c, float* host) {
  if (!c || !host) return SURR_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(host, c->p, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SURR_ECUDA;
  return SURR_OK;
}

surr_status surr_set_params(surr_t c, const float* host) {
  if (!c || !host) return SURR_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(c->p, host, sizeof(float) * c->nparam, cudaMemcpyHostToDevice) != cudaSuccess)
    return SURR_ECUDA;
  to_bf16<<<grid_for(c->nparam), NT, 0, c->stream>>>(c->nparam, c->p, c->pb);
  return cudaGetLastError() == cudaSuccess ? SURR_OK : SURR_ECUDA;
}

surr_status surr_forward(surr_t c, const float* X_dev, int batch, float* Y_dev) {
  if (!c || !X_dev || !Y_dev || batch < 1 || batch > c->cap) return SURR_EINVAL;
  surr_status st = forward(c, X_dev, batch);
  if (st) return st;
  const int64_t n = (int64_t)batch * c->out;
  return cudaMemcpyAsync(Y_dev, c->Z[c->layers - 1], sizeof(float) * n, cudaMemcpyDeviceToDevice, c->stream) ==
                 cudaSuccess
             ? SURR_OK
             : SURR_ECUDA;
}

surr_status surr_gradients(surr_t c, const float* X_dev, const float* T_dev, int batch, double* loss_host) {
  if (!c || !X_dev || !T_dev || batch < 1 || batch > c->cap) return SURR_EINVAL;
  cudaStream_t s = c->stream;
  surr_status st = forward(c, X_dev, batch);
  if (st) return st;
  if (cudaMemsetAsync(c->dloss, 0, sizeof(double), s) != cudaSuccess) return SURR_ECUDA;
  const int L = c->layers;
  float* dcur = c->d0;
  float* dnext = c->d1;
  mse<<<grid_for((int64_t)batch * c->out), NT, 0, s>>>(batch, c->out, c->Z[L - 1], T_dev, dcur, c->dloss);
  if (cudaGetLastError() != cudaSuccess) return SURR_ECUDA;
  for (int l = L - 1; l >= 0; --l) {
    const int I = c->dims[l], O = c->dims[l + 1];
    const __nv_bfloat16* X = (l == 0) ? c->xb : c->H[l - 1];
    // dW = dZ^T X  (O x I), db = column sums of dZ
    if (gemm(s, O, I, batch, dcur, (int64_t)1, (int64_t)O, X, (int64_t)I, (int64_t)1, c->g + c->woff[l], (int64_t)I,
             0, c->ws, c->ws_elems) != cudaSuccess)
      return SURR_ECUDA;
    bias_grad<<<O, 256, 0, s>>>(batch, O, dcur, c->g + c->boff[l]);
    if (cudaGetLastError() != cudaSuccess) return SURR_ECUDA;
    if (l > 0) {
      // dX = dZ W (batch x I), then through GELU of the previous layer
      if (gemm(s, batch, I, O, dcur, (int64_t)O, (int64_t)1, c->pb + c->woff[l], (int64_t)I, (int64_t)1, dnext,
               (int64_t)I, 0) != cudaSuccess)
        return SURR_ECUDA;
      act_back<<<grid_for((int64_t)batch * I), NT, 0, s>>>((int64_t)batch * I, c->Z[l - 1], dnext);
      if (cudaGetLastError() != cudaSuccess) return SURR_ECUDA;
      float* t = dcur;
      dcur = dnext;
      dnext = t;
    }
  }
  if (loss_host) {
    if (cudaMemcpyAsync(loss_host, c->dloss, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return SURR_ECUDA;
  }
  return SURR_OK;
}

surr_status surr_get_grads(surr_t c, float* host) {
  if (!c || !host) return SURR_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(host, c->g, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SURR_ECUDA;
  return SURR_OK;
}

surr_status surr_adamw(surr_t c, float lr, float beta1, float beta2, float eps, float weight_decay) {
  if (!c) return SURR_EINVAL;
  c->step += 1;
  const float c1 = 1.f - std::pow(beta1, (float)c->step), c2 = 1.f - std::pow(beta2, (float)c->step);
  // weights decay, biases do not
  for (int l = 0; l < c->layers; ++l) {
    int64_t nw = (int64_t)c->dims[l] * c->dims[l + 1], nb = c->dims[l + 1];
    adamw<<<grid_for(nw), NT, 0, c->stream>>>(nw, c->p + c->woff[l], c->g + c->woff[l], c->m + c->woff[l],
                                                c->v + c->woff[l], c->pb + c->woff[l], lr, beta1, beta2, eps,
                                                weight_decay, c1, c2, 1);
    adamw<<<grid_for(nb), NT, 0, c->stream>>>(nb, c->p + c->boff[l], c->g + c->boff[l], c->m + c->boff[l],
                                                c->v + c->boff[l], c->pb + c->boff[l], lr, beta1, beta2, eps,
                                                weight_decay, c1, c2, 0);
  }
  return cudaGetLastError() == cudaSuccess ? SURR_OK : SURR_ECUDA;
}

surr_status surr_train_step(surr_t c, const float* X_dev, const float* T_dev, int batch, float lr, float weight_decay,
                            double* loss_host) {
  surr_status st = surr_gradients(c, X_dev, T_dev, batch, loss_host);
  if (st) return st;
  return surr_adamw(c, lr, 0.9f, 0.999f, 1e-8f, weight_decay);
}

surr_status surr_sync(surr_t c) {
  if (!c) return SURR_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SURR_ECUDA;
  int fail = 0;
  if (surr_tc::read_fail_flag(&fail) != cudaSuccess || fail) return SURR_ECUDA;
  return SURR_OK;
}

}  // extern "C"
