// Complex64 GEMM on the 5th-generation tensor cores (tcgen05.mma kind::tf32, accumulators in tensor
// memory) with FP32-level accuracy, for the dense contractions of the two-site update.
//
//   C[z](i, j) = alpha * sum_k opA[z](i, k) opB[z](k, j) + beta * C[z](i, j)
//
// Precision.  Each FP32 operand x is split into x_hi = tf32(x) and x_lo = tf32(x - x_hi), and a real
// product is taken as hi*hi + hi*lo + lo*hi (the dropped lo*lo term and the residual of the split are
// about 2^-22 of the product, with random signs).  A complex product is four real products
// (Re = ArBr - AiBi with the tensor core's negate-A bit, Im = ArBi + AiBr): 12 MMAs per k-step of 8.
// The tensor core rounds its FP32 accumulator once per MMA, so TMEM accumulates only one k-block of
// 16 at a time: a fresh partial that eight fold warps add into FP32 register sums with Knuth's TwoSum,
// which keeps the error of long sums at the level of the compensated CUDA-core GEMM.
//
// Data movement.  A pre-pass reads both operands through their strided views once and writes the
// hi/lo planes, conjugation applied, already in the tensor core's K-major core-matrix layout (8 rows x
// 16 bytes per core matrix), tile by tile: one pipeline stage (a 128 x 8 tile of A, a 64 x 8 tile of
// B, four planes each, 24 KB) is one contiguous chunk that the TMA engine moves with two
// cp.async.bulk copies completing on an mbarrier.  No operand passes through registers in the GEMM.
//
// Roles in a CTA (one 128 x 64 output tile): warp 0 issues the bulk copies into a ring of STAGES
// stages, warp 1 owns the tensor memory (two partial buffers of 64 + 64 columns) and one of its
// threads issues the MMAs, warps 2-9 fold the partials and write the tile through the output view.
// Every mbarrier wait is bounded in time: on timeout the CTA records kStatusTimeout, stops issuing,
// waits (bounded) for what it already issued, frees its tensor memory and skips its output.
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "device_once.cuh"
#include "kernels.h"
#include "mpdo.h"
#include "wait.cuh"

namespace mpdo {

namespace {
constexpr int TM = 128, TN = 64, TK = 8;       // output tile, k-step of one MMA
constexpr int KSB = 2;                         // k-steps per folded block (16 k)
constexpr int STAGES = 4;
constexpr int NWARPS = 10, NTH = NWARPS * 32;  // producer, MMA, 8 fold warps
constexpr int NFOLD = (NWARPS - 2) * 32;
constexpr int A_PLANE = TM * TK * 4;           // 4 KB: one 128 x 8 TF32 plane
constexpr int B_PLANE = TN * TK * 4;           // 2 KB
constexpr int A_STAGE = 4 * A_PLANE, B_STAGE = 4 * B_PLANE;
constexpr int STAGE_BYTES = A_STAGE + B_STAGE;  // 24 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr int TMEM_COLS = 256;                 // two partial buffers x (64 re + 64 im)

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// byte offset of (row, k) inside one K-major plane of 8 columns: core matrices of 8 rows x 16 bytes,
// the two k-halves 128 bytes apart (leading-dimension offset), row groups 256 bytes apart (stride)
__host__ __device__ __forceinline__ int core_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 256;
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of tcgen05
  return d;                // base offset 0, no swizzle
}
// kind::tf32 instruction descriptor: D F32, A and B TF32, both K-major, M = TM, N = TN
__device__ __forceinline__ uint32_t instr_desc(int negate_a) {
  uint32_t d = 0;
  d |= 1u << 4;                    // D format F32
  d |= 2u << 7;                    // A format TF32
  d |= 2u << 10;                   // B format TF32
  d |= (uint32_t)negate_a << 13;   // negate A
  d |= (uint32_t)(TN >> 3) << 17;  // N / 8
  d |= (uint32_t)(TM >> 4) << 24;  // M / 16
  return d;
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
// TMA 1-D bulk copy global -> shared, completion counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
// 32 consecutive 32-bit TMEM columns of the warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t addr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// Bounded wait taken by lane 0 and broadcast, so the lanes of a warp that goes on to warp-collective
// tcgen05 instructions never diverge on a timeout.
__device__ __forceinline__ bool warp_wait(uint32_t mbar, uint32_t parity) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_bounded(mbar, parity) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}
__device__ __forceinline__ void two_sum_add(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  s = t;
  c = __fadd_rn(c, err);
}

// ---- pre-pass: operand -> hi/lo TF32 planes in tiles of (rows_per_tile x 8 k), four planes per tile
// (re_hi, re_lo, im_hi, im_lo); tile (z, rt, ks) starts at ((z * RT + rt) * KS + ks) * 4 planes.
// A (transpose = 0): rows i of op(A) (M x K).  B (transpose = 1): columns j of op(B) (K x N), K-major.
// Outside the matrix the planes hold zeros.  The index order follows the operand's contiguous
// direction (k for A's rows, j for B's columns of a row-major site), so reads coalesce.
__global__ void tc_split_kernel(int rows, int K, int rows_per_tile, int RT, int KS, const cplx<float>* src,
                                View v, int transpose, float* dst) {
  const int z = blockIdx.y;
  const cplx<float>* S = src + view_batch(v, z);
  const int plane = rows_per_tile * TK;  // floats per plane
  const int64_t per_z = (int64_t)RT * KS * 4 * plane;
  const int rows_pad = RT * rows_per_tile, k_pad = KS * TK;
  const int64_t total = (int64_t)rows_pad * k_pad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int r, k;
    if (transpose) {
      r = (int)(e % rows_pad);
      k = (int)(e / rows_pad);
    } else {
      k = (int)(e % k_pad);
      r = (int)(e / k_pad);
    }
    cplx<float> x = mk<float>(0.f, 0.f);
    if (r < rows && k < K) {
      x = transpose ? GX(S, view_row(v, k) + view_col(v, r)) : GX(S, view_row(v, r) + view_col(v, k));
      if (v.conj) x.y = -x.y;
    }
    const float rh = tf32_rna(x.x), ih = tf32_rna(x.y);
    const int rt = r / rows_per_tile, rr = r % rows_per_tile, ks = k / TK, kk = k % TK;
    float* T = dst + per_z * z + ((int64_t)rt * KS + ks) * 4 * plane;
    const int o = core_off(rr, kk) / 4;
    GX(T, o) = rh;
    GX(T, plane + o) = tf32_rna(x.x - rh);
    GX(T, 2 * plane + o) = ih;
    GX(T, 3 * plane + o) = tf32_rna(x.y - ih);
  }
}

struct TcParams {
  int M, N, K, MT, NT, KS;
  const float* Ap;  // A planes
  const float* Bp;  // B planes
  cplx<float> alpha, beta;
  cplx<float>* C;
  View vc;
  int herm;
  int* status;
};

__global__ void __launch_bounds__(NTH, 1) tc_cgemm_kernel(TcParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;                // [STAGES] producer -> MMA (bytes)
  uint64_t* empty = bars + STAGES;      // [STAGES] MMA commit -> producer
  uint64_t* pfull = bars + 2 * STAGES;  // [2] MMA commit -> fold warps
  uint64_t* pempty = pfull + 2;         // [2] fold warps (NFOLD arrivals) -> MMA
  uint64_t* done = pempty + 2;          // [1] final commit (drain before freeing TMEM)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* s_fail = reinterpret_cast<int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = blockIdx.x, mt = blockIdx.y, z = blockIdx.z;
  if (p.herm && nt * TN > mt * TM + TM - 1) return;  // tile strictly above the diagonal of a Hermitian result

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_addr(&full[s]), 1);
      mbar_init(smem_addr(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_addr(&pfull[b]), 1);
      mbar_init(smem_addr(&pempty[b]), NFOLD);
    }
    mbar_init(smem_addr(done), 1);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int KS = p.KS, NB = (KS + KSB - 1) / KSB;
  const unsigned char* Abase = reinterpret_cast<const unsigned char*>(p.Ap) + ((int64_t)z * p.MT + mt) * KS * A_STAGE;
  const unsigned char* Bbase = reinterpret_cast<const unsigned char*>(p.Bp) + ((int64_t)z * p.NT + nt) * KS * B_STAGE;
  // fold state of a thread of warps 2..9: row 32 (warp % 4) + lane, columns 32 h .. 32 h + 31
  const int q = warp & 3, h = (warp - 2) >> 2;
  float sre[32], sim[32], cre[32], cim[32];

  if (warp == 0) {
    if (lane == 0) {  // producer: one 16 KB and one 8 KB bulk copy per k-step
      int issued = 0;
      for (int ks = 0; ks < KS; ++ks) {
        const int s = ks % STAGES;
        if (ks >= STAGES && !mbar_wait_bounded(smem_addr(&empty[s]), ((ks / STAGES) - 1) & 1)) {
          atomicExch(s_fail, 1);
          break;
        }
        if (*(volatile int*)s_fail) break;
        const uint32_t fb = smem_addr(&full[s]);
        const uint32_t dst = smem_addr(smem + s * STAGE_BYTES);
        mbar_expect_tx(fb, STAGE_BYTES);
        bulk_g2s(dst, GRANGE(Abase + (int64_t)ks * A_STAGE, A_STAGE), A_STAGE, fb);
        bulk_g2s(dst + A_STAGE, GRANGE(Bbase + (int64_t)ks * B_STAGE, B_STAGE), B_STAGE, fb);
        issued = ks + 1;
      }
      // every copy in flight has landed before the shared memory is given up (each stage's last phase)
      for (int ks = issued - STAGES < 0 ? 0 : issued - STAGES; ks < issued; ++ks)
        if (!mbar_wait_bounded(smem_addr(&full[ks % STAGES]), (ks / STAGES) & 1)) atomicExch(s_fail, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t pos = instr_desc(0), neg = instr_desc(1);
      bool ok = true;
      for (int kb = 0; kb < NB && ok; ++kb) {
        const int buf = kb & 1;
        if (kb >= 2 && !mbar_wait_bounded(smem_addr(&pempty[buf]), ((kb >> 1) - 1) & 1)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dre = tmem + buf * 128, dim = dre + 64;
        for (int j = 0; j < KSB; ++j) {
          const int ks = kb * KSB + j;
          if (ks >= KS) break;
          const int s = ks % STAGES;
          if (!mbar_wait_bounded(smem_addr(&full[s]), (ks / STAGES) & 1)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a = smem_addr(smem + s * STAGE_BYTES), b = a + A_STAGE;
          const uint64_t arh = smem_desc(a), arl = smem_desc(a + A_PLANE), aih = smem_desc(a + 2 * A_PLANE),
                         ail = smem_desc(a + 3 * A_PLANE);
          const uint64_t brh = smem_desc(b), brl = smem_desc(b + B_PLANE), bih = smem_desc(b + 2 * B_PLANE),
                         bil = smem_desc(b + 3 * B_PLANE);
          const uint32_t acc = j > 0 ? 1u : 0u;  // a fresh partial at the start of every block
          // Re += Ar Br - Ai Bi
          mma_tf32(dre, arh, brh, pos, acc);
          mma_tf32(dre, arh, brl, pos, 1);
          mma_tf32(dre, arl, brh, pos, 1);
          mma_tf32(dre, aih, bih, neg, 1);
          mma_tf32(dre, aih, bil, neg, 1);
          mma_tf32(dre, ail, bih, neg, 1);
          // Im += Ar Bi + Ai Br
          mma_tf32(dim, arh, bih, pos, acc);
          mma_tf32(dim, arh, bil, pos, 1);
          mma_tf32(dim, arl, bih, pos, 1);
          mma_tf32(dim, aih, brh, pos, 1);
          mma_tf32(dim, aih, brl, pos, 1);
          mma_tf32(dim, ail, brh, pos, 1);
          mma_commit(smem_addr(&empty[s]));  // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        mma_commit(smem_addr(&pfull[buf]));  // the block's partial is complete
      }
      if (!ok) atomicExch(s_fail, 1);
      // drain: every MMA issued so far is complete when this commit arrives
      mma_commit(smem_addr(done));
      if (!mbar_wait_bounded(smem_addr(done), 0)) atomicExch(s_fail, 1);
    }
    __syncwarp();
  } else {
#pragma unroll
    for (int c = 0; c < 32; ++c) sre[c] = sim[c] = cre[c] = cim[c] = 0.f;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    for (int kb = 0; kb < NB; ++kb) {
      const int buf = kb & 1;
      if (!warp_wait(smem_addr(&pfull[buf]), (kb >> 1) & 1)) {
        if (lane == 0) atomicExch(s_fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float part[32];
      tmem_ld32(tmem + lane_base + buf * 128 + h * 32, part);
#pragma unroll
      for (int c = 0; c < 32; ++c) two_sum_add(sre[c], cre[c], part[c]);
      tmem_ld32(tmem + lane_base + buf * 128 + 64 + h * 32, part);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_addr(&pempty[buf]));  // the buffer may take the next block's MMAs
#pragma unroll
      for (int c = 0; c < 32; ++c) two_sum_add(sim[c], cim[c], part[c]);
    }
  }
  // every role has finished (the MMA issuer after draining its MMAs, the producer after its copies)
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool ok = *(volatile int*)s_fail == 0;
  if (warp >= 2 && ok) {
    const int i = mt * TM + q * 32 + lane;
    if (i < p.M) {
      const bool use_beta = (p.beta.x != 0.f || p.beta.y != 0.f);
      cplx<float>* C = p.C + view_batch(p.vc, z);
      const int64_t ro = view_row(p.vc, i);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int j = nt * TN + h * 32 + c;
        if (j >= p.N || (p.herm && j > i)) continue;
        const int64_t o = ro + view_col(p.vc, j);
        cplx<float> v = p.alpha * mk<float>(sre[c] + cre[c], sim[c] + cim[c]);
        if (use_beta) {
          cplx<float> old = GX(C, o);
          if (p.vc.conj) old.y = -old.y;
          v = v + p.beta * old;
        }
        if (p.vc.conj) v.y = -v.y;
        GX(C, o) = v;
      }
    }
  }
  if (tid == 0 && !ok && p.status) atomicOr(GP(p.status), kStatusTimeout);
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }
}  // namespace

int64_t tc_plane_floats_a(int M, int K) { return (int64_t)cdiv(M, TM) * cdiv(K, TK) * (A_STAGE / 4); }
int64_t tc_plane_floats_b(int N, int K) { return (int64_t)cdiv(N, TN) * cdiv(K, TK) * (B_STAGE / 4); }

bool tc_gemm_applicable(const GemmArgs<float>& g, int batch) {
  if (!g.tc_a || !g.tc_b || g.M < TM || g.N < TN || g.K < 2 * TK) return false;
  return tc_plane_floats_a(g.M, g.K) * batch <= g.tc_a_cap && tc_plane_floats_b(g.N, g.K) * batch <= g.tc_b_cap;
}

cudaError_t tc_gemm(cudaStream_t s, int batch, const GemmArgs<float>& g) {
  if (batch <= 0 || g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  static PerDevice setup;
  cudaError_t e = setup.once([](int) {
    return cudaFuncSetAttribute(tc_cgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  });
  if (e != cudaSuccess) return e;
  const int MT = cdiv(g.M, TM), NTt = cdiv(g.N, TN), KS = cdiv(g.K, TK);
  {  // operand planes (contiguous per batch item)
    const int64_t ta = (int64_t)MT * TM * KS * TK, tb = (int64_t)NTt * TN * KS * TK;
    dim3 ga((unsigned)std::min<int64_t>((ta + 255) / 256, 4096), batch);
    tc_split_kernel<<<ga, 256, 0, s>>>(g.M, g.K, TM, MT, KS, g.A, g.va, 0, g.tc_a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 gb((unsigned)std::min<int64_t>((tb + 255) / 256, 4096), batch);
    tc_split_kernel<<<gb, 256, 0, s>>>(g.N, g.K, TN, NTt, KS, g.B, g.vb, 1, g.tc_b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  TcParams p;
  p.M = g.M;
  p.N = g.N;
  p.K = g.K;
  p.MT = MT;
  p.NT = NTt;
  p.KS = KS;
  p.Ap = g.tc_a;
  p.Bp = g.tc_b;
  p.alpha = g.alpha;
  p.beta = g.beta;
  p.C = g.C;
  p.vc = g.vc;
  p.herm = g.herm;
  p.status = g.status;
  dim3 grid(NTt, MT, batch);
  tc_cgemm_kernel<<<grid, NTH, SMEM_BYTES, s>>>(p);
  return cudaGetLastError();
}

}  // namespace mpdo

namespace mpdo {
namespace {
// One thread waits on an mbarrier that nothing arrives on: the bounded wait must give up after
// limit_ns and record the timeout in the status word.
__global__ void wait_timeout_probe(uint64_t limit_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t a = smem_addr(&bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait_bounded(a, 0, limit_ns)) atomicOr(GP(status), kStatusTimeout);
}
}  // namespace
}  // namespace mpdo

extern "C" mpdo_status mpdo_wait_selftest(int limit_us, int* status_out) {
  using namespace mpdo;
  if (limit_us < 1 || limit_us > 1000000 || !status_out) return MPDO_EINVAL;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return MPDO_ENOMEM;
  mpdo_status ret = MPDO_OK;
  int h = 0;
  if (cudaMemset(d, 0, sizeof(int)) != cudaSuccess) ret = MPDO_ECUDA;
  if (!ret) {
    wait_timeout_probe<<<1, 1>>>((uint64_t)limit_us * 1000ull, d);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      ret = MPDO_ECUDA;
  }
  cudaFree(d);
  if (ret) return ret;
  *status_out = h;
  return (h & kStatusTimeout) ? MPDO_ETIMEOUT : MPDO_OK;
}

// ---------------------------------------------------------------------------------------------
// Self-test: random complex64 operands, the tensor-core product against the CUDA-core GEMM.
extern "C" mpdo_status mpdo_tc_selftest(int M, int N, int K, double* max_rel_err, int* err_flag) {
  using namespace mpdo;
  if (M < 1 || N < 1 || K < 1 || !max_rel_err || !err_flag) return MPDO_EINVAL;
  std::vector<cplx<float>> ha((size_t)M * K), hb((size_t)K * N);
  uint64_t st = 12345;
  auto rnd = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (float)((int64_t)(st >> 40) - (1ll << 23)) / (float)(1 << 23);
  };
  for (auto& v : ha) v = mk<float>(rnd(), rnd());
  for (auto& v : hb) v = mk<float>(rnd(), rnd());
  cplx<float>*da = nullptr, *db = nullptr, *dc = nullptr, *dr = nullptr;
  float *pa = nullptr, *pb = nullptr;
  int* dstat = nullptr;
  const int64_t na = tc_plane_floats_a(M, K), nb = tc_plane_floats_b(N, K);
  mpdo_status ret = MPDO_OK;
  if (cudaMalloc(&da, sizeof(cplx<float>) * ha.size()) != cudaSuccess ||
      cudaMalloc(&db, sizeof(cplx<float>) * hb.size()) != cudaSuccess ||
      cudaMalloc(&dc, sizeof(cplx<float>) * (size_t)M * N) != cudaSuccess ||
      cudaMalloc(&dr, sizeof(cplx<float>) * (size_t)M * N) != cudaSuccess ||
      cudaMalloc(&pa, sizeof(float) * na) != cudaSuccess || cudaMalloc(&pb, sizeof(float) * nb) != cudaSuccess ||
      cudaMalloc(&dstat, sizeof(int)) != cudaSuccess) {
    ret = MPDO_ENOMEM;
  } else {
    cudaMemcpy(da, ha.data(), sizeof(cplx<float>) * ha.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(db, hb.data(), sizeof(cplx<float>) * hb.size(), cudaMemcpyHostToDevice);
    cudaMemset(dstat, 0, sizeof(int));
    GemmArgs<float> g;
    g.M = M;
    g.N = N;
    g.K = K;
    g.alpha = mk<float>(1, 0);
    g.beta = mk<float>(0, 0);
    g.A = da;
    g.va = row_major(K, 0);
    g.B = db;
    g.vb = row_major(N, 0);
    g.C = dc;
    g.vc = row_major(N, 0);
    g.herm = 0;
    g.tc_a = pa;
    g.tc_b = pb;
    g.tc_a_cap = na;
    g.tc_b_cap = nb;
    g.status = dstat;
    if (!tc_gemm_applicable(g, 1)) ret = MPDO_EINVAL;
    if (!ret && tc_gemm(nullptr, 1, g) != cudaSuccess) ret = MPDO_ECUDA;
    g.C = dr;
    g.tc_a = g.tc_b = nullptr;
    if (!ret && gemm<float>(nullptr, 1, g) != cudaSuccess) ret = MPDO_ECUDA;
    if (!ret && cudaDeviceSynchronize() != cudaSuccess) ret = MPDO_ECUDA;
    if (!ret) {
      std::vector<cplx<float>> hc((size_t)M * N), hr((size_t)M * N);
      cudaMemcpy(hc.data(), dc, sizeof(cplx<float>) * hc.size(), cudaMemcpyDeviceToHost);
      cudaMemcpy(hr.data(), dr, sizeof(cplx<float>) * hr.size(), cudaMemcpyDeviceToHost);
      int hs = 0;
      cudaMemcpy(&hs, dstat, sizeof(int), cudaMemcpyDeviceToHost);
      double num = 0, den = 0;
      for (size_t e = 0; e < hc.size(); ++e) {
        double dx = (double)hc[e].x - hr[e].x, dy = (double)hc[e].y - hr[e].y;
        num = std::max(num, std::sqrt(dx * dx + dy * dy));
        den = std::max(den, std::sqrt((double)hr[e].x * hr[e].x + (double)hr[e].y * hr[e].y));
      }
      *max_rel_err = den > 0 ? num / den : num;
      *err_flag = hs;
    }
  }
  cudaFree(da);
  cudaFree(db);
  cudaFree(dc);
  cudaFree(dr);
  cudaFree(pa);
  cudaFree(pb);
  cudaFree(dstat);
  return ret;
}
