// Surrogate linear layers on the 5th-generation tensor cores: Z = act W^T with BF16 operands and
// FP32 accumulation in tensor memory (tcgen05.mma kind::f16).
//
// act is Bn x I (BF16, row-major), W is O x I (BF16, row-major), Z is Bn x O (FP32, row-major); both
// operands are K-major as stored, so they are copied to shared memory as they are, 16 bytes (8 BF16) per
// thread, into the no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix).  A CTA of 128
// threads owns 128 rows of Z and all O <= 256 columns: the FP32 accumulator occupies O TMEM columns.
// K is staged in chunks of up to 64 through two shared-memory stages; one thread issues the K/16
// MMAs of a chunk and commits them to the stage's mbarrier.  Every mbarrier wait is bounded: on
// timeout the kernel raises a device flag (read by surr_sync) and leaves its output unwritten.
#include <cuda_bf16.h>
#include <stdint.h>

#include "device_once.cuh"
#include "surrogate_tc.h"
#include "wait.cuh"

namespace surr_tc {

namespace {
constexpr int TM = 128, NTH = 128, STAGES = 2, KC = 64;

__device__ int g_fail = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// K-major no-swizzle descriptor: lbo = bytes between K-adjacent core matrices, sbo = bytes between
// 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;
}
// kind::f16 instruction descriptor: D F32, A and B BF16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t instr_desc(int n) {
  uint32_t d = 0;
  d |= 1u << 4;                    // D format F32
  d |= 1u << 7;                    // A format BF16
  d |= 1u << 10;                   // B format BF16
  d |= (uint32_t)(n >> 3) << 17;   // N / 8
  d |= (uint32_t)(TM >> 4) << 24;  // M / 16
  return d;
}
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  return mpdo::mbar_wait_bounded(mbar, parity);
}

// byte offset of the 16-byte chunk (row, c8) of a rows x kc K-major tile (c8 = k / 8)
__device__ __forceinline__ int chunk_off(int row, int c8, int kc) { return (row >> 3) * (kc / 8) * 128 + c8 * 128 + (row & 7) * 16; }

__global__ void __launch_bounds__(NTH) linear_kernel(int Bn, int O, int I, const __nv_bfloat16* act,
                                                     const __nv_bfloat16* W, float* Z, int ncols) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int a_bytes = TM * KC * 2, b_bytes = ncols * KC * 2;
  const int stage_bytes = a_bytes + b_bytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + STAGES * stage_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + STAGES * stage_bytes + 64);
  int* s_fail = reinterpret_cast<int*>(smem + STAGES * stage_bytes + 128);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TM;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])) : "memory");
    *s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int nk = (I + KC - 1) / KC;
  uint32_t phase[STAGES] = {0, 0};
  const uint32_t idesc = instr_desc(ncols);
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt % STAGES;
    unsigned char* st = smem + s * stage_bytes;
    const int k0 = kt * KC, kc = (I - k0 < KC) ? I - k0 : KC;  // a multiple of 16
    if (kt >= STAGES) {  // the MMAs that read this stage two chunks ago must be done
      if (!mbar_wait(smem_u32(&mbar[s]), phase[s])) *s_fail = 1;
      phase[s] ^= 1;
    }
    const int c8n = kc / 8;
    for (int e = tid; e < TM * c8n; e += NTH) {
      const int row = e / c8n, c8 = e % c8n;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (m0 + row < Bn) v = *reinterpret_cast<const uint4*>(act + (int64_t)(m0 + row) * I + k0 + c8 * 8);
      *reinterpret_cast<uint4*>(st + chunk_off(row, c8, kc)) = v;
    }
    for (int e = tid; e < ncols * c8n; e += NTH) {
      const int n = e / c8n, c8 = e % c8n;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (n < O) v = *reinterpret_cast<const uint4*>(W + (int64_t)n * I + k0 + c8 * 8);
      *reinterpret_cast<uint4*>(st + a_bytes + chunk_off(n, c8, kc)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy stores -> MMA reads
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(st);
      const uint32_t sbo = (uint32_t)(kc / 8) * 128;
      for (int kk = 0; kk < kc / 16; ++kk) {
        const uint64_t ad = smem_desc(base + kk * 256, 128, sbo);
        const uint64_t bd = smem_desc(base + a_bytes + kk * 256, 128, sbo);
        const int accumulate = (kt > 0 || kk > 0) ? 1 : 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[s]))
                   : "memory");
    }
    __syncthreads();
  }
  // every stage used has exactly one commit not yet waited for
  for (int s = 0; s < STAGES && s < nk; ++s) {
    if (!mbar_wait(smem_u32(&mbar[s]), phase[s])) *s_fail = 1;
    phase[s] ^= 1;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  const bool ok = (*s_fail == 0);
  if (!ok && tid == 0) atomicExch(&g_fail, 1);

  // epilogue: warp w reads TMEM lanes 32w..32w+31 (tile rows), 16 columns at a time
  const int row = m0 + warp * 32 + lane;
  for (int c0 = 0; c0 < ncols; c0 += 16) {
    uint32_t r[16];
    const uint32_t lane_addr = ((uint32_t)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(tmem + lane_addr + c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (!ok || row >= Bn) continue;
    float* zr = Z + (int64_t)row * O;
    for (int c = 0; c < 16; ++c) {
      const int j = c0 + c;
      if (j < O) zr[j] = __uint_as_float(r[c]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}
}  // namespace

bool applicable(int O, int I, const void* act, const void* W) {
  return O >= 32 && O <= 256 && I >= 16 && I % 16 == 0 && (reinterpret_cast<uintptr_t>(act) & 15) == 0 &&
         (reinterpret_cast<uintptr_t>(W) & 15) == 0;
}

cudaError_t linear(cudaStream_t s, int Bn, int O, int I, const __nv_bfloat16* act, const __nv_bfloat16* W, float* Z) {
  if (Bn <= 0) return cudaSuccess;
  if (!applicable(O, I, act, W)) return cudaErrorInvalidValue;
  int ncols = 32;  // TMEM columns: a power of two >= 32 that holds O
  while (ncols < O) ncols *= 2;
  const int bytes = STAGES * (TM * KC * 2 + ncols * KC * 2) + 256;
  static mpdo::PerDevice setup;
  cudaError_t e = setup.once([](int) {
    // at most 97 KB per CTA at O = 256: two CTAs per SM hold 2 x 256 of the 512 TMEM columns
    return cudaFuncSetAttribute(linear_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                STAGES * (TM * KC * 2 + 256 * KC * 2) + 256);
  });
  if (e != cudaSuccess) return e;
  linear_kernel<<<(Bn + TM - 1) / TM, NTH, bytes, s>>>(Bn, O, I, act, W, Z, ncols);
  return cudaGetLastError();
}

cudaError_t read_fail_flag(int* fail) { return cudaMemcpyFromSymbol(fail, g_fail, sizeof(int)); }

}  // namespace surr_tc
