// Address checks of the debug build (libmpdo_bounds.so, compiled with -DMPDO_BOUNDS).
//
// In that build every global-memory access the MPDO kernels make goes through GX / GP / GRANGE / GPTR, which
// look the accessed bytes up in a table of the live device ranges: every allocation the library makes
// (cudaMalloc / cudaFree below are routed through a registry) plus the ranges a caller registers for
// its own buffers (mpdo_bounds_register).  An access outside every range is not made: the check
// counts it, records the first one (source file, line, address, size) and hands back a pointer into a
// scratch buffer, so the kernel runs on without a fault or a trap and the host reads the record with
// mpdo_bounds_read.  In the release library the macros are the plain access or pointer and nothing else.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#ifdef MPDO_BOUNDS

namespace mpdo {

// layout of the state block every translation unit points at (device memory, 64-bit words)
constexpr int kBoundsTable = 0;     // address of the current table: [n, 0, lo_0, hi_0, lo_1, hi_1, ...]
constexpr int kBoundsFails = 1;     // failed checks since the last read
constexpr int kBoundsSite = 2;      // first failure: file-name hash << 32 | line
constexpr int kBoundsAddr = 3;      // first failure: address
constexpr int kBoundsBytes = 4;     // first failure: size of the access
constexpr int kBoundsSinkWord = 8;  // the scratch buffer starts here
constexpr long long kBoundsCap = 16384;                // ranges per table
constexpr unsigned long long kBoundsSinkBytes = 1u << 18;  // largest redirected access

// FNV-1a of the file name after its last '/': identifies the source file of a check site
__host__ __device__ constexpr uint32_t bounds_name_hash(const char* s) {
  const char* b = s;
  for (const char* c = s; *c; ++c)
    if (*c == '/') b = c + 1;
  uint32_t h = 2166136261u;
  for (const char* c = b; *c; ++c) h = (h ^ (uint32_t)(unsigned char)*c) * 16777619u;
  return h;
}

template <uint32_t H>
struct BoundsFile {
  static constexpr uint32_t value = H;  // forces the hash to a compile-time constant
};

namespace bounds_unit {
// per translation unit: the state block (set once, when the registry starts)
static __device__ unsigned long long* g_cell = nullptr;

static cudaError_t set_cell(unsigned long long* cell, cudaStream_t s) {
  cudaError_t e = cudaMemcpyToSymbolAsync(g_cell, &cell, sizeof cell, 0, cudaMemcpyHostToDevice, s);
  return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
}

// the check: p (bytes long) must lie inside one range of the current table
static __device__ __noinline__ const void* check(const void* p, unsigned long long bytes, unsigned long long site) {
  unsigned long long* cell = g_cell;
  if (cell == nullptr) return p;  // registry not started (no allocation made yet)
  const unsigned long long* t =
      reinterpret_cast<const unsigned long long*>(*reinterpret_cast<volatile unsigned long long*>(cell + kBoundsTable));
  if (t == nullptr) return p;  // registry disabled (table overflow)
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  long long n = (long long)t[0];
  if (n > kBoundsCap) n = kBoundsCap;
  long long lo = 0, hi = n - 1, f = -1;  // last range whose start is <= a
  while (lo <= hi) {
    const long long m = (lo + hi) >> 1;
    if (t[2 + 2 * m] <= a) {
      f = m;
      lo = m + 1;
    } else {
      hi = m - 1;
    }
  }
  if (f >= 0 && a <= t[3 + 2 * f] && bytes <= t[3 + 2 * f] - a) return p;
  if (atomicAdd(cell + kBoundsFails, 1ull) == 0ull) {
    cell[kBoundsSite] = site;
    cell[kBoundsAddr] = a;
    cell[kBoundsBytes] = bytes;
  }
  return cell + kBoundsSinkWord;
}
}  // namespace bounds_unit

template <typename T>
__device__ __forceinline__ T* bounds_safe(T* p, unsigned long long site) {
  return (T*)bounds_unit::check((const void*)p, sizeof(T), site);
}
template <typename T>
__device__ __forceinline__ T* bounds_range(T* p, unsigned long long bytes, unsigned long long site) {
  return (T*)bounds_unit::check((const void*)p, bytes, site);
}

// a pointer whose subscripts are checked (kernels with many accesses through a few base pointers
// declare those with GPTR); the recorded line is the declaration's
template <typename T>
struct CheckedPtr {
  T* p;
  unsigned long long site;
  __device__ CheckedPtr(T* q, unsigned long long s) : p(q), site(s) {}
  __device__ T& operator[](int64_t i) const { return *bounds_safe(p + i, site); }
  __device__ CheckedPtr operator+(int64_t i) const { return CheckedPtr(p + i, site); }
  __device__ operator T*() const { return p; }
};

// host side of the registry (bounds.cu)
void bounds_add_unit(cudaError_t (*set)(unsigned long long*, cudaStream_t));
cudaError_t bounds_malloc(void** p, size_t bytes);
cudaError_t bounds_free(void* p);

namespace bounds_unit {
struct Registration {
  Registration() { bounds_add_unit(&set_cell); }
};
static Registration g_registration;  // per translation unit: hands set_cell to the registry
}  // namespace bounds_unit

}  // namespace mpdo

#define MPDO_BSITE                                                                            \
  (((unsigned long long)::mpdo::BoundsFile<::mpdo::bounds_name_hash(__FILE__)>::value << 32) | \
   (unsigned long long)__LINE__)
#define GX(p, i) (*::mpdo::bounds_safe((p) + (i), MPDO_BSITE))
#define GP(p) (::mpdo::bounds_safe((p), MPDO_BSITE))
#define GRANGE(p, bytes) (::mpdo::bounds_range((p), (unsigned long long)(bytes), MPDO_BSITE))
#define GPTR(T, name, init) ::mpdo::CheckedPtr<T> name((init), MPDO_BSITE)

#ifndef MPDO_BOUNDS_REGISTRY
#define cudaMalloc(p, bytes) ::mpdo::bounds_malloc((void**)(p), (bytes))
#define cudaFree(p) ::mpdo::bounds_free((void*)(p))
#endif

#else  // release build: the plain access

#define GX(p, i) ((p)[i])
#define GP(p) (p)
#define GRANGE(p, bytes) (p)
#define GPTR(T, name, init) T* name = (init)

#endif
