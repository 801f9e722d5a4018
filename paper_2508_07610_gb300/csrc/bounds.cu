// Registry of the device ranges the address checks of the debug build accept, and its C-ABI calls
// (include/mpdo.h).  The release library keeps only the calls: mpdo_bounds_enabled returns 0,
// registering a range does nothing and mpdo_bounds_read reports MPDO_ESTATE.
//
// The registry keeps every live range (the library's own allocations and the caller's registered
// buffers) and, after each change, publishes a sorted table of their union to the device: the table
// goes into the next of kSlots preallocated slots and the slot's address into the state block that
// every translation unit's checks read.  A kernel that is still searching an older table keeps
// reading memory that stays allocated; only the pointer to the current table changes.  The copies
// run on a private non-blocking stream, so publishing is allowed while another stream is being
// captured into a CUDA graph.
#define MPDO_BOUNDS_REGISTRY
#include "bounds.cuh"
#include "mpdo.h"

#include <cstring>

#ifdef MPDO_BOUNDS

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

namespace mpdo {

namespace {
constexpr int kSlots = 64;
constexpr size_t kCellBytes = 64 + kBoundsSinkBytes;
constexpr size_t kSlotWords = 2 + 2 * (size_t)kBoundsCap;

struct Registry {
  std::mutex mu;
  std::vector<cudaError_t (*)(unsigned long long*, cudaStream_t)> units;
  std::vector<std::pair<unsigned long long, unsigned long long>> lib, user;  // [lo, hi)
  unsigned long long* cell = nullptr;   // device state block
  unsigned long long* slots = nullptr;  // device tables, kSlots x kSlotWords
  cudaStream_t stream = nullptr;
  int next = 0;
  bool started = false, overflow = false;
  cudaError_t error = cudaSuccess;
};

Registry& reg() {
  static Registry* r = new Registry;  // never destroyed: kernels may read its buffers until exit
  return *r;
}

// first use: allocate the state block and the table slots, point every translation unit at them
cudaError_t start(Registry& R) {
  if (R.started) return R.error;
  R.started = true;
  cudaError_t e = cudaStreamCreateWithFlags(&R.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&R.cell, kCellBytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&R.slots, sizeof(unsigned long long) * kSlotWords * kSlots);
  if (e == cudaSuccess) e = cudaMemsetAsync(R.cell, 0, kCellBytes, R.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(R.stream);
  for (size_t u = 0; e == cudaSuccess && u < R.units.size(); ++u) e = R.units[u](R.cell, R.stream);
  R.error = e;
  return e;
}

cudaError_t publish(Registry& R) {
  cudaError_t e = start(R);
  if (e != cudaSuccess) return e;
  std::vector<std::pair<unsigned long long, unsigned long long>> v(R.lib);
  v.insert(v.end(), R.user.begin(), R.user.end());
  std::sort(v.begin(), v.end());
  std::vector<unsigned long long> t(2, 0ull);
  for (const auto& r : v) {
    if (t.size() > 2 && r.first <= t.back()) {
      t.back() = std::max(t.back(), r.second);  // overlapping or touching: extend the last range
    } else {
      t.push_back(r.first);
      t.push_back(r.second);
    }
  }
  const unsigned long long n = (t.size() - 2) / 2;
  unsigned long long* table = nullptr;
  if ((long long)n > kBoundsCap) {
    R.overflow = true;  // checks switch off (table pointer 0); mpdo_bounds_read reports it
  } else {
    t[0] = n;
    table = R.slots + (size_t)R.next * kSlotWords;
    R.next = (R.next + 1) % kSlots;
    e = cudaMemcpyAsync(table, t.data(), sizeof(unsigned long long) * t.size(), cudaMemcpyHostToDevice, R.stream);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemcpyAsync(R.cell + kBoundsTable, &table, sizeof table, cudaMemcpyHostToDevice, R.stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(R.stream);
}
}  // namespace

void bounds_add_unit(cudaError_t (*set)(unsigned long long*, cudaStream_t)) {
  Registry& R = reg();
  std::lock_guard<std::mutex> lk(R.mu);
  R.units.push_back(set);
}

cudaError_t bounds_malloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return e;
  Registry& R = reg();
  std::lock_guard<std::mutex> lk(R.mu);
  const unsigned long long a = reinterpret_cast<unsigned long long>(*p);
  R.lib.emplace_back(a, a + bytes);
  e = publish(R);
  if (e != cudaSuccess) {
    R.lib.pop_back();
    cudaFree(*p);
    *p = nullptr;
  }
  return e;
}

cudaError_t bounds_free(void* p) {
  if (p == nullptr) return cudaFree(p);
  // cudaFree waits for the device anyway; waiting before the range leaves the table keeps a kernel
  // still running on it from being reported
  cudaDeviceSynchronize();
  Registry& R = reg();
  {
    std::lock_guard<std::mutex> lk(R.mu);
    const unsigned long long a = reinterpret_cast<unsigned long long>(p);
    for (size_t i = 0; i < R.lib.size(); ++i)
      if (R.lib[i].first == a) {
        R.lib.erase(R.lib.begin() + (std::ptrdiff_t)i);
        break;
      }
    publish(R);
  }
  return cudaFree(p);
}

// names of the files that hold checks, to turn a recorded hash back into a file name
static const char* const kCheckedFiles[] = {"engine.cu", "mpdo_kernels.cu", "gemm.cu", "qr.cu",  "eig.cu",
                                            "tc_gemm.cu", "noalloc.cu",     "batch.cu", "panel.cuh", "bounds.cuh"};

}  // namespace mpdo

using namespace mpdo;

extern "C" int mpdo_bounds_enabled(void) { return 1; }

extern "C" mpdo_status mpdo_bounds_register(const void* p, size_t bytes) {
  if (p == nullptr || bytes == 0) return MPDO_EINVAL;
  Registry& R = reg();
  std::lock_guard<std::mutex> lk(R.mu);
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  R.user.emplace_back(a, a + bytes);
  return publish(R) == cudaSuccess ? MPDO_OK : MPDO_ECUDA;
}

extern "C" mpdo_status mpdo_bounds_unregister(const void* p) {
  Registry& R = reg();
  std::lock_guard<std::mutex> lk(R.mu);
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  for (size_t i = 0; i < R.user.size(); ++i)
    if (R.user[i].first == a) {
      R.user.erase(R.user.begin() + (std::ptrdiff_t)i);
      return publish(R) == cudaSuccess ? MPDO_OK : MPDO_ECUDA;
    }
  return MPDO_EINVAL;
}

extern "C" mpdo_status mpdo_bounds_read(unsigned long long* failures, char* file, int file_cap, int* line,
                                        unsigned long long* addr, unsigned long long* bytes) {
  Registry& R = reg();
  std::lock_guard<std::mutex> lk(R.mu);
  if (cudaDeviceSynchronize() != cudaSuccess) return MPDO_ECUDA;
  unsigned long long w[5] = {0, 0, 0, 0, 0};
  if (R.started && R.error == cudaSuccess) {
    if (cudaMemcpy(w, R.cell, sizeof w, cudaMemcpyDeviceToHost) != cudaSuccess) return MPDO_ECUDA;
    const unsigned long long zero[4] = {0, 0, 0, 0};
    if (cudaMemcpy(R.cell + kBoundsFails, zero, sizeof zero, cudaMemcpyHostToDevice) != cudaSuccess) return MPDO_ECUDA;
  }
  if (failures) *failures = w[kBoundsFails];
  if (line) *line = (int)(w[kBoundsSite] & 0xffffffffull);
  if (addr) *addr = w[kBoundsAddr];
  if (bytes) *bytes = w[kBoundsBytes];
  if (file && file_cap > 0) {
    const char* name = w[kBoundsFails] ? "?" : "";
    for (const char* f : kCheckedFiles)
      if (w[kBoundsFails] && bounds_name_hash(f) == (uint32_t)(w[kBoundsSite] >> 32)) name = f;
    std::strncpy(file, name, (size_t)file_cap - 1);
    file[file_cap - 1] = '\0';
  }
  if (R.overflow) return MPDO_ENOMEM;
  return R.error == cudaSuccess ? MPDO_OK : MPDO_ECUDA;
}

#else  // release library

extern "C" int mpdo_bounds_enabled(void) { return 0; }
extern "C" mpdo_status mpdo_bounds_register(const void*, size_t) { return MPDO_OK; }
extern "C" mpdo_status mpdo_bounds_unregister(const void*) { return MPDO_OK; }
extern "C" mpdo_status mpdo_bounds_read(unsigned long long* failures, char* file, int file_cap, int* line,
                                        unsigned long long* addr, unsigned long long* bytes) {
  if (failures) *failures = 0;
  if (file && file_cap > 0) file[0] = '\0';
  if (line) *line = 0;
  if (addr) *addr = 0;
  if (bytes) *bytes = 0;
  return MPDO_ESTATE;
}

#endif
