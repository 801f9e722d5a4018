// Tensor-core (tcgen05, BF16 x BF16 -> FP32) linear layer of the surrogate MLP: Z = act W^T.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace surr_tc {
// shapes and alignments the kernel takes: 32 <= O <= 256, I a multiple of 16, 16-byte aligned rows
bool applicable(int O, int I, const void* act, const void* W);
// act: Bn x I BF16 row-major, W: O x I BF16 row-major, Z: Bn x O FP32 row-major (device pointers)
cudaError_t linear(cudaStream_t s, int Bn, int O, int I, const __nv_bfloat16* act, const __nv_bfloat16* W, float* Z);
// 1 if a tensor-core launch gave up waiting for its MMAs (its output was not written)
cudaError_t read_fail_flag(int* fail);
}  // namespace surr_tc
