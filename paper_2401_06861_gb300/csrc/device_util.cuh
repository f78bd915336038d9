// Small device helpers shared by the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nwq {

template <class R>
struct Cplx;
template <>
struct Cplx<double> {
  using T = double2;
};
template <>
struct Cplx<float> {
  using T = float2;
};

// Scatter the low bits of v onto the set bits of mask (ascending).
__device__ __forceinline__ uint64_t deposit(uint64_t v, uint64_t mask) {
  uint64_t out = 0;
  while (v && mask) {
    uint64_t lowbit = mask & (~mask + 1ull);
    if (v & 1ull) out |= lowbit;
    v >>= 1;
    mask ^= lowbit;
  }
  return out;
}

// 16-byte asynchronous global -> shared copies (completion by group waits).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace nwq
