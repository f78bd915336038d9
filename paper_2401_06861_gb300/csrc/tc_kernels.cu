// Tensor-core pass of one dense five-qubit block over a complex64 state
// vector: tcgen05 MMAs of kind TF32 with the accumulator in tensor memory.
//
// A tile is 2^12 amplitudes: the block's 5 qubits and the 7 lowest other
// qubits (so qubits 0..6 are always in the tile and each warp access covers
// >= 256 contiguous bytes).  Its 128 columns (one per setting of the 7 row
// qubits) are the rows of the MMA operand A (128 x 64 reals, interleaved
// re/im of the 32 block amplitudes); B is the 64 x 64 real form of the block
// matrix.  D = A B^T (128 x 64 FP32) is the updated tile.  FP32 accuracy from
// TF32 inputs uses the three-term split x = hi + lo, D = lo*hi + hi*lo + hi*hi
// (the lo*lo term is below FP32 rounding).
//
// Operands sit in shared memory in the 128-byte-swizzled K-major layout
// (rows of 128 bytes, 16-byte chunk c of row r stored at chunk c ^ (r & 7),
// 8-row groups 1024 bytes apart), in two K halves of 32 reals.  Each CTA
// (128 threads, one thread issuing the MMAs; 3 CTAs per SM) walks its
// tiles with one A buffer: the TF32 lo parts go in and the lo * B_hi MMAs
// run, then the hi parts replace them for hi * B_lo + hi * B_hi while the
// next tile's loads go out (small products first in the FP32 accumulator).
// Every MMA group is committed to an mbarrier and waited on (bounded); the
// accumulator rows then move from tensor memory to shared memory and the
// tile is written back with the pattern it was read with.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "kernels.hpp"
#include "tc.hpp"

namespace nwq {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcCtasPerSm = 3;
constexpr uint32_t kSmA = 32768;  // the A operand: 128 rows x 64 FP32, two K halves of 16 KiB
constexpr uint32_t kSmB = 16384;  // one B operand: 64 rows x 64 FP32, two K halves of 8 KiB
constexpr uint32_t kOffA = 0, kOffBhi = kSmA, kOffBlo = kSmA + kSmB;
constexpr uint32_t kOffFw = kSmA + 2 * kSmB;  // kTcMaxFree x u64: tile-index bit weights
constexpr uint32_t kOffBar = kOffFw + 8 * kTcMaxFree;
constexpr uint32_t kOffTmem = kOffBar + 8;
constexpr uint32_t kSmUsed = kOffTmem + 8;
constexpr size_t kTcSmem = kSmUsed + 1024;  // + room to align the operands to 1024 bytes
constexpr uint32_t kTmemCols = 64;          // accumulator: 128 lanes x 64 FP32 columns
constexpr uint32_t kWaitPolls = 1u << 20;   // bound on polls of the MMA-completion barrier
static_assert(kOffBar % 8 == 0, "mbarrier alignment");

// Instruction descriptor: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2),
// both K-major, N = 64 (bits 17-22 = N/8), M = 128 (bits 24-28 = M/16).
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ int g_tc_timeouts;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, 128-byte swizzle, K-major: start address,
// leading offset 16 bytes (unused for this layout), 8-row groups 1024 bytes
// apart, descriptor version 1 (bit 46), swizzle mode 2 (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024u >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void st16(uint32_t a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
__device__ __forceinline__ float4 ld16(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a)
               : "memory");
  return v;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __noinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t polls) {
  for (uint32_t i = 0; i < polls; i++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive FP32 columns of this thread's accumulator lane (load and wait in one statement).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// The two amplitudes of a pair (block bit 0 = 0 and 1, same column): one
// 16-byte access when that bit is qubit 0, else two 8-byte accesses.
__device__ __forceinline__ float4 load_pair(const float2* psi, uint64_t amp, uint64_t gp, bool q0) {
  if (q0) return __ldcs((const float4*)(psi + amp));
  const float2 a = __ldcs(psi + amp), b = __ldcs(psi + amp + gp);
  return make_float4(a.x, a.y, b.x, b.y);
}
// Bring the lines of a pair into L2 (no register, no wait: the loads of that
// tile one iteration later then hit L2 instead of HBM).
__device__ __forceinline__ void prefetch_pair(const float2* psi, uint64_t amp, uint64_t gp, bool q0) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(psi + amp));
  if (!q0) asm volatile("prefetch.global.L2 [%0];" ::"l"(psi + amp + gp));
}
__device__ __forceinline__ void store_pair(float2* psi, uint64_t amp, uint64_t gp, bool q0, float4 v) {
  if (q0) {
    __stcs((float4*)(psi + amp), v);
  } else {
    __stcs(psi + amp, make_float2(v.x, v.y));
    __stcs(psi + amp + gp, make_float2(v.z, v.w));
  }
}

// Tile bits by role (host-chosen, TcGeom): bit 0 = block bit 0 (the pair,
// 8 operand bytes apart, so a pair is one 16-byte operand chunk), bits 1..5 =
// lane, 6..7 = warp, 8..11 = loop step i.  The lane bits are the five lowest
// other tile qubits (a warp covers >= 256 contiguous bytes), lane bits 0..2
// chosen so that each quarter-warp writes 8 distinct 16-byte bank groups.
__global__ void __launch_bounds__(kTcThreads, kTcCtasPerSm)
    tc_block_kernel(float2* __restrict__ psi, const float4* __restrict__ mats, const __grid_constant__ TcGeom g,
                    uint32_t wait_polls, int issue_mma) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sb = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (sb - raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  uint64_t* fw = (uint64_t*)(sm + kOffFw);
  const uint32_t bar = sb + kOffBar;
  const uint32_t sA = sb + kOffA;

  if (tid < kTcMaxFree) fw[tid] = g.fw[tid];
  // B operands: TF32 hi and lo parts of the block's real 64 x 64 matrix (row n, reals k)
  for (int idx = tid; idx < 1024; idx += kTcThreads) {
    const int n = idx >> 4, c = idx & 15;
    const uint32_t off = (uint32_t)(c >> 3) * 8192u + (uint32_t)n * 128u + ((uint32_t)((c & 7) ^ (n & 7)) << 4);
    st16(sb + kOffBhi + off, mats[idx]);
    st16(sb + kOffBlo + off, mats[1024 + idx]);
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sb + kOffTmem),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *(volatile uint32_t*)(sm + kOffTmem);
  const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 accumulator lanes

  // this thread's pairs: tile-index bits 1..7 from tid, 8..11 from the loop step i
  uint64_t goff = 0;
  uint32_t soff = 0;
  for (int b = 1; b < 8; b++)
    if ((tid >> (b - 1)) & 1) {
      goff += g.gw[b];
      soff ^= g.sw[b];
    }
  const uint64_t gp = g.gw[0];
  const bool q0 = gp == 1;
  const uint64_t l0 = g.gw[8], l1 = g.gw[9], l2 = g.gw[10], l3 = g.gw[11];
  const uint32_t s0 = g.sw[8], s1 = g.sw[9], s2 = g.sw[10], s3 = g.sw[11];
#define TC_GI(i) (((i)&1 ? l0 : 0) + ((i)&2 ? l1 : 0) + ((i)&4 ? l2 : 0) + ((i)&8 ? l3 : 0))
#define TC_SI(i) (((i)&1 ? s0 : 0) ^ ((i)&2 ? s1 : 0) ^ ((i)&4 ? s2 : 0) ^ ((i)&8 ? s3 : 0))
  auto tile_base = [&](uint32_t x) {
    uint64_t b = 0;
    while (x) {
      b += fw[__ffs(x) - 1];
      x &= x - 1;
    }
    return b;
  };
  uint32_t phase = 0;
  bool timed_out = false;
  // Issue one product group (lo or hi A parts already in shared memory) and commit it.
  auto mma_group = [&](bool lo_pass) {
    fence_async_smem();
    __syncthreads();
    if (tid == 0 && issue_mma) {  // issue_mma = 0 only in the wait test: nothing arrives on the barrier
      tc_fence_after();
#pragma unroll
      for (int p = 0; p < 2; p++) {
        if (lo_pass && p == 1) break;  // lo pass: lo * B_hi only
        const uint32_t b0 = sb + (!lo_pass && p == 0 ? kOffBlo : kOffBhi);
#pragma unroll
        for (int k = 0; k < 8; k++) {
          const uint32_t ka = (uint32_t)(k >> 2) * 16384u + (uint32_t)(k & 3) * 32u;
          const uint32_t kb = (uint32_t)(k >> 2) * 8192u + (uint32_t)(k & 3) * 32u;
          mma_tf32(tmem, sw128_desc(sA + ka), sw128_desc(b0 + kb), (!lo_pass || p || k) ? 1u : 0u);
        }
      }
      mma_commit(bar);
    }
  };
  auto mma_wait = [&]() -> bool {
    const bool ok = mbar_wait_bounded(bar, phase, wait_polls);
    if (__syncthreads_or(!ok)) return false;
    phase ^= 1u;
    tc_fence_after();
    return true;
  };

  float4 r[16];
  uint32_t tile = blockIdx.x;
  if (tile < g.ntiles) {
    const uint64_t a = tile_base(tile) + goff;
#pragma unroll
    for (int i = 0; i < 16; i++) r[i] = load_pair(psi, a + TC_GI(i), gp, q0);
  }
  for (; tile < g.ntiles; tile += gridDim.x) {
    // 1. A <- TF32 lo parts, MMAs lo * B_hi (the small products accumulate first)
#pragma unroll
    for (int i = 0; i < 16; i++) {
      const float4 v = r[i];
      const float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
      st16(sA + (soff ^ TC_SI(i)),
           make_float4(tf32_rna(v.x - h.x), tf32_rna(v.y - h.y), tf32_rna(v.z - h.z), tf32_rna(v.w - h.w)));
      r[i] = h;  // keep the hi parts
    }
    mma_group(true);
    if (!mma_wait()) {
      timed_out = true;
      break;
    }
    // 2. A <- TF32 hi parts (A is free: the lo MMAs completed); MMAs hi * B_lo + hi * B_hi
#pragma unroll
    for (int i = 0; i < 16; i++) st16(sA + (soff ^ TC_SI(i)), r[i]);
    mma_group(false);
    // 3. the next tile's loads are in flight while these MMAs and the write-back run
    const uint64_t cur = tile_base(tile) + goff;
    const uint32_t next = tile + gridDim.x;
    if (next < g.ntiles) {
      const uint64_t a = tile_base(next) + goff;
#pragma unroll
      for (int i = 0; i < 16; i++) r[i] = load_pair(psi, a + TC_GI(i), gp, q0);
      const uint32_t after = next + gridDim.x;  // the tile after that: into L2 now
      if (after < g.ntiles) {
        const uint64_t b = tile_base(after) + goff;
#pragma unroll
        for (int i = 0; i < 16; i++) prefetch_pair(psi, b + TC_GI(i), gp, q0);
      }
    }
    if (!mma_wait()) {
      timed_out = true;
      break;
    }
    if (g.direct) {
      // 4'. this thread's accumulator lane is its own column (row tid of A) and columns 4i..4i+3
      // are its pair i: stored straight back, 32 columns at a time; no shared-memory pass, and
      // A is not read here, so the next tile's split needs no extra barrier (the one before
      // its MMAs also orders these accumulator reads before them)
#pragma unroll
      for (int hh = 0; hh < 2; hh++) {
        float d[32];
        tmem_ld32(tmem_row + 32u * (uint32_t)hh, d);
#pragma unroll
        for (int c = 0; c < 8; c++)
          store_pair(psi, cur + TC_GI(8 * hh + c), gp, q0, make_float4(d[4 * c], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]));
      }
      tc_fence_before();
      continue;
    }
    // 4. accumulator lane tid (one state column) -> shared memory (the A layout), 32 columns at a time
#pragma unroll
    for (int hh = 0; hh < 2; hh++) {
      float d[32];
      tmem_ld32(tmem_row + 32u * (uint32_t)hh, d);
#pragma unroll
      for (int c = 0; c < 8; c++) {
        const uint32_t off = (uint32_t)hh * 16384u + (uint32_t)tid * 128u + ((uint32_t)(c ^ (tid & 7)) << 4);
        st16(sA + off, make_float4(d[4 * c], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]));
      }
    }
    tc_fence_before();
    __syncthreads();
    // 5. write the tile back with the load pattern
#pragma unroll
    for (int i = 0; i < 16; i++) store_pair(psi, cur + TC_GI(i), gp, q0, ld16(sA + (soff ^ TC_SI(i))));
    __syncthreads();
  }
#undef TC_GI
#undef TC_SI
  if (timed_out) {
    if (tid == 0) atomicAdd(&g_tc_timeouts, 1);
    mbar_wait_bounded(bar, phase, wait_polls);  // one more bounded wait for the MMAs in flight
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

cudaError_t launch_tc_block(void* psi, const TcGeom& g, const float* mats_dev, int sm_count, cudaStream_t s,
                            bool wait_test) {
  static std::atomic<int> attr_dev{-1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev.load() != dev) {
    cudaError_t e = cudaFuncSetAttribute(tc_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(tc_block_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  // Three CTAs per SM (65 KB of shared memory and 64 of the SM's 512
  // tensor-memory columns each, so allocation never waits).  The grid is not
  // taken from the occupancy query, which under-reports this kernel.
  uint64_t grid = (uint64_t)sm_count * kTcCtasPerSm;
  if (grid > g.ntiles) grid = g.ntiles;
  // the wait test withholds the MMAs and bounds each wait at 4096 polls
  tc_block_kernel<<<(unsigned)grid, kTcThreads, kTcSmem, s>>>((float2*)psi, (const float4*)mats_dev, g,
                                                                wait_test ? 4096u : kWaitPolls, wait_test ? 0 : 1);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t tc_timeouts(int* count) { return cudaMemcpyFromSymbol(count, g_tc_timeouts, sizeof(int)); }

}  // namespace nwq
