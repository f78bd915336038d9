// State-vector Pauli expectations, host side (see expect_host.cpp).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nwqgb.h"
#include "kernels.hpp"
#include "state.hpp"

namespace nwq {

struct SvChunk {  // general-kernel terms h.fb[off .. off + cnt) share x
  uint64_t x;
  int off, cnt;
};

// Caller-owned host arrays for nt terms: passes and eterms hold nt + 1
// entries, fb and chunks nt, work 2 nt + 2.
struct SvExpectHost {
  ExpPass* passes;
  ExpTerm* eterms;
  int* fb;
  SvChunk* chunks;
  int* work;
};
struct SvExpectCounts {
  int npass, nterms, nfb, nchunk;
};

void plan_sv_expect(int n, const nwq_pauli_term* terms, size_t nt, bool norm, SvExpectHost& h, SvExpectCounts& c);

// Host staging bytes and device scratch bytes for nt terms (upper bounds):
// [terms | z | y | idx | coef] staged, then [values | tiled partials |
// general partials] on the device only.
constexpr size_t sv_expect_up16(size_t v) { return (v + 15) & ~(size_t)15; }
constexpr size_t sv_expect_stage_bytes(size_t nt) {
  return sv_expect_up16((nt + 1) * sizeof(ExpTerm)) + 4 * sv_expect_up16(nt * 8);
}
constexpr size_t sv_expect_scratch_bytes(size_t nt, int grid, int fblocks) {
  return sv_expect_stage_bytes(nt) + sv_expect_up16((nt + 2) * 8) + sv_expect_up16((size_t)grid * (nt + 1) * 8) +
         sv_expect_up16((size_t)fblocks * kExpectChunk * 8);
}

// Launch shape of the state-vector passes: tiled-kernel grid and general-
// kernel blocks.  The allocating entry point uses one tiled block per tile up
// to 2 (FP64) / 4 (FP32) per SM and one general block per 256 amplitudes up to
// 4 per SM.  The allocation-free entry point (scratch_limit > 0) caps the
// general blocks at kNoallocMaxGeneralBlocks and shrinks the tiled grid until
// sv_expect_scratch_bytes fits scratch_limit; both change only how the FP64
// partial sums are partitioned, not which products are summed.
constexpr int kNoallocMaxGeneralBlocks = 256;
void sv_expect_shape(const nwq_state* st, size_t nt, size_t scratch_limit, int* grid, int* fblocks);

// A state left in the double-word layout by a plan run back to its FP64
// layout (stream-ordered, allocates nothing); no-op otherwise.
cudaError_t state_to_f64(nwq_state* st);

// Stage the tables (stage: sv_expect_stage_bytes(nt) host bytes), copy them
// to dev (sv_expect_scratch_bytes(nt, grid, fblocks) device bytes) and enqueue
// every launch on st's stream, ending with the copy of the result to out_host.
// A state in the double-word layout is read as it is when every pass is a
// full complex128 tile pass, and converted back to FP64 first otherwise.
// The caller synchronises the stream before reading out_host.
cudaError_t sv_expect_enqueue(nwq_state* st, const nwq_pauli_term* terms, size_t nt, uint32_t flags,
                              double* out_host, const SvExpectHost& h, const SvExpectCounts& c, int grid,
                              int fblocks, unsigned char* stage, unsigned char* dev);

}  // namespace nwq
