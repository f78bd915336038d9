// Launch wrappers of the device kernels (host-callable, no torch types).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "nwq_internal.h"

#include <atomic>

namespace nwq {

// Kernels launched by this library (all launch wrappers add to it).
extern std::atomic<unsigned long long> g_launches;

constexpr int kSweepThreads = 256;
constexpr int kExpectChunk = 16;         // terms per launch of the general (per-x) expectation kernel
constexpr int kMaxDynSmem = 200 * 1024;      // dynamic shared memory cap of the sweep kernel
constexpr int kTableSmemLimit = 112 * 1024;  // stage a sweep's tables in shared memory up to this total

// Tiled SV expectations: 128 threads, tiles of at most 2^12 amplitudes, at
// most 256 terms per pass.  A pass's tile holds the low m bits (contiguous) and
// h = T - m high bits (hmask); fmask holds the remaining bits of the index.
constexpr int kExpThreads = 128;
constexpr int kExpTileBits = 12;
constexpr int kExpPassTerms = 256;
struct ExpTerm {
  uint64_t zh;      // z bits outside the tile (global positions)
  uint32_t xl, zl;  // x and z bits inside the tile (tile-local positions)
  int32_t y;        // |x & z| mod 4
  int32_t out;      // output column
};
struct ExpPass {
  uint64_t hmask, fmask;
  int32_t T, m, h, k0, nk;
  int32_t zt;    // 1 when a term of the pass has no X support (Z-type: read from the probabilities)
  int32_t dwin;  // 1: the state holds the double-word layout (complex128, full tiles only)
};
static_assert(sizeof(ExpTerm) == 24, "ExpTerm layout");

struct PhaseTables {
  const PhaseDesc* ph;
  const PhaseOp* po;
  const void* pc;
};

// Interpreted sweeps (the run-time specialised kernels of jit.cpp take the
// sweeps of large states): complex sweeps with register phases run the phase
// kernel; everything else (real DM sweeps, tiny tiles) the row kernel.
cudaError_t launch_sweep(bool cplx, bool f64, void* state, int B, const SweepDesc& sd, const DevOp* ops,
                         const void* ents, const PhaseTables* pt, int sm_count, cudaStream_t s);
cudaError_t launch_init(bool cplx, bool f64, void* state, int n, int sm_count, cudaStream_t s, bool dw = false);
// NWQ_EXPECT_FP64=1 in the environment: complex128 expectation passes on the FP64 pipe
bool expect_fp64_only();
// FP64 array of ndouble values (even) to the double-word layout (to_dw) or back, in place.
cudaError_t launch_dw_convert(void* data, uint64_t ndouble, bool to_dw, int sm_count, cudaStream_t s);
cudaError_t launch_dw_renormalize(void* data, uint64_t ndouble, int sm_count, cudaStream_t s);
cudaError_t launch_real_to_cplx(bool f64, const void* in, void* out, uint64_t count, int sm_count, cudaStream_t s);
cudaError_t launch_cplx_to_real(bool f64, const void* in, void* out, uint64_t count, int sm_count, cudaStream_t s);
cudaError_t launch_sv_abs2(bool f64, const void* psi, double* p, uint64_t count, int sm_count, cudaStream_t s);
cudaError_t launch_dm_diag(bool f64, const void* r, double* g, int n, double e, int sm_count, cudaStream_t s,
                           bool dw = false);
cudaError_t launch_sv_expect_group(bool f64, const void* psi, int n, uint64_t x, const uint64_t* zm, const int* ym,
                                   int nt, double* part, int nblocks, const int* idx, double* out, cudaStream_t s);
size_t sv_expect_tiled_smem(bool f64, const ExpPass& P);
cudaError_t launch_sv_expect_tiled(bool f64, const void* psi, int n, const ExpPass& P, const ExpTerm* terms,
                                   double* part, int ncols, int grid, cudaStream_t s);
cudaError_t launch_reduce_partials(const double* part, int nblocks, int nt, const int* idx, double* out,
                                   cudaStream_t s);
cudaError_t launch_dm_expect(bool f64, const void* r, int n, const uint64_t* xm, const uint64_t* zm,
                             const double* coef, int nt, double* out, int sum, int normalize, cudaStream_t s,
                             bool dw = false);
cudaError_t launch_weighted_sum(const double* v, const double* coef, int nt, double* out, cudaStream_t s);
cudaError_t launch_scale(double* v, int nt, const double* denom, cudaStream_t s);

}  // namespace nwq
