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
constexpr int kExpectChunk = 16;         // terms per expectation launch
constexpr int kMaxDynSmem = 200 * 1024;      // dynamic shared memory cap of the sweep kernel
constexpr int kTableSmemLimit = 112 * 1024;  // stage a sweep's tables in shared memory up to this total

struct PhaseTables {
  const PhaseDesc* ph;
  const PhaseOp* po;
  const void* pc;
};

// Complex sweeps with register phases run the phase kernel; everything else
// (real DM sweeps, tiny tiles) the row kernel.
cudaError_t launch_sweep(bool cplx, bool f64, void* state, int B, const SweepDesc& sd, const DevOp* ops,
                         const void* ents, const PhaseTables* pt, int sm_count, cudaStream_t s);
cudaError_t launch_init(bool cplx, bool f64, void* state, int n, int sm_count, cudaStream_t s);
cudaError_t launch_real_to_cplx(bool f64, const void* in, void* out, uint64_t count, int sm_count, cudaStream_t s);
cudaError_t launch_cplx_to_real(bool f64, const void* in, void* out, uint64_t count, int sm_count, cudaStream_t s);
cudaError_t launch_sv_abs2(bool f64, const void* psi, double* p, uint64_t count, int sm_count, cudaStream_t s);
cudaError_t launch_dm_diag(bool f64, const void* r, double* g, int n, double e, int sm_count, cudaStream_t s);
cudaError_t launch_sv_expect_group(bool f64, const void* psi, int n, uint64_t x, const uint64_t* zm, const int* ym,
                                   int nt, double* part, int nblocks, double* out, cudaStream_t s);
cudaError_t launch_dm_expect(bool f64, const void* r, int n, const uint64_t* xm, const uint64_t* zm,
                             const double* coef, int nt, double* out, int sum, int normalize, cudaStream_t s);
cudaError_t launch_weighted_sum(const double* v, const double* coef, int nt, double* out, cudaStream_t s);
cudaError_t launch_scale(double* v, int nt, const double* denom, cudaStream_t s);

}  // namespace nwq
