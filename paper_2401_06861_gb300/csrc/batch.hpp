// Device tables of the batched parametrised-circuit kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nwq {

constexpr int kBatchThreads = 256;  // default threads per CTA
constexpr int kBatchMaxSmem = 220 * 1024;  // per-CTA dynamic shared memory cap of the batched kernel

// Gate types of the batched kernel.
enum : uint8_t { BT_FIXED1 = 0, BT_CX, BT_CZ, BT_SWAP, BT_RX, BT_RY, BT_RZ, BT_P, BT_U3, BT_RZZ, BT_FUSED };
// BT_FUSED: a run of one-qubit gates on qubit q0, applied as the one 2x2 matrix
// product computed per job in FP64; its `cls` members are the gates
// gates[pidx .. pidx + cls) in application order.

struct BGate {
  uint8_t type;   // BT_*
  uint8_t cls;    // BT_FIXED1: structure class of m (dense / real / diagonal)
  uint8_t q0, q1;
  int32_t pidx;   // parameter slot of theta[0], -1 = fixed
  double th[3];
  double m[8];    // BT_FIXED1: 2x2 complex, re/im interleaved
};

struct BTemplate {
  int32_t n, g0, ng, t0, nt, c0, ne, pad;
};

struct BTerm {
  uint32_t x, z;
  int32_t y;  // |x & z| mod 4
  int32_t pad;
};

struct BatchArgs {
  const BGate* gates;
  const BTemplate* templates;
  const BTerm* terms;
  const double* coeffs;
  const double* params;
  const int32_t* job_template;  // NULL = every job uses template 0
  double* out;
  double* norms;                // optional per-job <psi|psi>
  int* counter;                 // work-queue head (reset before each launch)
  int njobs, nparams, out_stride, ntemplates;
  int max_n, max_gates, max_terms;
  int threads;  // threads per CTA: 128, 256 or 512
  int dw;       // FP64 batches: 1 = double-word arithmetic on the FP32 pipe, 0 = the FP64 pipe
};
constexpr int kBatchThreadChoices[3] = {128, 256, 512};

// Noise after one gate of a quantum-trajectory circuit: the depolarising
// parameter (one draw when > 0) and, when `relax` is set, amplitude damping
// then phase damping on each gate qubit (two draws each).
struct TNoise {
  double pdep;
  double gamma[2], lambda[2];
  int32_t k, relax;
};

struct TrajArgs {
  const BGate* gates;
  const TNoise* noise;
  const BTerm* terms;
  const double* coeffs;
  const double* u;  // draws, `draws` per trajectory
  double* out;      // ntraj x ne energies
  int* counter;
  int n, ng, nt, ne, draws, ntraj, threads;
  int dw;  // FP64: 1 = double-word arithmetic on the FP32 pipe, 0 = the FP64 pipe
};

size_t batch_smem_bytes(bool f64, int max_n, int max_gates, int max_terms);
size_t traj_smem_bytes(bool f64, int n, int ng, int nt);
cudaError_t launch_traj(bool f64, const TrajArgs& a, int sm_count, cudaStream_t s);
cudaError_t launch_batch(bool f64, const BatchArgs& a, int sm_count, cudaStream_t s);

}  // namespace nwq
