// Host planner: lowers a gate list (plus noise model) to device sweeps.
#pragma once
#include <complex>
#include <cstddef>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nwqgb.h"
#include "nwq_internal.h"
#include "tc.hpp"

#include <cuda_runtime.h>

namespace nwq {

using cd = std::complex<double>;

// One operator on k bits of the state index, before it is placed in a sweep.
struct BitOp {
  int k = 0;
  int bits[4] = {0, 0, 0, 0};  // global bit of local operator bit j
  std::vector<cd> m;           // 2^k x 2^k, row-major (imaginary parts 0 for DM)
  int gate0 = 0, ngates = 1;   // provenance
};

struct PlanOptions {
  int tile_bits = 12;     // T
  int min_low = 3;        // coalescing: low contiguous bits always in the tile
  bool merge = true;      // algebraic merging of adjacent operators
  bool plain = false;     // one operator per sweep
  bool commute = false;   // complex plans: diagonal operators may pass one another when grouping
  int max_merge_bits = 4;
  int lookahead = 4096;   // operators scanned when filling a sweep
  int rescale_qubits = 0; // DM: deferred per-qubit scaling over this many qubits (0 = off)
  int register_bits = 0;  // complex sweeps: register-group bits per thread (0: 3 for FP64, 4 for FP32)
  int max_sweep_ops = 0;  // operators per sweep at most (0: no limit)
};

struct Plan {
  int kind = 0, n = 0, dtype = 0, B = 0;
  bool is_complex = true;
  size_t elem_bytes = 0, ent_bytes = 0;
  std::vector<SweepDesc> sweeps;
  std::vector<DevOp> ops;
  std::vector<unsigned char> ents;  // EntR<R> or EntC<R> records
  std::vector<int> op_gate0, op_ngates;
  // complex plans: register phases (see nwq_internal.h)
  std::vector<PhaseDesc> phases;
  std::vector<PhaseOp> pops;
  std::vector<unsigned char> pcoef;  // complex coefficients (float2 or double2)
  size_t pt_off[3] = {0, 0, 0};      // device offsets of phases, phase operators, coefficients
  double fma_per_elem = 0.0;  // summed over operators, per state element
  double bytes = 0.0;         // algorithmic bytes per run
  // device copy (lazy upload on first run)
  std::mutex mu;
  void* dev = nullptr;
  size_t dev_bytes = 0;
  // Plans internal to one state allocate their tables stream-ordered on the
  // state's stream and free them there (no device-wide synchronisation).
  bool stream_ordered = false;
  cudaStream_t dev_stream = nullptr;
  // run-time specialised kernels of this plan's sweeps (built on first launch)
  std::shared_ptr<void> jit;
  bool interpreted = false;  // never use them
  // FP64 plans: run the sweeps in double-word arithmetic (each FP64 value as
  // an unevaluated sum of two floats, FP32 pipe) when every sweep has such a
  // kernel; set before build_plan, which then keeps stored values within the
  // float exponent range (deferred scales and scalars)
  bool dw = false;
  bool last_run_dw = false;  // the latest run took the double-word path
  // the merged operators in execution order (nwq_plan_ops)
  std::vector<BitOp> exec_ops;
  // tensor-core plans (NWQ_PLAN_TC): dense five-qubit blocks, one pass each
  bool tc = false;
  std::vector<TcBlock> tcb;
  std::vector<TcGeom> tcg;
  std::vector<float> tctab;  // kTcMatFloats per block (TF32 hi, then lo)
  size_t tc_off = 0;         // device offset of tctab
  ~Plan();
};

// Gate matrix in the local basis j = b(q0) + 2 b(q1).  Returns the number of
// qubits (1 or 2), 0 for an unknown kind.
int gate_matrix(const nwq_gate& g, double theta0, cd* U);

// Lowering.  On error returns false and sets err.
bool lower_sv(const nwq_gate* g, size_t ng, int n, std::vector<BitOp>& out, std::string& err);
bool lower_dm(const nwq_gate* g, size_t ng, int n, const nwq_noise_model* nm, std::vector<BitOp>& out,
              std::string& err);

// Tensor-core plans (tc_plan.cpp): fuse one- and two-qubit operators into
// dense five-qubit blocks; fill the plan's block tables.
bool tc_fuse(const std::vector<BitOp>& ops, int n, std::vector<TcBlock>& out, std::string& err);
bool build_tc_plan(const std::vector<BitOp>& ops, Plan& plan, std::string& err);

// Merge + sweep grouping + device table layout.  The operators end up moved
// into plan.exec_ops (execution order); `ops` is left spent.
void build_plan(std::vector<BitOp>& ops, const PlanOptions& opt, Plan& plan);

// Verify the device tables of a built plan against the kernels' bounds
// (plan_check.cpp); false with a message on the first violation.
bool verify_plan(const Plan& p, std::string& err);

// Cost model: floating-point operations (multiply or add) per state element.
double op_cost(const BitOp& op, bool is_complex);

// Matrices used by the measurement helpers.
void pauli_to_rho_matrix(cd M[16]);   // per-qubit Pauli -> standard vec(rho) map
void rho_to_pauli_matrix(cd M[16]);   // its inverse

}  // namespace nwq
