/*
 * nwqgb.h -- C ABI of the GB300 state-vector / density-matrix simulator.
 *
 * The library simulates quantum circuits the way the NWQ-Sim paper frames
 * the problem (Sec. II: a circuit run on a state-vector back end, SV-Sim, or
 * on a noise-aware density-matrix back end, DM-Sim; Sec. III: a device noise
 * model made of depolarising, thermal-relaxation and measurement noise).
 *
 * Conventions used by every call:
 *   - qubit q is bit q of a basis index (little-endian);
 *   - a two-qubit gate acts in the local basis j = b(q[0]) + 2 b(q[1]); for
 *     CX, q[0] is the control and q[1] the target;
 *   - Pauli string (x_mask, z_mask) means i^{|x & z|} X^x Z^z (Hermitian);
 *   - all device work is issued on the state's CUDA stream; calls that return
 *     host results synchronise that stream;
 *   - every call returns NWQ_OK or a negative status and never throws;
 *     nwq_last_error() gives a message for the calling thread.
 * One state must be used by one host thread at a time; different states may
 * be used concurrently on different streams.
 */
#ifndef NWQGB_H
#define NWQGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nwq_state nwq_state; /* opaque: one SV or DM state on one device */
typedef struct nwq_plan nwq_plan;   /* opaque: a circuit lowered to device sweeps */

enum nwq_status {
  NWQ_OK = 0,
  NWQ_EINVAL = -1,       /* bad argument (qubit out of range, size mismatch, NULL) */
  NWQ_ENOMEM = -2,       /* device or host allocation failed */
  NWQ_ECUDA = -3,        /* a CUDA call failed (message has the CUDA error string) */
  NWQ_EBUDGET = -4,      /* a memory budget would be exceeded */
  NWQ_ETIMEOUT = -5,     /* a bounded device wait ran out */
  NWQ_EUNSUPPORTED = -6  /* valid request this build does not support */
};

/* Precision of the stored state.  SV: complex64 / complex128 amplitudes.
 * DM: float / double Pauli-basis coefficients (see nwq_dm_create). */
enum nwq_dtype { NWQ_F32 = 1, NWQ_F64 = 2, NWQ_C64 = 1, NWQ_C128 = 2 };

enum nwq_kind { NWQ_SV = 1, NWQ_DM = 2 };

/* Gate kinds.  Matrices (radians):
 *   RX/RY/RZ(t) = exp(-i t P / 2);  P(l) = diag(1, e^{il});  S = P(pi/2);
 *   T = P(pi/4);  SX = sqrt(X) = ((1+i) I + (1-i) X) / 2;
 *   U3(t, p, l) = [[cos t/2, -e^{il} sin t/2], [e^{ip} sin t/2, e^{i(p+l)} cos t/2]];
 *   RZZ(t) = exp(-i t Z(x)Z / 2);  CX flips q[1] when q[0] = 1;
 *   MAT1 / MAT2: caller matrix (2x2 / 4x4, row-major, re/im interleaved). */
enum nwq_gate_kind {
  NWQ_GATE_ID = 1, NWQ_GATE_X, NWQ_GATE_Y, NWQ_GATE_Z, NWQ_GATE_H, NWQ_GATE_S, NWQ_GATE_SDG,
  NWQ_GATE_T, NWQ_GATE_TDG, NWQ_GATE_SX, NWQ_GATE_RX, NWQ_GATE_RY, NWQ_GATE_RZ, NWQ_GATE_P,
  NWQ_GATE_U3, NWQ_GATE_MAT1,
  NWQ_GATE_CX = 64, NWQ_GATE_CZ, NWQ_GATE_SWAP, NWQ_GATE_RZZ, NWQ_GATE_MAT2
};

typedef struct {
  uint16_t kind;      /* nwq_gate_kind */
  uint16_t reserved;  /* must be 0 */
  int32_t q[2];       /* qubits; q[1] ignored for one-qubit gates */
  double theta[3];    /* angles; U3 uses all three, rotations theta[0] */
  int32_t param_idx;  /* batched calls: theta[0] := params[set * nparams + param_idx]; -1 = fixed */
  int32_t reserved2;
  const double* mat;  /* MAT1/MAT2 only; host memory, read during the call */
} nwq_gate;

typedef struct {
  uint64_t x_mask;
  uint64_t z_mask;
  double coeff;
} nwq_pauli_term;

/* Device noise model (paper Sec. III).  After every gate the library applies
 * depolarising noise on the gate's qubits (p1 for one-qubit gates, p2 for
 * two-qubit gates) in the form E(rho) = (1-p) rho + p Tr_S(rho) (x) I/2^|S|,
 * then thermal relaxation on each of the gate's qubits for the gate duration
 * (t1q_ns / t2q_ns) with gamma = 1 - exp(-t/T1) and coherence factor
 * eta = exp(-t/T2).  readout_e records the device's symmetric readout error
 * for callers; nwq_probs takes the readout error as an argument. */
enum nwq_noise_flags {
  NWQ_NOISE_RZ_VIRTUAL = 1u,      /* RZ is error-free and instantaneous */
  NWQ_NOISE_DEPOL_PAULI_FORM = 2u /* p is the total Pauli-error probability (p/3 each) */
};
typedef struct {
  int32_t n;            /* entries in T1_us / T2_us (>= number of qubits) */
  uint32_t flags;       /* nwq_noise_flags */
  const double* T1_us;  /* per-qubit T1, microseconds (host) */
  const double* T2_us;  /* per-qubit T2, microseconds (host) */
  double t1q_ns;        /* one-qubit gate duration */
  double t2q_ns;        /* two-qubit gate duration */
  double p1;            /* one-qubit depolarising parameter */
  double p2;            /* two-qubit depolarising parameter */
  double readout_e;     /* symmetric readout error */
} nwq_noise_model;

/* Plan / apply flags. */
enum nwq_plan_flags {
  NWQ_PLAN_FUSED = 0u,      /* default: gates fused into shared-memory sweeps */
  NWQ_PLAN_PLAIN = 1u,      /* one gate (plus its noise) per pass over the state */
  NWQ_PLAN_NO_MERGE = 2u,   /* fused sweeps, but no algebraic merging of operators */
  NWQ_PLAN_NO_RESCALE = 4u, /* DM: no deferred per-qubit scale factors (see nwq_plan_create) */
  NWQ_PLAN_INTERPRETED = 8u, /* never the run-time specialised sweep kernels (see nwq_plan_jit_check) */
  NWQ_PLAN_TC = 16u,         /* dense five-qubit blocks on the tensor cores (see below) */
  NWQ_PLAN_COMMUTE = 32u,    /* state vectors: when grouping sweeps, a diagonal operator may move ahead of
                                skipped diagonal operators (they commute): fewer passes for circuits
                                of diagonal gates (the default; kept for callers that name it) */
  NWQ_PLAN_DW = 64u,         /* FP64 plans: double-word sweeps (the default; see below) */
  NWQ_PLAN_FP64 = 128u,      /* FP64 plans: FP64-pipe sweeps only, never double words */
  NWQ_PLAN_NO_COMMUTE = 256u /* state vectors: group sweeps in operator order only */
};

/* Double-word sweeps (the default for FP64 plans; NWQ_PLAN_FP64 or NWQ_DW=0 in
 * the environment selects the FP64-pipe kernels, NWQ_DW=1 forces double words
 * even over NWQ_PLAN_FP64).  GB300 issues FP32 FMAs at 64 times
 * its FP64 rate, so an FP64 plan may run its sweeps with every FP64 value
 * held as an unevaluated sum hi + lo of two floats (|lo| <= ulp(hi) / 2,
 * about 48 significant bits) and every FP64 FMA done as a double-word
 * multiply-add on the FP32 pipe (error-free product and sum transformations,
 * relative error a few 2^-48 of the operands; Dekker, and Joldes, Muller and
 * Popescu, "Tight and rigorous error bounds for basic building blocks of
 * double-word arithmetic", 2017).  A plan run converts the state to the
 * double-word layout (same bytes) before its first sweep.  A caller-owned
 * buffer (dev_buf) is converted back after the last sweep, so it holds
 * complex128 / FP64 values whenever a call returns.  A library-owned state
 * keeps the double-word layout until a call needs FP64 values: a reset writes
 * |0..0> (|0..0><0..0|) in that layout, complex128 expectation passes over
 * full tiles and density-matrix expectations and probabilities read it as it
 * is, and every other call (copies, state-vector probabilities, strings wider
 * than a tile, FP64-pipe, FP32 and interpreted plans) converts it back first;
 * loads replace it.  Results are the
 * same either way up to the double words' rounding.  It applies when every sweep of
 * the plan runs a specialised kernel (states of >= NWQ_JIT_MIN_BITS index
 * bits, the kernels compiled); otherwise the plan runs its FP64 kernels.
 * Such plans keep deferred scale factors within the float exponent range. */

/* Tensor-core plans (NWQ_PLAN_TC; complex64 state vectors of >= 12 qubits,
 * else NWQ_EUNSUPPORTED).  The gate stream is fused into dense blocks of 5
 * qubits (paper Sec. III, "we optimize the quantum circuit", read as gate
 * fusion): a gate on a subset of the qubits of the latest gate on each of them
 * is first multiplied into it (CX RZ CX becomes one diagonal gate) unless a
 * diagonal gate would stop being diagonal; then blocks are built one at a
 * time from the gates not yet placed, in order, taking each gate that fits in
 * 5 qubits and may move ahead of the gates skipped so far (it shares no qubit
 * with them, or it and they are diagonal, so they commute); each block's
 * 32 x 32 matrix is multiplied out in FP64 (blocks under 5 qubits are padded
 * with idle qubits).  One pass over
 * the state per block applies it as a dense contraction on the tensor cores
 * (tcgen05, TF32 inputs split as hi + lo with the three products
 * hi*hi + hi*lo + lo*hi, FP32 accumulation).  nwq_plan_info: sweeps = ops =
 * blocks; fma_per_elem = 384 TF32 multiply-adds per amplitude per block. */

/* Expectation flags.  NWQ_EXPECT_NORMALIZE divides every value by the FP64
 * norm <psi|psi> (SV) or trace (DM) measured in the same call: the physical
 * expectation of an unnormalised state.  The raw norm is the value of the
 * identity string (x_mask = z_mask = 0) without this flag. */
enum nwq_expect_flags { NWQ_EXPECT_TERMS = 0u, NWQ_EXPECT_SUM = 1u, NWQ_EXPECT_NORMALIZE = 2u };

/* ---------------------------------------------------------------- states */

/* Bytes a state occupies on the device.  SV: 2^n amplitudes of 8 (F32) or
 * 16 (F64) bytes.  DM: 4^n real Pauli coefficients of 4 or 8 bytes. */
size_t nwq_state_bytes(int kind, int n, int dtype);

/* Create an n-qubit state vector |0..0> (paper Sec. II, SV-Sim).
 * dev_buf: NULL = the library allocates the state stream-ordered from the
 *   device's default memory pool (nwq_destroy frees it);
 *   otherwise a caller-owned device buffer of >= nwq_state_bytes() bytes,
 *   16-byte aligned, which the library never frees.
 * stream: a cudaStream_t (NULL = the legacy default stream).
 * n in [1, 34].  Errors: NWQ_EINVAL, NWQ_ENOMEM, NWQ_ECUDA. */
int nwq_sv_create(int n, int dtype, void* dev_buf, size_t buf_bytes, void* stream, nwq_state** out);

/* Create an n-qubit density matrix rho = |0..0><0..0| (paper Sec. II, DM-Sim).
 * The device copy holds the Pauli-basis coefficients r[x + 2^n z] = Tr(rho P(x,z)),
 * which are real for a Hermitian rho; nwq_state_copy returns the standard
 * column-stacked vec(rho).  n in [1, 16].  Arguments as nwq_sv_create. */
int nwq_dm_create(int n, int dtype, void* dev_buf, size_t buf_bytes, void* stream, nwq_state** out);

/* Reset to |0..0> (SV) or |0..0><0..0| (DM).  Asynchronous. */
int nwq_state_reset(nwq_state* st);

/* Load a state.  SV: 2^n complex amplitudes in the state's precision.
 * DM: the column-stacked vec(rho), 4^n complex entries in the state's
 * precision (element r + 2^n c = <r|rho|c>); rho must be Hermitian.
 * src_on_device selects the memory space of src.  Synchronises the stream. */
int nwq_state_load(nwq_state* st, const void* src, size_t bytes, int src_on_device);

/* Copy the state out.  SV: the amplitudes.  DM: vec(rho) as 4^n complex entries
 * in the state's precision.  dst_on_device selects the memory space of dst.
 * Synchronises the stream. */
int nwq_state_copy(nwq_state* st, void* dst, size_t bytes, int dst_on_device);

/* DM only: copy the raw Pauli-basis coefficients (4^n reals). */
int nwq_dm_copy_pauli(nwq_state* st, void* dst, size_t bytes, int dst_on_device);

/* DM only: load raw Pauli-basis coefficients (4^n reals in the state's
 * precision, as nwq_dm_copy_pauli writes them): with nwq_dm_copy_pauli /
 * nwq_state_copy and nwq_state_load for state vectors, a bit-exact checkpoint
 * of a run between two circuits (a long run resumes from host memory): the
 * resumed run ends bit-identical to the checkpointed state going on.  (A copy
 * of a state in the double-word layout first rounds it to its FP64 values in
 * place, see the double-word notes; a run that takes no copy keeps the double
 * words and agrees to the FP64 tolerance.)  Synchronises the stream. */
int nwq_dm_load_pauli(nwq_state* st, const void* src, size_t bytes, int src_on_device);

/* Free the handle.  Library-owned device memory is released stream-ordered
 * on the state's stream (work queued there completes first; no device-wide
 * synchronisation).  A caller-owned buffer is left alone. */
int nwq_destroy(nwq_state* st);

/* ---------------------------------------------------------------- circuits */

/* Apply a circuit to a state vector: psi <- U_ng ... U_1 psi (paper Sec. II).
 * Gates are validated, lowered to sweeps (nwq_plan_create) and launched on
 * the state's stream; the operator tables are uploaded (the call waits for
 * that copy) and released stream-ordered, and the call returns without
 * waiting for the sweeps.  gates: host array, read during the call only. */
int nwq_sv_apply_circuit(nwq_state* st, const nwq_gate* gates, size_t ng, uint32_t flags);

/* Apply a circuit with the device noise model to a density matrix
 * (paper Sec. II DM-Sim, Sec. III noise model): per gate
 * rho <- R_q ... D_S(U rho U^dag), with D and R as in nwq_noise_model.
 * nm NULL = noiseless.  Asynchronous like nwq_sv_apply_circuit. */
int nwq_dm_apply_circuit_noisy(nwq_state* st, const nwq_gate* gates, size_t ng,
                               const nwq_noise_model* nm, uint32_t flags);

/* Lower a circuit once for repeated runs (same n, kind and dtype).  Lowering
 * (paper Sec. III, "we optimize the quantum circuit"): each gate, with its
 * noise channels for DM, becomes one operator; adjacent operators sharing
 * qubits are multiplied together when that does not add arithmetic; DM
 * operators defer per-qubit diagonal scale factors to the next operator on
 * the same qubit (flushed on its last one); operators are grouped into sweeps
 * that each read and write the state once.  The plan's operator tables are
 * uploaded to the device on its first run (stream is unused; kept for ABI
 * stability).  Host-only: needs no device. */
int nwq_plan_create(int kind, int n, int dtype, const nwq_gate* gates, size_t ng,
                    const nwq_noise_model* nm, uint32_t flags, void* stream, nwq_plan** out);

/* Plan form by environment: NWQ_PLAN=plain (one gate per pass), fused (the
 * default), tc (tensor-core blocks where supported: complex64 state vectors
 * of >= 12 qubits) or commute (NWQ_PLAN_COMMUTE) applies to nwq_plan_create,
 * nwq_sv_apply_circuit and nwq_dm_apply_circuit_noisy calls whose flags name
 * none of NWQ_PLAN_PLAIN, NWQ_PLAN_TC, NWQ_PLAN_COMMUTE and that give no
 * tuning; read once per process. */

/* Run a plan on a state of matching kind, n and dtype.  Asynchronous. */
int nwq_plan_run(nwq_state* st, const nwq_plan* plan);

/* Plan statistics: number of sweeps, number of device operators, the
 * algorithmic bytes one run moves (one read and one write of the state per
 * sweep), the floating-point instructions (multiply, add or fused
 * multiply-add, each counted once) one run issues per state element, and the
 * bytes of operator tables uploaded to the device.  Any pointer may be NULL. */
int nwq_plan_info(const nwq_plan* plan, int* sweeps, int* ops, double* bytes, double* fma_per_elem,
                  size_t* table_bytes);

/* Debug / test hook: copy the plan's sweep structure to host arrays.
 * sweep_nops[s]: operators in sweep s; op_gate[k]: index of the first input
 * gate folded into operator k (operators listed sweep by sweep).  Sizes from
 * nwq_plan_info.  Host-only; needs no device. */
int nwq_plan_layout(const nwq_plan* plan, int* sweep_nops, int* op_gate, int* op_ngates);

/* Plan shape, chosen by nwq_plan_autotune or by hand (0 = the default):
 *   tile_bits      shared-memory tile of a sweep = 2^tile_bits state elements
 *                  (default 10 for 16-byte, 12 for 8-byte, 13 for 4-byte elements);
 *   fusion_bits    widest operator the planner merges gates into, in state-index
 *                  bits, 2..4 (default 4; a density-matrix qubit spans 2 bits);
 *                  5 = dense five-qubit blocks on the tensor cores (NWQ_PLAN_TC:
 *                  complex64 state vectors of >= 12 qubits; the other fields
 *                  are then unused);
 *   register_bits  complex sweeps: state elements per thread group = 2^register_bits,
 *                  3 or 4 (default 3 for complex128, 4 for complex64). */
typedef struct {
  int tile_bits, fusion_bits, register_bits;
} nwq_plan_tuning;

/* nwq_plan_create with an explicit plan shape (tuning may be NULL). */
int nwq_plan_create_tuned(int kind, int n, int dtype, const nwq_gate* gates, size_t ng,
                          const nwq_noise_model* noise, uint32_t flags, const nwq_plan_tuning* tuning,
                          void* cuda_stream, nwq_plan** out);

/* Autotuner: build the circuit's plan for each candidate shape (tile bits of
 * the default -1, +0, +1; fusion bits 3 and 4 (density matrix: 2 and 4);
 * register bits 3 and 4 for state vectors; for complex64 state vectors of >= 12
 * qubits also the tensor-core plan, fusion bits 5), run each on `scratch` (a state of
 * the circuit's kind, size and dtype; its contents are overwritten) once to
 * warm up and `reps` times under CUDA events on the state's stream, and return
 * the fastest shape in *best with its mean time in *best_ms.  When `tried` is
 * not NULL the first max_tried candidates and their times (ms; negative when
 * the shape could not be built or run) are written there, their count in
 * *ntried.  Synchronises the stream. */
int nwq_plan_autotune(nwq_state* scratch, const nwq_gate* gates, size_t ng, const nwq_noise_model* noise,
                      uint32_t flags, int reps, nwq_plan_tuning* best, double* best_ms,
                      nwq_plan_tuning* tried, double* tried_ms, int max_tried, int* ntried);

/* Test hook: verify the plan's device tables against the bounds the kernels
 * assume (tile geometry, masks, operator and entry offsets, register phases,
 * coefficient ranges); NWQ_EINVAL with the first violation in
 * nwq_last_error().  With the environment variable NWQ_CHECKS=1 every plan
 * is verified when it is created.  Host only. */
int nwq_plan_verify(const nwq_plan* plan);

/* Test hook: the blocks of a tensor-core plan (count = sweeps of
 * nwq_plan_info): qubits[5 b + i] = qubit of local index bit i of block b
 * (ascending), mats[2048 b + 2 (32 r + c) + {0, 1}] = re / im of its FP64
 * matrix entry (r, c), applied in block order.  Either pointer may be NULL.
 * NWQ_EINVAL if the plan is not a tensor-core plan.  Host only. */
int nwq_plan_tc_blocks(const nwq_plan* plan, int* qubits, double* mats);

/* Test hook: the merged operators of a sweep plan (not a tensor-core plan),
 * in the order the sweeps apply them (count = ops of nwq_plan_info): k[o]
 * index bits, bits[4 o + t] = state-index bit of local bit t (-1 past k),
 * mats[2 (256 o + 16 r + c) + {0, 1}] = re / im of entry (r, c) of its
 * 2^k x 2^k matrix (zero outside).  State vectors: bits are qubits.
 * Density matrices: real Pauli-transfer operators on the 2n-bit index of the
 * coefficients r[x + 2^n z] (qubit q owns bits q and q + n), deferred
 * per-qubit scales included.  Any pointer may be NULL.  Host only. */
int nwq_plan_ops(const nwq_plan* plan, int* k, int* bits, double* mats);

/* Test hook: the pass plan nwq_expect_pauli_sum makes for nt terms on an
 * n-qubit state vector (host only).  *npass tiled passes; pass p reads the
 * index bits tile_masks[p] of each tile (its low bits contiguous) and
 * evaluates term records term_range[2p] .. term_range[2p] + term_range[2p+1]
 * - 1; record r: xl[r], zl[r] = the term's x and z bits inside the tile
 * (tile-local positions), zh[r] = its z bits outside, y[r] = |x & z| mod 4,
 * out[r] = its term index (nt: the identity string, for NWQ_EXPECT_NORMALIZE).
 * *nfb terms fb[0 ..] whose X support fits no tile go to the general kernel.
 * Sizes: tile_masks nt + 1 entries, term_range 2 (nt + 1) ints, xl, zl, zh,
 * y and out nt + 1 entries, fb nt entries; any pointer may be NULL. */
int nwq_expect_plan(int n, const nwq_pauli_term* terms, size_t nt, int normalize, int* npass, uint64_t* tile_masks,
                    int* term_range, uint32_t* xl, uint32_t* zl, uint64_t* zh, int* y, int* out, int* nfb, int* fb);

/* Test hook: number of bounded waits (MMA completion) that ran out in the
 * tensor-core kernel on the current device since the library was loaded;
 * 0 in a healthy run.  A wait that runs out leaves its tile unwritten.
 * Synchronises the device. */
int nwq_tc_timeouts(int* count);

/* Test hook of the bounded waits: runs the first block of a tensor-core plan
 * on the state with its MMAs withheld and each MMA-completion wait bounded at
 * 4096 polls, so every wait runs out with nothing in flight; each CTA counts
 * its timeout, frees its tensor memory and returns, leaving its tiles
 * unwritten (the state is unchanged).  *timeouts = waits that ran out in this
 * call; returns NWQ_ETIMEOUT when there were any (the expected outcome).
 * Synchronises the state's stream. */
int nwq_tc_wait_test(nwq_state* st, const nwq_plan* plan, int* timeouts);

/* Test hook: generate and compile (host only; nothing is loaded on a device)
 * the run-time specialised kernel of every eligible sweep of a plan.  Sweeps
 * over at least NWQ_JIT_MIN_BITS index bits (default 18: state vectors of
 * >= 18 qubits, density matrices of >= 9) run such kernels: one per distinct
 * sweep structure, compiled by NVRTC for sm_103a on first use and cached for
 * the process (reusable plans compile before their first run, one-shot plans
 * in the background); set NWQ_JIT=0 to run the interpreted kernels instead.  *eligible: sweeps whose structure and tables
 * fit the specialised kernel; *built: those compiled.  NWQ_EUNSUPPORTED when
 * NVRTC cannot be loaded, with the reason (or the first compiler message) in
 * nwq_last_error(). */
int nwq_plan_jit_check(const nwq_plan* plan, int* eligible, int* built);

/* *dw = 1 when the plan's latest nwq_plan_run took the double-word path
 * (NWQ_PLAN_DW with every sweep's double-word kernel ready), else 0. */
int nwq_plan_last_run_dw(const nwq_plan* plan, int* dw);

/* Arithmetic of the plan's run-time specialised sweep kernels, for roofline
 * accounting (host only): per state element, summed over the sweeps that
 * have such a kernel (*sweeps of them, may be NULL), the multiply-adds and
 * multiplies of the kernels' value type as generated, and *instr_per_elem the
 * arithmetic-pipe instructions they make.  dw = 0: the kernels of the plan's
 * own precision (one FP64 / FP32 instruction each); dw = 1: the double-word
 * kernels of an FP64 plan (a multiply-add is 12 FP32 instructions, a
 * multiply 4). */
int nwq_plan_kernel_arith(const nwq_plan* plan, int dw, double* fma_per_elem, double* mul_per_elem,
                          double* instr_per_elem, int* sweeps);

/* Queue background compilation of the plan's specialised sweep kernels that
 * are not compiled yet (one compiler thread per process) and return at once;
 * *pending (may be NULL): sweeps whose kernel is queued or still compiling.  Sweeps whose
 * kernel is not ready run the interpreted kernel; a serving loop can call
 * this ahead of time for circuit structures it expects.  Host only. */
int nwq_plan_jit_prefetch(const nwq_plan* plan, int* pending);

/* Stop the background kernel compiler: queued compiles are dropped, the one
 * in progress finishes, its thread is joined; later one-shot plans run the
 * interpreted kernel for structures not compiled yet.  Call before the
 * process exits (the Python binding does so from atexit); idempotent. */
int nwq_jit_shutdown(void);

int nwq_plan_destroy(nwq_plan* plan);

/* ---------------------------------------------------------------- measurement */

/* Expectation values of Pauli strings (SV: <psi|P|psi>; DM: Tr(rho P)).
 * Sums are FP64; for complex64 state vectors the products and each warp's
 * partial sum (at most 1024 products) are FP32, everything above FP64.
 * State vectors: one read of the state per group of terms whose X support
 * fits a shared-memory tile (all Z-type strings and the low X supports share
 * the first pass).  flags NWQ_EXPECT_TERMS: out_host[t] = <P_t> (the
 * coefficients are ignored); NWQ_EXPECT_SUM: out_host[0] = sum_t coeff_t <P_t>;
 * NWQ_EXPECT_NORMALIZE: divided by <psi|psi> (Tr rho) of the same pass.
 * Synchronises the stream. */
int nwq_expect_pauli_sum(nwq_state* st, const nwq_pauli_term* terms, size_t nt, double* out_host,
                         uint32_t flags);

/* Outcome distribution of a computational-basis measurement with symmetric
 * readout error e on every bit (paper Sec. III, measurement noise):
 * out_host[b] = sum_b' prod_i C(b_i | b'_i) p(b'), C = [[1-e, e], [e, 1-e]].
 * 2^n doubles.  n <= 30.  Synchronises the stream. */
int nwq_probs(nwq_state* st, double readout_e, double* out_host);

/* Same result as nwq_expect_pauli_sum, computed without allocating any memory.
 * The paper has no counterpart: this variant is for callers that cannot
 * allocate device memory, because another allocator owns all of it (a
 * framework's caching pool, a serving loop admitting work against a fixed
 * memory budget) or because a latency-critical loop must neither wait for
 * nor fail on an allocation.  It calls no cudaMalloc, cudaFree or other
 * allocating routine; its device scratch is one library-owned array of at
 * most 192 KiB that every GPU which loads the library keeps until the
 * process exits.
 *   - nt <= NWQ_NOALLOC_MAX_TERMS, else NWQ_EINVAL (nothing is computed);
 *   - the first call on a device looks up the scratch array's device address
 *     on that device, making that device current for the lookup and then
 *     restoring the caller's device (host threads that change the current
 *     device at the same moment race with it);
 *   - the call cannot be captured in a CUDA graph: it synchronises the
 *     state's stream and copies the results into pageable host memory;
 *   - a state left in the double-word layout by a plan run is read as it is
 *     or converted back in place (no allocation either way);
 *   - all calls share the scratch array (it keeps the last call's contents),
 *     so calls that overlap on the GPU race: serialise them;
 *   - state vectors: at most 256 blocks for strings whose X support fits no
 *     tile, and the tiled grid reduced until its partial sums fit the array;
 *     the results differ from nwq_expect_pauli_sum only in FP64 summation order;
 *   - arguments, flags and results as nwq_expect_pauli_sum; every call
 *     synchronises the state's stream before it returns. */
#define NWQ_NOALLOC_MAX_TERMS 256
int nwq_expect_pauli_sum_noalloc(nwq_state* st, const nwq_pauli_term* terms, size_t nt, double* out_host,
                                 uint32_t flags);

/* Test hook: the launch shape of the state-vector expectation passes for nt
 * terms: *grid tiled-kernel blocks and *fblocks general-kernel blocks, of
 * nwq_expect_pauli_sum (noalloc = 0) or nwq_expect_pauli_sum_noalloc
 * (noalloc = 1).  NWQ_EINVAL for density matrices.  Host only. */
int nwq_expect_launch_shape(const nwq_state* st, size_t nt, int noalloc, int* grid, int* fblocks);

/* ---------------------------------------------------------------- batched VQE */

/* Batched evaluation of parametrised circuits: the inner loop of the VQE use
 * case of paper Sec. III (VQE for the Ising model, where an optimiser such
 * as COBYLA asks for energies of many parameter sets).  Every job starts
 * from |0..0>, runs its template's gates with theta[0] of gate k taken from
 * params[job * nparams + param_idx] when param_idx >= 0, and produces the
 * template's ne energies
 *   out[job * out_stride + e] = sum_t coeffs[e * nterms + t] <P_t> / <psi|psi>
 * (the division removes the norm drift of FP32 storage; <psi|psi> is
 * written to norms[job] when norms is not NULL).  One CTA evaluates one job
 * with the whole 2^n state in shared memory; jobs of different templates
 * (different qubit counts) share one launch.  F64 batches compute in
 * double words by default: the state in shared memory as float pairs
 * (h + l, |x - h - l| <= 2^-47 |x| when split from FP64), gates, norms and
 * term products in double-word arithmetic on the FP32 pipe (Joldes, Muller,
 * Popescu 2017: exact FMA-based products, TwoSum), per-thread sums as
 * compensated float pairs added across the CTA in FP64; gate matrices and
 * energies in FP64.  NWQ_BATCH_FP64_PIPE selects FP64 arithmetic throughout.
 * Limits: n <= 13 (F64) or
 * 14 (F32); gate kinds CX, CZ, SWAP, RZZ and every one-qubit kind (angles
 * from parameters on RX, RY, RZ, P, U3 and RZZ); MAT2 is not supported. */
typedef struct {
  int32_t n;                    /* qubits */
  const nwq_gate* gates;        /* host, read during nwq_batch_create */
  size_t ngates;
  const nwq_pauli_term* terms;  /* host; coeff fields ignored */
  size_t nterms;
  const double* coeffs;         /* host, ne * nterms energy weights */
  int32_t ne;                   /* energies per job (>= 1) */
} nwq_batch_template;

typedef struct nwq_batch nwq_batch;

enum nwq_batch_flags {
  NWQ_BATCH_GRAPH = 1u,     /* launch through a captured CUDA graph, captured on first use and
                               recaptured when pointers or the job count change */
  NWQ_BATCH_FP64_PIPE = 2u  /* F64 batches: arithmetic on the FP64 pipe instead of the default
                               double words (below) */
};

/* Validate and upload templates.  The device tables are allocated and
 * uploaded stream-ordered on stream (the call synchronises that stream) and
 * freed on it by nwq_batch_destroy. */
int nwq_batch_create(int dtype, const nwq_batch_template* templates, int ntemplates, int nparams,
                     void* stream, nwq_batch** out);

/* Evaluate njobs jobs, asynchronous on stream.  params: device, njobs *
 * nparams doubles.  job_template: device, njobs ints (template of each job;
 * NULL = template 0 for all jobs, allowed only with one template; a job whose
 * index is out of range gets NaN energies).  out:
 * device, njobs * out_stride doubles (out_stride >= the largest ne).
 * norms: device, njobs doubles, or NULL.  Runs of one batch object must not
 * overlap (they share its work-queue counter). */
int nwq_batch_run(nwq_batch* b, const double* params, const int32_t* job_template, int njobs, double* out,
                  int out_stride, double* norms, void* stream, uint32_t flags);

/* Free the batch: its tables are released stream-ordered on the creation
 * stream, so runs queued on that stream complete first; runs on other
 * streams must have completed (synchronise them) before this call. */
/* Kernel shape of a batch: threads per CTA (128, 256 or 512; default 256)
 * and gate-fusion width (0, default: gates applied one by one; 1: every run
 * of one-qubit gates on a qubit, up to the next two-qubit gate on it, is one
 * 2x2 matrix per job, multiplied out in FP64 when the job starts). */
int nwq_batch_set_shape(nwq_batch* b, int threads, int fusion);

/* Autotuner of the batched kernel: run (params, job_template, njobs, out)
 * once to warm up and `reps` times timed (CUDA events on `stream`) for every
 * shape, keep the fastest on b and return it (best_* may be NULL).  `out` is
 * overwritten; synchronises the stream. */
int nwq_batch_autotune(nwq_batch* b, const double* params, const int32_t* job_template, int njobs, double* out,
                       int out_stride, int reps, void* stream, int* best_threads, int* best_fusion,
                       double* best_ms);

int nwq_batch_destroy(nwq_batch* b);

/* ---------------------------------------------------------------- trajectories */

/* Noisy state vectors by quantum trajectories: the Monte-Carlo unravelling of
 * the device noise model of nwq_dm_apply_circuit_noisy (paper Sec. III), a
 * stochastic alternative to the density matrix whose memory grows as 2^n
 * instead of 4^n; the average over trajectories of <psi|P|psi> converges to
 * Tr(rho P).  Every trajectory starts from |0..0> and, after each gate:
 *   - depolarising p (one draw x when p > 0): if x < (4^k - 1) p / 4^k the
 *     Pauli string s = 1 + floor(x 4^k / p) (<= 4^k - 1) is applied, s & 3
 *     on the gate's first qubit and s >> 2 on its second (0 I, 1 X, 2 Y, 3 Z);
 *   - thermal relaxation on each gate qubit q (when the gate time > 0):
 *     amplitude damping gamma then phase damping lambda (sqrt(1-gamma)
 *     sqrt(1-lambda) = exp(-t/T2); needs T2 <= 2 T1), one draw x each: with
 *     P1 = prob(q = 1), the jump |0><1| (resp. |1><1|) when x < rate P1, else
 *     diag(1, sqrt(1 - rate)); the state is renormalised in FP64.
 * The random draws are inputs: `uniforms` (device) holds ntraj rows of
 * nwq_traj_draws(...) values in [0, 1), consumed in the order above.
 * out (device) [t * ne + e] = sum_k coeffs[e * nt + k] <P_k> / <psi|psi> of
 * trajectory t.  Gates: the kinds of the batched kernel with fixed angles
 * (param_idx = -1), no MAT2; n <= 13 (F64) / 14 (F32).  Arithmetic as the
 * batched kernel: F64 in double words (NWQ_DW=0 in the environment, read on
 * every call, selects the FP64 pipe), F32 with FP64-accurate reductions
 * (exact products, compensated float-pair sums); the P1 sums and the
 * renormalisation factors are FP64.  Synchronises the stream. */
int nwq_traj_draws(const nwq_gate* gates, size_t ng, int n, const nwq_noise_model* noise, size_t* draws);
int nwq_traj_run(int n, int dtype, const nwq_gate* gates, size_t ng, const nwq_noise_model* noise,
                 const nwq_pauli_term* terms, size_t nt, const double* coeffs, int ne, const double* uniforms,
                 int ntraj, double* out, void* stream);

/* One template, nsets parameter sets: create + run + destroy.  params and
 * out are device pointers (out: nsets * ne doubles); terms, coeffs host.
 * Synchronises the stream before returning. */
int nwq_batch_energy(int n, int dtype, const nwq_gate* gates, size_t ng, const double* params,
                     int nsets, int nparams, const nwq_pauli_term* terms, size_t nt,
                     const double* coeffs, int ne, double* out, void* stream);

/* ---------------------------------------------------------------- misc */

/* Message of the last failed call on the calling thread. */
const char* nwq_last_error(void);

/* Wait for the state's stream. */
int nwq_device_sync(nwq_state* st);

/* Number of device kernels this library has launched in this process
 * (monotonic; for accounting in benchmarks). */
uint64_t nwq_launch_count(void);

/* Measurement helper (the paper has no counterpart): the arithmetic rate of
 * one pipe of the current device, for roofline denominators.  A grid of
 * several CTAs per SM runs independent FMA chains per thread (8 FP64 or 16
 * FP32 chains, enough to cover the pipe latency) for about 60 ms after a
 * warm-up launch, timed with CUDA events on a private stream; *fma_per_second
 * = thread-level FMA instructions retired per second (2 flops each).  Uses
 * and frees a small device buffer; synchronises its own stream only. */
enum nwq_probe { NWQ_PROBE_FP64_FMA = 0, NWQ_PROBE_FP32_FMA = 1 };
int nwq_peak_probe(int what, double* fma_per_second);

#ifdef __cplusplus
}
#endif
#endif /* NWQGB_H */
