// Internal layout shared by the host planner and the device kernels.
//
// A circuit is lowered to a list of *operators*: a 2^k x 2^k matrix acting on
// k <= 4 bits of the state index (SV: complex matrix on the gate's qubits;
// DM: real Pauli-transfer matrix on bits q and q+n of every touched qubit).
// Operators are grouped into *sweeps*: one sweep stages tiles of 2^T
// elements (T tile bits = the low contiguous bits 0..m-1 plus h strided high
// bits) in shared memory, applies its operators in order, and writes the tile
// back, so the state is read and written once per sweep.
#pragma once
#include <cstdint>

namespace nwq {

constexpr int kMaxK = 4;          // bits per operator
constexpr int kMaxTileBits = 15;  // shared-memory tile <= 2^15 elements
constexpr int kMaxHigh = 15;

// Row kinds: how output row i of an operator is produced.
enum : uint8_t {
  ROW_ID = 0,    // unchanged (no arithmetic, no store)
  ROW_MOVE = 1,  // copy (or negated copy) of one input: no arithmetic
  ROW_GEN = 2    // optional +-input (the row's unit entry) plus coefficient * input terms
};

// Complex entry kinds (coefficient structure, selects the cheapest arithmetic).
enum : uint8_t { CE_RE = 0, CE_IM = 1, CE_GEN = 2 };

// Output row i of an operator:
//   ROW_MOVE: out = sgn * in[boff]
//   ROW_GEN : out = [sgn * in[boff] if has_base] + sum_e c_e in[off_e]
// Real operators keep all terms in one entry list (cnt[0] entries); complex
// operators keep three kind-homogeneous lists: cnt[0] real-coefficient,
// cnt[1] imaginary-coefficient and cnt[2] general entries, in that order.
struct RowMeta {
  uint16_t out;    // tile-local offset of output i
  uint16_t boff;   // tile-local offset of the unit entry's input
  uint16_t beg;    // first entry of the row (relative to DevOp::ent)
  uint8_t kind;    // ROW_*
  uint8_t base;    // 0: no unit entry, 1: +input, 2: -input
  uint8_t cnt[3];  // entry counts (see above)
  uint8_t pad;
};

struct alignas(16) DevOp {
  uint8_t k;              // number of operator bits
  uint8_t lb[4];          // tile-local bit position of operator bit j
  uint8_t slb[4];         // the same positions sorted ascending (k used)
  uint8_t pad[3];
  uint32_t ent;           // first entry (index into the plan's entry array)
  RowMeta row[16];
};

template <class R>
struct EntR {  // real entry: out += c * in[off]
  R c;
  uint32_t off;
};

template <class R>
struct EntC {  // complex entry: out += (re + i im) * in[off]
  R re, im;
  uint32_t off;
  uint32_t kind;  // CE_*
};

struct SweepDesc {
  uint64_t hmask;  // global mask of the high tile bits
  uint64_t fmask;  // global mask of the bits that index tiles (not in the tile)
  int32_t T;       // tile bits
  int32_t m;       // low contiguous tile bits (global bits 0..m-1)
  int32_t h;       // high tile bits
  int32_t nops;    // operators in this sweep
  uint32_t op0;    // index of the first operator
  uint32_t ent0;   // index of the first entry of the sweep's operators
  uint32_t nent;   // number of entries of the sweep's operators
  uint32_t ph0;    // complex sweeps: first phase (absolute index)
  uint32_t nph;    //                 number of phases
  uint32_t pop0;   //                 first phase operator
  uint32_t npop;   //                 number of phase operators
  uint32_t pc0;    //                 first coefficient
  uint32_t npc;    //                 number of coefficients
  uint8_t hpos[kMaxHigh];  // global position of high tile bit i (ascending, >= m)
  uint8_t prb;             // complex sweeps: register bits per thread group (3 or 4)
};

}  // namespace nwq

namespace nwq {

// ---------------------------------------------------------------- register phases
// Complex (state-vector) sweeps run as *phases*: a phase fixes 4 tile bits U;
// every thread holds the 16 elements of a group (all values of the U bits)
// in registers and applies the phase's operators there, so shared memory is
// read and written once per phase instead of once per operator.  Dense and
// permutation operators act on a subset of U; diagonal operators may act on
// any tile bits (their factor depends only on the element's index).
enum : uint8_t { PO_DIAG = 0, PO_PERM = 1, PO_DENSE = 2, PO_KRON = 3 };

// DENSE structure classes (select the arithmetic at compile time).
// PD_XROTU: X-rotation with a unit diagonal [[1, i y01], [i y10, 1]] (its cos
// factor deferred by the planner into a later diagonal): 2 FMA per entry pair.
enum : uint8_t { PD_GEN = 0, PD_REAL = 1, PD_XROT = 2, PD_XROTU = 3 };

// Dispatch code of a phase operator (one switch in the kernel):
//   0..15   DIAG, register-bit mask SU       16 + m  PERM on register mask m
//   32 + m  DENSE general   48 + m  real     64 + m  X-rotation form
//   80      KRON: one 2x2 matrix per register bit set in `mask`
constexpr uint8_t PCODE_KRON = 80;

struct PhaseOp {
  uint8_t cls;       // PO_*
  uint8_t k;         // operator bits (DIAG: up to 8)
  uint8_t mask;      // PERM / DENSE: register positions (operator bit t = t-th set bit);
                     // DIAG: register part SU; KRON: register bits that carry a matrix
  uint8_t form;      // DENSE: PD_*; KRON: 2 bits per register bit
  uint32_t coef;     // DIAG: 2^k factors; DENSE: 2^k x 2^k row-major; KRON: 4 entries per register bit
  uint8_t dnu;       // DIAG: operator bits outside the register bits (their positions in dpos)
  uint8_t code;      // dispatch code (above)
  uint8_t pad[6];
  uint8_t dpos[8];   // DIAG: tile-local bit positions of the out-of-register bits, low to high
  uint8_t perm[8];   // PERM: output i = (perm[i] & 0x80 ? -1 : 1) * input (perm[i] & 15), k <= 2
};
static_assert(sizeof(PhaseOp) == 32, "PhaseOp must be 32 bytes");

struct alignas(16) PhaseDesc {
  uint8_t u[4];      // tile-local positions of the register bits, ascending
  uint32_t op0;      // first PhaseOp (absolute index)
  uint32_t nops;
  uint32_t pad;      // 16-byte records keep the shared-memory copies aligned
};
static_assert(sizeof(PhaseDesc) == 16, "PhaseDesc must be 16 bytes");

}  // namespace nwq
