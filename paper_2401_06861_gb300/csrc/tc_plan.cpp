// Host planner of tensor-core plans: the gate stream fused into dense
// five-qubit blocks (each one 32 x 32 complex matrix, multiplied out in FP64),
// the blocks' tile geometry, and the TF32 hi / lo tables of their real form.
//
// Fusion (this build's reading of "we optimize the quantum circuit",
// paper Sec. III, in the form that feeds tensor cores), in two steps:
//   1. fold: a gate whose qubits are a subset of those of the latest gate on
//      each of them is multiplied into that gate (CX * RZ * CX becomes one
//      diagonal two-qubit gate), unless that would turn a diagonal gate into
//      a non-diagonal one;
//   2. blocks, one at a time: scan the gates not yet placed, in order, and
//      place each that fits the block's 5 qubits and may move ahead of every
//      gate skipped so far on its qubits (a gate may pass a skipped gate it
//      shares no qubit with, and a diagonal gate may pass a skipped diagonal
//      gate, since diagonal matrices commute); a skipped gate keeps its
//      qubits from later gates that may not pass it.  Blocks with fewer than
//      5 qubits are padded with idle qubits (identity).
#include <algorithm>
#include <cstring>
#include <vector>

#include "planner.hpp"
#include "tc.hpp"

namespace nwq {

namespace {

struct Building {
  std::vector<int> qs;  // local bit i <-> qubit qs[i] (insertion order)
  std::vector<cd> M;    // 2^|qs| square, row-major
  int gate0 = 0, ngates = 0;
};

int local_pos(const Building& b, int q) {
  for (size_t i = 0; i < b.qs.size(); i++)
    if (b.qs[i] == q) return (int)i;
  return -1;
}

// Add qubit q as the next local bit: M <- I (x) M.
void add_qubit(Building& b, int q) {
  const int nq = (int)b.qs.size(), d = 1 << nq, d2 = 2 * d;
  std::vector<cd> E((size_t)d2 * d2, 0.0);
  for (int i = 0; i < d2; i++)
    for (int j = 0; j < d2; j++)
      if ((i >> nq) == (j >> nq)) E[(size_t)i * d2 + j] = b.M[(size_t)(i & (d - 1)) * d + (j & (d - 1))];
  b.qs.push_back(q);
  b.M.swap(E);
}

// M <- G M for a gate G on qubits already in the block.
void apply_gate(Building& b, const BitOp& op) {
  const int d = 1 << b.qs.size(), dk = 1 << op.k;
  int pos[4];
  int opmask = 0;
  for (int t = 0; t < op.k; t++) {
    pos[t] = local_pos(b, op.bits[t]);
    opmask |= 1 << pos[t];
  }
  std::vector<cd> R(b.M.size());
  for (int base = 0; base < d; base++) {
    if (base & opmask) continue;
    int idx[16];
    for (int a = 0; a < dk; a++) {
      int r = base;
      for (int t = 0; t < op.k; t++)
        if ((a >> t) & 1) r |= 1 << pos[t];
      idx[a] = r;
    }
    for (int col = 0; col < d; col++)
      for (int a = 0; a < dk; a++) {
        cd s = 0.0;
        for (int c = 0; c < dk; c++) s += op.m[(size_t)a * dk + c] * b.M[(size_t)idx[c] * d + col];
        R[(size_t)idx[a] * d + col] = s;
      }
  }
  b.M.swap(R);
}

// Pad to 5 qubits with the lowest idle qubits and order the local bits by qubit.
void finish(Building& b, TcBlock& out) {
  for (int q = 0; (int)b.qs.size() < kTcBits; q++)
    if (local_pos(b, q) < 0) add_qubit(b, q);
  int order[kTcBits];
  for (int i = 0; i < kTcBits; i++) order[i] = i;
  std::sort(order, order + kTcBits, [&](int x, int y) { return b.qs[x] < b.qs[y]; });
  for (int i = 0; i < kTcBits; i++) out.q[i] = b.qs[order[i]];
  // new local index bit i = old local bit order[i]
  auto old_index = [&](int j) {
    int o = 0;
    for (int i = 0; i < kTcBits; i++)
      if ((j >> i) & 1) o |= 1 << order[i];
    return o;
  };
  out.U.assign(32 * 32, 0.0);
  for (int i = 0; i < 32; i++)
    for (int j = 0; j < 32; j++) out.U[(size_t)i * 32 + j] = b.M[(size_t)old_index(i) * 32 + old_index(j)];
  out.gate0 = b.gate0;
  out.ngates = b.ngates;
}

// Round to TF32 (10 explicit mantissa bits), to nearest with ties away from
// zero, on the FP32 bit pattern (finite inputs).
float tf32_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

}  // namespace

namespace {

bool diagonal(const std::vector<cd>& m, int k) {
  const int d = 1 << k;
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++)
      if (i != j && m[(size_t)i * d + j] != cd(0.0)) return false;
  return true;
}

constexpr size_t kTcLookahead = 1u << 16;  // gates scanned per block

}  // namespace

bool tc_fuse(const std::vector<BitOp>& ops, int n, std::vector<TcBlock>& out, std::string& err) {
  if (n < kTcMinQubits) {
    err = "tensor-core plans need at least 12 qubits";
    return false;
  }
  // 1. fold gates into the latest gate on their qubits (matrices on that gate's qubit order)
  std::vector<Building> g;
  std::vector<char> diag;
  std::vector<int> last(n, -1);
  for (const BitOp& op : ops) {
    if (op.k < 1 || op.k > 2) {
      err = "tensor-core fusion takes one- and two-qubit gates";
      return false;
    }
    const int a = last[op.bits[0]];
    bool fold = a >= 0;
    for (int t = 1; t < op.k; t++) fold = fold && last[op.bits[t]] == a;
    for (int t = 0; fold && t < op.k; t++) fold = local_pos(g[a], op.bits[t]) >= 0;
    if (fold) {
      Building c = g[a];
      apply_gate(c, op);
      const bool dg = diagonal(c.M, (int)c.qs.size());
      if (!diag[a] || dg) {
        c.ngates += op.ngates;
        g[a] = std::move(c);
        diag[a] = dg;
        continue;
      }
    }
    Building b;
    b.M.assign(1, 1.0);
    b.gate0 = op.gate0;
    for (int t = 0; t < op.k; t++) add_qubit(b, op.bits[t]);
    apply_gate(b, op);
    b.ngates = op.ngates;
    diag.push_back(diagonal(b.M, op.k));
    g.push_back(std::move(b));
    for (int t = 0; t < op.k; t++) last[op.bits[t]] = (int)g.size() - 1;
  }
  // 2. blocks, one at a time, over the gates not yet placed
  const size_t m = g.size();
  const uint64_t full = (n >= 64) ? ~0ull : ((1ull << n) - 1);
  std::vector<char> placed(m, 0);
  out.clear();
  size_t pos = 0;
  while (pos < m) {
    Building b;
    b.M.assign(1, 1.0);
    b.gate0 = g[pos].gate0;
    uint64_t S = 0, blk_all = 0, blk_nd = 0;
    size_t scanned = 0;
    for (size_t i = pos; i < m && scanned < kTcLookahead; i++) {
      if (placed[i]) continue;
      scanned++;
      uint64_t Q = 0;
      for (int q : g[i].qs) Q |= 1ull << q;
      const bool ok = !(Q & blk_all) && (diag[i] || !(Q & blk_nd)) && __builtin_popcountll(S | Q) <= kTcBits;
      if (ok) {
        S |= Q;
        placed[i] = 1;
        BitOp op;  // the folded gate on its own qubits
        op.k = (int)g[i].qs.size();
        for (int t = 0; t < op.k; t++) op.bits[t] = g[i].qs[t];
        op.m = g[i].M;
        for (int q : g[i].qs)
          if (local_pos(b, q) < 0) add_qubit(b, q);
        apply_gate(b, op);
        b.ngates += g[i].ngates;
        b.gate0 = std::min(b.gate0, g[i].gate0);
      } else if (diag[i]) {
        blk_nd |= Q;
      } else {
        blk_all |= Q;
        if (blk_all == full) break;
      }
    }
    out.emplace_back();
    finish(b, out.back());
    while (pos < m && placed[pos]) pos++;
  }
  return true;
}

void tc_geometry(const int* q, int n, TcGeom& g) {
  std::memset(&g, 0, sizeof(g));
  uint64_t smask = 0;
  for (int i = 0; i < kTcBits; i++) smask |= 1ull << q[i];
  int rows[kTcRowBits], nr = 0;
  for (int b = 0; nr < kTcRowBits; b++)
    if (!((smask >> b) & 1)) rows[nr++] = b;
  // Operand byte offset of column m (row bits) and block index j:
  // (j >> 4) * 16384 + m * 128 + (((j >> 1) & 7) ^ (m & 7)) * 16 + (j & 1) * 8,
  // the XOR of one weight per set bit.  bank[] = the weight's share of
  // offset bits 4..6 (the 16-byte bank group).
  static const uint32_t jw[kTcBits] = {8, 16, 32, 64, 16384};
  static const uint32_t mw[kTcRowBits] = {128 ^ 16, 256 ^ 32, 512 ^ 64, 1024, 2048, 4096, 8192};
  struct Bit {
    int qubit;
    uint32_t w, bank;
  };
  std::vector<Bit> other;  // tile bits except block bit 0, ascending by qubit
  for (int b = 0; b < n; b++) {
    int i = 0;
    while (i < kTcBits && q[i] != b) i++;
    if (i < kTcBits) {
      if (i > 0) other.push_back({b, jw[i], (jw[i] >> 4) & 7u});
      continue;
    }
    int r = 0;
    while (r < kTcRowBits && rows[r] != b) r++;
    if (r < kTcRowBits) other.push_back({b, mw[r], (mw[r] >> 4) & 7u});
  }
  // roles: 0 = block bit 0 (the pair); 1..5 = lane bits, the five lowest other
  // tile qubits with lane bits 0..2 covering bank bits 1, 2, 4 (always possible:
  // the five hold m0..m(a-1) and j1..j(b) with a + b = 5); 6..7 warp; 8..11 loop.
  int role_q[kTcTileBits];
  uint32_t role_w[kTcTileBits];
  role_q[0] = q[0];
  role_w[0] = jw[0];
  bool low = false;  // a block qubit among 0..3
  for (int i = 0; i < kTcBits; i++) low |= q[i] < 4;
  if (!low) {
    // rows m0..m6 on the lane and warp bits in order, K chunks j1..j4 on the loop steps:
    // each thread's accumulator lane is the column it loaded (direct write-back), the lane
    // bits 0..2 (m0..m2) cover bank bits 1, 2, 4, and with qubits 0..3 rows a warp access
    // still covers runs of 16 consecutive amplitudes (128 bytes)
    for (int r = 0; r < kTcRowBits; r++) {
      role_q[1 + r] = rows[r];
      role_w[1 + r] = mw[r];
    }
    for (int i = 1; i < kTcBits; i++) {
      role_q[kTcRowBits + i] = q[i];
      role_w[kTcRowBits + i] = jw[i];
    }
  } else {
    std::vector<int> order;  // indices into other, in role order 1..11
    std::vector<char> used(other.size(), 0);
    for (int k = 0; k < 3; k++)
      for (int c = 0; c < 5; c++)
        if (!used[c] && other[c].bank == (1u << k)) {
          used[c] = 1;
          order.push_back(c);
          break;
        }
    for (int c = 0; c < (int)other.size(); c++)
      if (!used[c]) order.push_back(c);
    for (int p = 1; p < kTcTileBits; p++) {
      role_q[p] = other[order[p - 1]].qubit;
      role_w[p] = other[order[p - 1]].w;
    }
  }
  g.direct = 1;
  for (int p = 0; p < kTcTileBits; p++) {
    g.gw[p] = 1ull << role_q[p];
    g.sw[p] = role_w[p];
    if (p >= 1 && role_w[p] != (p <= kTcRowBits ? mw[p - 1] : jw[p - kTcRowBits])) g.direct = 0;
  }
  uint64_t tmask = smask;
  for (int r = 0; r < kTcRowBits; r++) tmask |= 1ull << rows[r];
  int f = 0;
  for (int b = 0; b < n; b++)
    if (!((tmask >> b) & 1)) g.fw[f++] = 1ull << b;
  g.ntiles = 1u << (n - kTcTileBits);
}

void tc_matrix_tables(const TcBlock& b, float* out) {
  // real form over interleaved (re, im): row 2a / 2a+1 = re / im of output a
  for (int a = 0; a < 32; a++)
    for (int c = 0; c < 32; c++) {
      const cd u = b.U[(size_t)a * 32 + c];
      const double v[2][2] = {{u.real(), -u.imag()}, {u.imag(), u.real()}};
      for (int ra = 0; ra < 2; ra++)
        for (int rc = 0; rc < 2; rc++) {
          const size_t idx = (size_t)(2 * a + ra) * 64 + (2 * c + rc);
          const double x = v[ra][rc];
          const float hi = tf32_host((float)x);
          out[idx] = hi;
          out[4096 + idx] = tf32_host((float)(x - (double)hi));
        }
    }
}

bool build_tc_plan(const std::vector<BitOp>& ops, Plan& plan, std::string& err) {
  std::vector<TcBlock> blocks;
  if (!tc_fuse(ops, plan.n, blocks, err)) return false;
  plan.tc = true;
  plan.tcb = std::move(blocks);
  const size_t nb = plan.tcb.size();
  plan.tcg.resize(nb);
  plan.tctab.assign(nb * kTcMatFloats, 0.f);
  plan.op_gate0.clear();
  plan.op_ngates.clear();
  for (size_t i = 0; i < nb; i++) {
    tc_geometry(plan.tcb[i].q, plan.n, plan.tcg[i]);
    tc_matrix_tables(plan.tcb[i], plan.tctab.data() + i * kTcMatFloats);
    plan.op_gate0.push_back(plan.tcb[i].gate0);
    plan.op_ngates.push_back(plan.tcb[i].ngates);
  }
  const double state_bytes = (double)plan.elem_bytes * (double)(1ull << plan.n);
  plan.bytes = 2.0 * state_bytes * (double)nb;
  plan.fma_per_elem = 384.0 * (double)nb;  // TF32 multiply-adds: 3 products x 64 per real x 2 reals
  return true;
}

}  // namespace nwq
