// Host-side verification of a plan's device tables (the library's
// replacement for a device sanitizer): every index a kernel derives from the
// tables is checked against the bounds the kernels assume, so a planner bug
// shows up as an error message on the host instead of an out-of-bounds access
// on the GPU.  Run on every plan when NWQ_CHECKS=1, and by the tests through
// nwq_plan_verify.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "planner.hpp"

namespace nwq {

namespace {

bool fail_at(std::string& err, const char* what, size_t sweep, long item) {
  char buf[160];
  std::snprintf(buf, sizeof(buf), "plan check: %s (sweep %zu, item %ld)", what, sweep, item);
  err = buf;
  return false;
}

// Bits of v outside `span` (tile-local positions of an operator's bits).
uint32_t outside(uint32_t v, uint32_t span) { return v & ~span; }

int popc(uint32_t v) { return __builtin_popcount(v); }

// Tensor-core plans: each block's tile geometry must place every amplitude
// of the state in exactly one tile position (global offsets are distinct
// single bits covering the n qubits, qubit 0 first so pairs are 16-byte
// vectors) and every tile position in a distinct operand slot (the operand
// weights are exactly the 12 weights of the shared-memory layout).
bool verify_tc(const Plan& p, std::string& err) {
  const size_t nb = p.tcb.size();
  if (p.n < kTcMinQubits || p.n > 34 || p.tcg.size() != nb || p.tctab.size() != nb * kTcMatFloats ||
      p.op_gate0.size() != nb || p.op_ngates.size() != nb)
    return fail_at(err, "tensor-core plan tables", 0, -1);
  static const uint32_t want[kTcTileBits] = {8, 16, 32, 64, 16384, 128 ^ 16, 256 ^ 32, 512 ^ 64, 1024, 2048, 4096, 8192};
  const uint64_t full = (1ull << p.n) - 1;
  for (size_t b = 0; b < nb; b++) {
    const TcBlock& blk = p.tcb[b];
    const TcGeom& g = p.tcg[b];
    for (int i = 0; i < kTcBits; i++)
      if (blk.q[i] < 0 || blk.q[i] >= p.n || (i && blk.q[i] <= blk.q[i - 1]))
        return fail_at(err, "tensor-core block qubits", b, i);
    if (blk.U.size() != 1024) return fail_at(err, "tensor-core block matrix", b, -1);
    uint64_t seen = 0;
    uint32_t wseen = 0;
    for (int t = 0; t < kTcTileBits; t++) {
      const uint64_t w = g.gw[t];
      if (!w || (w & (w - 1)) || (w & seen) || (w & ~full)) return fail_at(err, "tensor-core tile offsets", b, t);
      seen |= w;
      int k = 0;
      while (k < kTcTileBits && want[k] != g.sw[t]) k++;
      if (k == kTcTileBits || ((wseen >> k) & 1)) return fail_at(err, "tensor-core operand offsets", b, t);
      wseen |= 1u << k;
    }
    if (g.sw[0] != 8 || g.gw[0] != (1ull << blk.q[0])) return fail_at(err, "tensor-core pair bit", b, 0);
    for (int i = 0; i < kTcBits; i++)
      if (!((seen >> blk.q[i]) & 1)) return fail_at(err, "tensor-core block qubit outside its tile", b, i);
    for (int f = 0; f < kTcMaxFree; f++) {
      const uint64_t w = g.fw[f];
      if (f < p.n - kTcTileBits) {
        if (!w || (w & (w - 1)) || (w & seen) || (w & ~full)) return fail_at(err, "tensor-core tile index", b, f);
        seen |= w;
      } else if (w) {
        return fail_at(err, "tensor-core tile index", b, f);
      }
    }
    if (seen != full || g.ntiles != (1u << (p.n - kTcTileBits))) return fail_at(err, "tensor-core tile cover", b, -1);
    // Emulate the kernel's addressing of one tile (thread tid, step i, pair
    // element e): each amplitude must land in the operand slot of its column
    // m (the 7 lowest qubits outside the block) and block index j, a pair in
    // one 16-byte chunk, each slot once; each warp's accesses must be coalesced
    // (lane bits below qubit 6, or runs of 16 amplitudes); with the direct
    // write-back, thread tid must own column tid and step i chunk i.
    int rows[kTcRowBits], nr = 0;
    uint64_t bmask = 0;
    for (int i = 0; i < kTcBits; i++) bmask |= 1ull << blk.q[i];
    for (int q = 0; nr < kTcRowBits; q++)
      if (!((bmask >> q) & 1)) rows[nr++] = q;
    std::vector<char> slot(4096, 0);
    for (int tid = 0; tid < 128; tid++)
      for (int i = 0; i < 16; i++) {
        uint64_t goff = 0;
        uint32_t soff = 0;
        for (int k = 1; k < 8; k++)
          if ((tid >> (k - 1)) & 1) {
            goff += g.gw[k];
            soff ^= g.sw[k];
          }
        for (int k = 0; k < 4; k++)
          if ((i >> k) & 1) {
            goff += g.gw[8 + k];
            soff ^= g.sw[8 + k];
          }
        if (soff & 15) return fail_at(err, "tensor-core pair alignment", b, tid);
        for (int e = 0; e < 2; e++) {
          const uint64_t amp = goff + (e ? g.gw[0] : 0);
          const uint32_t s = soff ^ (e ? g.sw[0] : 0);
          uint32_t j = 0, m = 0;
          for (int k = 0; k < kTcBits; k++) j |= (uint32_t)((amp >> blk.q[k]) & 1) << k;
          for (int r = 0; r < kTcRowBits; r++) m |= (uint32_t)((amp >> rows[r]) & 1) << r;
          const uint32_t want_s = (j >> 4) * 16384u + m * 128u + ((((j >> 1) & 7u) ^ (m & 7u)) << 4) + (j & 1u) * 8u;
          if (s != want_s || s >= 32768u || (s & 7u) || slot[s >> 3]++)
            return fail_at(err, "tensor-core operand addressing", b, tid);
          if (g.direct && (m != (uint32_t)tid || (j >> 1) != (uint32_t)i))
            return fail_at(err, "tensor-core direct write-back mapping", b, tid);
          // coalescing: the lane bits are qubits below 6, or (direct write-back geometry) lane
          // bits 0..3 are qubits 0..3, so each warp access covers runs of 16 amplitudes
          const bool lanes_low = ((g.gw[1] | g.gw[2] | g.gw[3] | g.gw[4] | g.gw[5]) >> 6) == 0;
          const bool lanes_runs = g.direct && (g.gw[1] | g.gw[2] | g.gw[3] | g.gw[4]) == 15;
          if (e == 0 && !lanes_low && !lanes_runs)
            return fail_at(err, "tensor-core lane bits above qubit 5", b, tid);
        }
      }
  }
  return true;
}

}  // namespace

bool verify_plan(const Plan& p, std::string& err) {
  if (p.tc) return verify_tc(p, err);
  const uint64_t full = p.B >= 64 ? ~0ull : ((1ull << p.B) - 1);
  const size_t nent = p.ent_bytes ? p.ents.size() / p.ent_bytes : 0;
  const size_t cbytes = p.dtype == NWQ_F64 ? 16 : 8;
  const size_t ncoef = p.pcoef.size() / cbytes;
  size_t op_next = 0;
  for (size_t s = 0; s < p.sweeps.size(); s++) {
    const SweepDesc& sd = p.sweeps[s];
    if (sd.T < 1 || sd.T > kMaxTileBits || sd.T > p.B || sd.m < 0 || sd.h < 0 || sd.h > kMaxHigh ||
        sd.m + sd.h != sd.T)
      return fail_at(err, "tile geometry", s, -1);
    const uint64_t low = (1ull << sd.m) - 1;
    uint64_t hm = 0;
    for (int i = 0; i < sd.h; i++) {
      if (sd.hpos[i] < sd.m || sd.hpos[i] >= p.B || (i && sd.hpos[i] <= sd.hpos[i - 1]))
        return fail_at(err, "high tile bit positions", s, i);
      hm |= 1ull << sd.hpos[i];
    }
    if (hm != sd.hmask || (sd.fmask != (full & ~(low | hm))) || __builtin_popcountll(sd.fmask) != p.B - sd.T)
      return fail_at(err, "tile and tile-index masks do not partition the index bits", s, -1);
    if (sd.op0 != op_next || sd.op0 + (size_t)sd.nops > p.ops.size()) return fail_at(err, "operator range", s, -1);
    op_next = sd.op0 + sd.nops;
    if ((size_t)sd.ent0 + sd.nent > nent) return fail_at(err, "entry range", s, -1);
    const uint32_t tmask = (uint32_t)((1ull << sd.T) - 1);
    for (int o = 0; o < sd.nops; o++) {
      const DevOp& d = p.ops[sd.op0 + o];
      if (d.k < 1 || d.k > kMaxK) return fail_at(err, "operator width", s, o);
      uint32_t span = 0;
      for (int t = 0; t < d.k; t++) {
        if (d.lb[t] >= sd.T || ((span >> d.lb[t]) & 1)) return fail_at(err, "operator bit positions", s, o);
        span |= 1u << d.lb[t];
        if (t && d.slb[t] <= d.slb[t - 1]) return fail_at(err, "sorted operator bits", s, o);
      }
      uint32_t sspan = 0;
      for (int t = 0; t < d.k; t++) sspan |= 1u << d.slb[t];
      if (sspan != span) return fail_at(err, "sorted operator bits", s, o);
      if (d.ent < sd.ent0 || d.ent > sd.ent0 + sd.nent) return fail_at(err, "operator entry base", s, o);
      for (int i = 0; i < (1 << d.k); i++) {
        const RowMeta& rm = d.row[i];
        uint32_t want = 0;
        for (int t = 0; t < d.k; t++) want |= (uint32_t)((i >> t) & 1) << d.lb[t];
        if (rm.out != want || (rm.out & ~tmask)) return fail_at(err, "row output offset", s, o);
        if (rm.kind > ROW_GEN || rm.base > 2) return fail_at(err, "row kind", s, o);
        if (rm.kind == ROW_ID) continue;
        if (rm.base && outside(rm.boff, span)) return fail_at(err, "unit-entry offset outside the operator", s, o);
        const size_t cnt = (size_t)rm.cnt[0] + rm.cnt[1] + rm.cnt[2];
        if (rm.kind == ROW_MOVE && (cnt || !rm.base)) return fail_at(err, "copy row with entries", s, o);
        if (!p.is_complex && (rm.cnt[1] || rm.cnt[2])) return fail_at(err, "complex entries in a real plan", s, o);
        const size_t e0 = (size_t)d.ent + rm.beg;
        if (e0 + cnt > (size_t)sd.ent0 + sd.nent) return fail_at(err, "row entries beyond the sweep", s, o);
        for (size_t e = 0; e < cnt; e++) {
          uint32_t off;
          std::memcpy(&off, &p.ents[(e0 + e) * p.ent_bytes + (p.is_complex ? 2 : 1) * (p.dtype == NWQ_F64 ? 8 : 4)],
                      4);
          if (outside(off, span)) return fail_at(err, "entry offset outside the operator", s, o);
        }
      }
    }
    if (!p.is_complex || p.phases.empty() || sd.nops == 0 || sd.nph == 0) continue;
    // register phases of complex sweeps
    const int RB = sd.prb;
    if (RB != 3 && RB != 4) return fail_at(err, "register bits", s, -1);
    if ((size_t)sd.ph0 + sd.nph > p.phases.size() || (size_t)sd.pop0 + sd.npop > p.pops.size() ||
        (size_t)sd.pc0 + sd.npc > ncoef)
      return fail_at(err, "phase table ranges", s, -1);
    for (uint32_t ph = 0; ph < sd.nph; ph++) {
      const PhaseDesc& P = p.phases[sd.ph0 + ph];
      uint32_t umask = 0;
      for (int t = 0; t < RB; t++) {
        if (P.u[t] >= sd.T || (t && P.u[t] <= P.u[t - 1])) return fail_at(err, "phase register bits", s, ph);
        umask |= 1u << P.u[t];
      }
      if (P.op0 < sd.pop0 || (size_t)P.op0 + P.nops > (size_t)sd.pop0 + sd.npop)
        return fail_at(err, "phase operator range", s, ph);
      for (uint32_t q = 0; q < P.nops; q++) {
        const PhaseOp& po = p.pops[P.op0 + q];
        const int code = po.code, NR = 1 << RB;
        size_t need = 0;  // coefficients read from po.coef on
        if (code < 16) {
          if (code >= NR || po.dnu > 8) return fail_at(err, "diagonal operator", s, ph);
          for (int t = 0; t < po.dnu; t++)
            if (po.dpos[t] >= sd.T || ((umask >> po.dpos[t]) & 1)) return fail_at(err, "diagonal index bits", s, ph);
          need = (size_t)1 << (popc(code) + po.dnu);
        } else if (code == PCODE_KRON) {
          if (po.mask == 0 || po.mask >= NR) return fail_at(err, "KRON register mask", s, ph);
          for (int b = 0; b < 4; b++)
            if ((po.mask >> b) & 1) {
              need = 4 * (size_t)(b + 1);
              if (((po.form >> (2 * b)) & 3) > PD_XROTU) return fail_at(err, "KRON form", s, ph);
            }
        } else {
          const int M = code & 15, cls = code >> 4;
          if (cls < 1 || cls > 4 || M == 0 || M >= NR || popc(M) > 2) return fail_at(err, "operator code", s, ph);
          const int D = 1 << popc(M);
          if (cls == 1) {
            for (int i = 0; i < D; i++)
              if ((po.perm[i] & 15) >= D) return fail_at(err, "permutation index", s, ph);
          } else {
            if (cls == 4 && D != 2) return fail_at(err, "X-rotation width", s, ph);
            need = (size_t)D * D;
          }
        }
        if (need && (po.coef < sd.pc0 || (size_t)po.coef + need > (size_t)sd.pc0 + sd.npc))
          return fail_at(err, "coefficients beyond the sweep's table", s, ph);
      }
    }
  }
  if (op_next != p.ops.size()) return fail_at(err, "operators outside every sweep", p.sweeps.size(), -1);
  return true;
}

}  // namespace nwq
