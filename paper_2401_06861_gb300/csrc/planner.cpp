// Host planner: gate matrices, Pauli-transfer matrices of gates and noise
// channels, algebraic merging of adjacent operators, and the greedy grouping
// of operators into shared-memory sweeps.
//
// Paper mapping: Sec. II (SV-Sim applies a stream of gates to a state vector;
// DM-Sim applies gates and noise to a density matrix), Sec. III (noise model
// made of depolarising, thermal-relaxation and readout noise; "we optimize
// the quantum circuit" -- here: operator merging and sweep fusion).
#include "planner.hpp"

#include <algorithm>
#include <array>
#include <map>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <unordered_map>

namespace nwq {

static const cd I1(0.0, 1.0);

// ------------------------------------------------------------------ gates
static void set2(cd* U, cd a, cd b, cd c, cd d) {
  U[0] = a; U[1] = b; U[2] = c; U[3] = d;
}

int gate_matrix(const nwq_gate& g, double t0, cd* U) {
  const double* th = g.theta;
  const double r2 = std::sqrt(0.5);
  double c = std::cos(0.5 * t0), s = std::sin(0.5 * t0);
  switch (g.kind) {
    case NWQ_GATE_ID: set2(U, 1, 0, 0, 1); return 1;
    case NWQ_GATE_X: set2(U, 0, 1, 1, 0); return 1;
    case NWQ_GATE_Y: set2(U, 0, -I1, I1, 0); return 1;
    case NWQ_GATE_Z: set2(U, 1, 0, 0, -1); return 1;
    case NWQ_GATE_H: set2(U, r2, r2, r2, -r2); return 1;
    case NWQ_GATE_S: set2(U, 1, 0, 0, I1); return 1;
    case NWQ_GATE_SDG: set2(U, 1, 0, 0, -I1); return 1;
    case NWQ_GATE_T: set2(U, 1, 0, 0, cd(r2, r2)); return 1;
    case NWQ_GATE_TDG: set2(U, 1, 0, 0, cd(r2, -r2)); return 1;
    case NWQ_GATE_SX: set2(U, cd(0.5, 0.5), cd(0.5, -0.5), cd(0.5, -0.5), cd(0.5, 0.5)); return 1;
    case NWQ_GATE_RX: set2(U, c, cd(0, -s), cd(0, -s), c); return 1;
    case NWQ_GATE_RY: set2(U, c, -s, s, c); return 1;
    case NWQ_GATE_RZ: set2(U, std::polar(1.0, -0.5 * t0), 0, 0, std::polar(1.0, 0.5 * t0)); return 1;
    case NWQ_GATE_P: set2(U, 1, 0, 0, std::polar(1.0, t0)); return 1;
    case NWQ_GATE_U3:
      set2(U, c, -std::polar(s, th[2]), std::polar(s, th[1]), std::polar(c, th[1] + th[2]));
      return 1;
    case NWQ_GATE_MAT1:
      if (!g.mat) return 0;
      for (int k = 0; k < 4; k++) U[k] = cd(g.mat[2 * k], g.mat[2 * k + 1]);
      return 1;
    case NWQ_GATE_CX:
      for (int k = 0; k < 16; k++) U[k] = 0;
      U[0] = 1; U[2 * 4 + 2] = 1; U[1 * 4 + 3] = 1; U[3 * 4 + 1] = 1;
      return 2;
    case NWQ_GATE_CZ:
      for (int k = 0; k < 16; k++) U[k] = 0;
      U[0] = 1; U[5] = 1; U[10] = 1; U[15] = -1;
      return 2;
    case NWQ_GATE_SWAP:
      for (int k = 0; k < 16; k++) U[k] = 0;
      U[0] = 1; U[1 * 4 + 2] = 1; U[2 * 4 + 1] = 1; U[15] = 1;
      return 2;
    case NWQ_GATE_RZZ: {
      for (int k = 0; k < 16; k++) U[k] = 0;
      cd even = std::polar(1.0, -0.5 * t0), odd = std::polar(1.0, 0.5 * t0);
      U[0] = even; U[5] = odd; U[10] = odd; U[15] = even;
      return 2;
    }
    case NWQ_GATE_MAT2:
      if (!g.mat) return 0;
      for (int k = 0; k < 16; k++) U[k] = cd(g.mat[2 * k], g.mat[2 * k + 1]);
      return 2;
  }
  return 0;
}

static bool check_gate(const nwq_gate& g, int n, int nq, std::string& err) {
  for (int j = 0; j < nq; j++)
    if (g.q[j] < 0 || g.q[j] >= n) {
      err = "gate qubit out of range";
      return false;
    }
  if (nq == 2 && g.q[0] == g.q[1]) {
    err = "two-qubit gate on one qubit";
    return false;
  }
  return true;
}

// ------------------------------------------------------------------ snapping
static inline double snap(double v) {
  if (std::fabs(v) < 5e-16) return 0.0;
  if (std::fabs(v - 1.0) < 4e-16) return 1.0;
  if (std::fabs(v + 1.0) < 4e-16) return -1.0;
  return v;
}
static void snap_all(std::vector<cd>& m) {
  for (auto& z : m) z = cd(snap(z.real()), snap(z.imag()));
}

// ------------------------------------------------------------------ SV lowering
bool lower_sv(const nwq_gate* g, size_t ng, int n, std::vector<BitOp>& out, std::string& err) {
  out.clear();
  out.reserve(ng);
  for (size_t i = 0; i < ng; i++) {
    cd U[16];
    int k = gate_matrix(g[i], g[i].theta[0], U);
    if (!k) {
      err = "unknown gate kind or missing matrix";
      return false;
    }
    if (!check_gate(g[i], n, k, err)) return false;
    BitOp op;
    op.k = k;
    for (int j = 0; j < k; j++) op.bits[j] = g[i].q[j];
    op.m.assign(U, U + (1 << (2 * k)));
    snap_all(op.m);
    op.gate0 = (int)i;
    out.push_back(std::move(op));
  }
  return true;
}

// ------------------------------------------------------------------ Pauli transfer
// Local Pauli index of a k-qubit operator: j = x (k bits) + (z << k); the
// string is i^{|x&z|} X^x Z^z, i.e. per qubit (x,z) = (0,0) I, (1,0) X,
// (1,1) Y, (0,1) Z.  Its action: P|b> = i^{|x&z|} (-1)^{|b&z|} |b^x>.
static cd pauli_elem(int x, int z, int row, int col) {
  if (row != (col ^ x)) return 0.0;
  static const cd ip[4] = {cd(1, 0), cd(0, 1), cd(-1, 0), cd(0, -1)};
  cd ph = ip[__builtin_popcount(x & z) & 3];
  return (__builtin_popcount(col & z) & 1) ? -ph : ph;
}

// R[i][j] = Tr(P_i U P_j U^dag) / 2^k  (real for Hermitian P_i, P_j).
static void unitary_ptm(int k, const cd* U, std::vector<cd>& R) {
  int d = 1 << k, np = 1 << (2 * k), km = d - 1;
  R.assign((size_t)np * np, 0.0);
  std::vector<cd> A((size_t)d * d), T((size_t)d * d);
  for (int j = 0; j < np; j++) {
    int xj = j & km, zj = j >> k;
    // T = U P_j ; A = T U^dag
    for (int r = 0; r < d; r++)
      for (int c = 0; c < d; c++) T[r * d + c] = U[r * d + (c ^ xj)] * pauli_elem(xj, zj, c ^ xj, c);
    for (int r = 0; r < d; r++)
      for (int c = 0; c < d; c++) {
        cd acc = 0;
        for (int t = 0; t < d; t++) acc += T[r * d + t] * std::conj(U[c * d + t]);
        A[r * d + c] = acc;
      }
    for (int i = 0; i < np; i++) {
      int xi = i & km, zi = i >> k;
      cd tr = 0;
      for (int a = 0; a < d; a++) tr += pauli_elem(xi, zi, a ^ xi, a) * A[a * d + (a ^ xi)];
      R[(size_t)i * np + j] = cd(tr.real() / d, 0.0);
    }
  }
}

static void matmul(int d, const std::vector<cd>& A, const std::vector<cd>& B, std::vector<cd>& C) {
  std::vector<cd> out((size_t)d * d, 0.0);
  for (int i = 0; i < d; i++)
    for (int t = 0; t < d; t++) {
      cd a = A[(size_t)i * d + t];
      if (a == cd(0.0)) continue;
      for (int j = 0; j < d; j++) out[(size_t)i * d + j] += a * B[(size_t)t * d + j];
    }
  C.swap(out);
}

// Depolarising channel on all k qubits of the operator, as a Pauli-transfer
// matrix: every string that is not the identity on them is scaled by 1-p.
static void depol_ptm(int k, double p, std::vector<cd>& D) {
  int np = 1 << (2 * k);
  D.assign((size_t)np * np, 0.0);
  for (int j = 0; j < np; j++) D[(size_t)j * np + j] = j == 0 ? 1.0 : 1.0 - p;
}

// Thermal relaxation of operator qubit w: I -> I, X -> eta X, Y -> eta Y,
// Z -> (1-gamma) Z + gamma I.
static void relax_ptm(int k, int w, double gamma, double eta, std::vector<cd>& Rm) {
  int np = 1 << (2 * k);
  Rm.assign((size_t)np * np, 0.0);
  for (int j = 0; j < np; j++) {
    int xw = (j >> w) & 1, zw = (j >> (k + w)) & 1;
    if (!xw && !zw) Rm[(size_t)j * np + j] = 1.0;
    else if (xw) Rm[(size_t)j * np + j] = eta;
    else {
      Rm[(size_t)j * np + j] = 1.0 - gamma;
      Rm[(size_t)j * np + (j ^ (1 << (k + w)))] = gamma;
    }
  }
}

bool lower_dm(const nwq_gate* g, size_t ng, int n, const nwq_noise_model* nm, std::vector<BitOp>& out,
              std::string& err) {
  out.clear();
  out.reserve(ng);
  if (nm && nm->n < n) {
    err = "noise model covers fewer qubits than the state";
    return false;
  }
  if (nm && (!nm->T1_us || !nm->T2_us)) {
    err = "noise model without T1/T2 arrays";
    return false;
  }
  std::vector<cd> R, D, Rl;
  // A noisy circuit repeats the same gate on the same qubits (every Trotter
  // step): the transfer matrix of gate plus noise is built once per distinct
  // (kind, angles, qubits) in this call and reused.  Explicit-matrix gates are
  // not memoised (their key would be the matrix itself).
  std::map<std::array<double, 6>, std::vector<cd>> memo;
  for (size_t i = 0; i < ng; i++) {
    cd U[16];
    int k = gate_matrix(g[i], g[i].theta[0], U);
    if (!k) {
      err = "unknown gate kind or missing matrix";
      return false;
    }
    if (!check_gate(g[i], n, k, err)) return false;
    const bool memo_ok = g[i].kind != NWQ_GATE_MAT1 && g[i].kind != NWQ_GATE_MAT2;
    const std::array<double, 6> key{(double)g[i].kind, g[i].theta[0], g[i].theta[1], g[i].theta[2],
                                    (double)g[i].q[0], (double)(k == 2 ? g[i].q[1] : -1)};
    if (memo_ok) {
      auto hit = memo.find(key);
      if (hit != memo.end()) {
        BitOp op;
        op.k = 2 * k;
        for (int j = 0; j < k; j++) {
          op.bits[j] = g[i].q[j];
          op.bits[k + j] = g[i].q[j] + n;
        }
        op.m = hit->second;
        op.gate0 = (int)i;
        out.push_back(std::move(op));
        continue;
      }
    }
    unitary_ptm(k, U, R);
    snap_all(R);
    int np = 1 << (2 * k);
    bool noisy = nm && !((nm->flags & NWQ_NOISE_RZ_VIRTUAL) && g[i].kind == NWQ_GATE_RZ);
    if (noisy) {
      double p = k == 2 ? nm->p2 : nm->p1;
      if (nm->flags & NWQ_NOISE_DEPOL_PAULI_FORM) p = p * np / (np - 1.0);
      if (p < 0 || p > np / (np - 1.0)) {
        err = "depolarising parameter out of range";
        return false;
      }
      if (p > 0) {
        depol_ptm(k, p, D);
        matmul(np, D, R, R);
      }
      double t = k == 2 ? nm->t2q_ns : nm->t1q_ns;
      if (t > 0) {
        for (int w = 0; w < k; w++) {
          int q = g[i].q[w];
          double T1 = nm->T1_us[q], T2 = nm->T2_us[q];
          if (!(T1 > 0) || !(T2 > 0)) {
            err = "T1 and T2 must be positive";
            return false;
          }
          double gamma = 1.0 - std::exp(-t / (T1 * 1e3));
          double eta = std::exp(-t / (T2 * 1e3));
          relax_ptm(k, w, gamma, eta, Rl);
          matmul(np, Rl, R, R);
        }
      }
      snap_all(R);
    }
    BitOp op;
    op.k = 2 * k;
    for (int j = 0; j < k; j++) {
      op.bits[j] = g[i].q[j];
      op.bits[k + j] = g[i].q[j] + n;
    }
    op.m = R;
    op.gate0 = (int)i;
    if (memo_ok) memo.emplace(key, R);
    out.push_back(std::move(op));
  }
  return true;
}

// Per-qubit map from Pauli coefficients (local index x + 2z: I, X, Z, Y) to
// the standard vec(rho) entries (local index r + 2c): rho = (1/2) sum r_P P.
void pauli_to_rho_matrix(cd M[16]) {
  const cd h(0.5, 0.0), ih(0.0, 0.5);
  cd m[16] = {h, 0, h, 0,     // (r0,c0) = (I + Z)/2
              0, h, 0, ih,    // (r1,c0) = (X + iY)/2
              0, h, 0, -ih,   // (r0,c1) = (X - iY)/2
              h, 0, -h, 0};   // (r1,c1) = (I - Z)/2
  std::memcpy(M, m, sizeof(m));
}

void rho_to_pauli_matrix(cd M[16]) {
  const cd o(1.0, 0.0), i1(0.0, 1.0);
  cd m[16] = {o, 0, 0, o,      // I = rho00 + rho11
              0, o, o, 0,      // X = rho10 + rho01
              o, 0, 0, -o,     // Z = rho00 - rho11
              0, -i1, i1, 0};  // Y = i (rho01 - rho10)
  std::memcpy(M, m, sizeof(m));
}

// ------------------------------------------------------------------ cost model
// Floating-point instructions (multiply, add or FMA, each counted once) the
// kernels issue per state element.  A row is a copy of its first unit entry
// (+-1, handled with integer sign flips) plus one FMA per remaining entry:
// real coefficient 1 (DM), complex coefficient 4, real or imaginary 2 (SV).
// Identity rows and pure copies cost nothing.
static inline bool is_unit(cd v) { return v.imag() == 0.0 && (v.real() == 1.0 || v.real() == -1.0); }

double op_cost(const BitOp& op, bool is_complex) {
  int d = 1 << op.k;
  double total = 0;
  for (int i = 0; i < d; i++) {
    int cnt = 0;
    bool have_base = false, idrow = false;
    double c = 0;
    for (int j = 0; j < d; j++) {
      cd v = op.m[(size_t)i * d + j];
      if (v == cd(0.0)) continue;
      cnt++;
      if (j == i && v == cd(1.0)) idrow = true;
      if (!have_base && is_unit(v)) {
        have_base = true;
        continue;
      }
      if (is_complex)
        c += (v.imag() == 0.0 || v.real() == 0.0) ? 2 : 4;
      else
        c += 1;
    }
    if (cnt == 1 && idrow) continue;
    total += c;
  }
  return total / d;
}

// ------------------------------------------------------------------ DM rescaling
// Deferred per-qubit scale factors (Pauli basis).  Each operator's output rows
// of the form "one non-identity Pauli on qubit w, identity elsewhere" are
// divided by their pivot (largest entry, the diagonal on ties), which turns that entry
// into +-1 (free) and often the whole row into an identity row.  The divisor
// becomes a pending diagonal factor of qubit w, multiplied into the columns of
// the next operator on w; on the last operator of each qubit nothing is
// deferred, so the plan's result is the exact state.  This only changes the
// rounding (relative 1e-16 per operator).
// Reorder an operator's bits (permuting its matrix) to the DM layout
// [q_0 .. q_{m-1}, q_0+n .. q_{m-1}+n] with q ascending.
static void canonical_dm_bits(BitOp& op, int n) {
  int qs[2], kq = 0;
  for (int t = 0; t < op.k; t++)
    if (op.bits[t] < n) qs[kq++] = op.bits[t];
  std::sort(qs, qs + kq);
  int nb[4];
  for (int w = 0; w < kq; w++) {
    nb[w] = qs[w];
    nb[kq + w] = qs[w] + n;
  }
  bool same = true;
  for (int t = 0; t < op.k; t++) same &= nb[t] == op.bits[t];
  if (same) return;
  int src[4];  // new local bit t comes from old local bit src[t]
  for (int t = 0; t < op.k; t++)
    for (int u = 0; u < op.k; u++)
      if (op.bits[u] == nb[t]) src[t] = u;
  int dim = 1 << op.k;
  auto map = [&](int inew) {
    int iold = 0;
    for (int t = 0; t < op.k; t++) iold |= ((inew >> t) & 1) << src[t];
    return iold;
  };
  std::vector<cd> m((size_t)dim * dim);
  for (int i = 0; i < dim; i++)
    for (int j = 0; j < dim; j++) m[(size_t)i * dim + j] = op.m[(size_t)map(i) * dim + map(j)];
  op.m.swap(m);
  for (int t = 0; t < op.k; t++) op.bits[t] = nb[t];
}

// Per-qubit factors stay within [lim, 1/lim], so a stored coefficient is at
// most 1/lim^n times its true value (in range for FP32 with lim = 2^-6 and
// n <= 16 qubits; FP64 uses 2^-40).
static void rescale_dm(std::vector<BitOp>& ops, int n, double lim) {
  for (BitOp& op : ops) canonical_dm_bits(op, n);
  std::vector<std::array<double, 4>> pend((size_t)n, {1.0, 1.0, 1.0, 1.0});
  std::vector<long> last((size_t)n, -1);
  for (size_t i = 0; i < ops.size(); i++)
    for (int w = 0; w < ops[i].k / 2; w++) last[ops[i].bits[w]] = (long)i;
  for (size_t i = 0; i < ops.size(); i++) {
    BitOp& op = ops[i];
    const int kq = op.k / 2, dim = 1 << op.k;
    auto comp = [&](int j, int w) { return ((j >> w) & 1) | (((j >> (kq + w)) & 1) << 1); };
    for (int j = 0; j < dim; j++) {
      double dj = 1.0;
      for (int w = 0; w < kq; w++) dj *= pend[op.bits[w]][comp(j, w)];
      if (dj != 1.0)
        for (int r = 0; r < dim; r++) op.m[(size_t)r * dim + j] *= dj;
    }
    double s[2][4] = {{1, 1, 1, 1}, {1, 1, 1, 1}};
    for (int w = 0; w < kq; w++) {
      pend[op.bits[w]] = {1.0, 1.0, 1.0, 1.0};
      if (last[op.bits[w]] == (long)i) continue;  // flush on the qubit's last operator
      for (int a = 1; a < 4; a++) {
        int r = ((a & 1) << w) | ((a >> 1) << (kq + w));
        // pivot: the largest entry (the diagonal when it is among the largest),
        // so every normalised entry of that row is at most 1 in magnitude
        double piv = op.m[(size_t)r * dim + r].real();
        for (int j = 0; j < dim; j++) {
          double v = op.m[(size_t)r * dim + j].real();
          if (std::fabs(v) > std::fabs(piv)) piv = v;
        }
        if (std::isfinite(piv) && std::fabs(piv) >= lim && std::fabs(piv) <= 1.0 / lim) s[w][a] = piv;
      }
    }
    // Rows with a non-identity Pauli on both qubits are divided by a product of
    // two pivots; if that makes any coefficient larger than 4, defer less.
    auto trial_max = [&](const double (&sc)[2][4]) {
      double mx = 0;
      for (int r = 0; r < dim; r++) {
        double dr = 1.0;
        for (int w = 0; w < kq; w++) dr *= sc[w][comp(r, w)];
        for (int j = 0; j < dim; j++) mx = std::max(mx, std::fabs(op.m[(size_t)r * dim + j].real() / dr));
      }
      return mx;
    };
    if (kq == 2 && trial_max(s) > 4.0) {
      double only0[2][4] = {{s[0][0], s[0][1], s[0][2], s[0][3]}, {1, 1, 1, 1}};
      double only1[2][4] = {{1, 1, 1, 1}, {s[1][0], s[1][1], s[1][2], s[1][3]}};
      if (trial_max(only0) <= 4.0) {
        for (int a = 0; a < 4; a++) s[1][a] = 1.0;
      } else if (trial_max(only1) <= 4.0) {
        for (int a = 0; a < 4; a++) s[0][a] = 1.0;
      } else {
        for (int a = 0; a < 4; a++) s[0][a] = s[1][a] = 1.0;
      }
    }
    for (int r = 0; r < dim; r++) {
      double dr = 1.0;
      for (int w = 0; w < kq; w++) dr *= s[w][comp(r, w)];
      if (dr != 1.0)
        for (int j = 0; j < dim; j++) op.m[(size_t)r * dim + j] /= dr;
    }
    for (int w = 0; w < kq; w++) pend[op.bits[w]] = {s[w][0], s[w][1], s[w][2], s[w][3]};
    // no snapping here: the factors are exact scalings, and small entries
    // may multiply large stored values
  }
}

// ------------------------------------------------------------------ merging
static void embed(const BitOp& op, const int* ubits, int ku, std::vector<cd>& E) {
  int du = 1 << ku, d = 1 << op.k;
  int pos[4];
  for (int t = 0; t < op.k; t++)
    for (int u = 0; u < ku; u++)
      if (ubits[u] == op.bits[t]) pos[t] = u;
  int opmask = 0;
  for (int t = 0; t < op.k; t++) opmask |= 1 << pos[t];
  E.assign((size_t)du * du, 0.0);
  for (int i = 0; i < du; i++)
    for (int j = 0; j < du; j++) {
      if ((i & ~opmask) != (j & ~opmask)) continue;
      int si = 0, sj = 0;
      for (int t = 0; t < op.k; t++) {
        si |= ((i >> pos[t]) & 1) << t;
        sj |= ((j >> pos[t]) & 1) << t;
      }
      E[(size_t)i * du + j] = op.m[(size_t)si * d + sj];
    }
}

// B after A, as one operator on the union of their bits (or false if the
// union is wider than max_bits).
static bool compose(const BitOp& A, const BitOp& B, int max_bits, BitOp& C) {
  if (A.k > max_bits || B.k > max_bits) return false;  // an operand is already wider than the limit
  int ubits[8], ku = 0;
  for (int t = 0; t < A.k; t++) ubits[ku++] = A.bits[t];
  for (int t = 0; t < B.k; t++) {
    bool have = false;
    for (int u = 0; u < ku; u++) have |= ubits[u] == B.bits[t];
    if (!have) {
      if (ku >= max_bits) return false;
      ubits[ku++] = B.bits[t];
    }
  }
  std::vector<cd> EA, EB;
  embed(A, ubits, ku, EA);
  embed(B, ubits, ku, EB);
  C.k = ku;
  for (int u = 0; u < ku; u++) C.bits[u] = ubits[u];
  matmul(1 << ku, EB, EA, C.m);
  snap_all(C.m);
  C.gate0 = A.gate0;
  C.ngates = A.ngates + B.ngates;
  return true;
}

static uint64_t op_mask(const BitOp& op) {
  uint64_t m = 0;
  for (int t = 0; t < op.k; t++) m |= 1ull << op.bits[t];
  return m;
}

static bool is_diagonal(const BitOp& op) {
  int d = 1 << op.k;
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++)
      if (i != j && op.m[(size_t)i * d + j] != cd(0.0)) return false;
  return true;
}

static void merge_ops(std::vector<BitOp>& ops, bool is_complex, int max_bits) {
  if (ops.empty()) return;
  std::vector<BitOp> out;
  out.reserve(ops.size());
  BitOp cur = std::move(ops[0]);
  double ccur = op_cost(cur, is_complex);
  for (size_t i = 1; i < ops.size(); i++) {
    BitOp C;
    bool share = (op_mask(cur) & op_mask(ops[i])) != 0;
    if (share && compose(cur, ops[i], max_bits, C)) {
      // complex operators run in register phases: keep non-diagonal products
      // within 2 bits (diagonal ones may use all 4)
      if (is_complex && C.k > 2 && !is_diagonal(C)) {
        out.push_back(std::move(cur));
        cur = std::move(ops[i]);
        ccur = op_cost(cur, is_complex);
        continue;
      }
      double cc = op_cost(C, is_complex);
      double cb = op_cost(ops[i], is_complex);
      if (cc <= ccur + cb + 1e-12) {
        cur = std::move(C);
        ccur = cc;
        continue;
      }
    }
    out.push_back(std::move(cur));
    cur = std::move(ops[i]);
    ccur = op_cost(cur, is_complex);
  }
  out.push_back(std::move(cur));
  ops.swap(out);
}

// ------------------------------------------------------------------ register phases
static bool is_signed_perm(const BitOp& op) {
  int d = 1 << op.k;
  for (int i = 0; i < d; i++) {
    int cnt = 0;
    for (int j = 0; j < d; j++) {
      cd v = op.m[(size_t)i * d + j];
      if (v == cd(0.0)) continue;
      if (!is_unit(v)) return false;
      cnt++;
    }
    if (cnt != 1) return false;
  }
  return true;
}

// Group each complex sweep's operators into phases of RB register bits, then
// within a phase merge consecutive diagonal operators into one diagonal of at
// most 8 bits and consecutive one-bit dense operators on distinct register
// bits into one KRON operator, so one dispatch does the work of several.
// Register bits per thread group (elements per thread = 2^RB); NWQ_PHASE_RB
// overrides it for tuning experiments.
static int phase_register_bits(bool f64, int requested) {
  if (requested == 3 || requested == 4) return requested;
  if (const char* e = std::getenv("NWQ_PHASE_RB")) {
    int v = std::atoi(e);
    if (v == 3 || v == 4) return v;
  }
  return f64 ? 3 : 4;
}

struct PDiag {  // diagonal over up to 8 tile-local bits
  int k = 0;
  int lbits[8];
  std::vector<cd> f;  // 2^k factors, operator index bit t = lbits[t]
};

static void build_phases(const std::vector<BitOp>& ops, const std::vector<int>& order, Plan& plan, int rb) {
  const bool f64 = plan.dtype == NWQ_F64;
  const int RB = phase_register_bits(f64, rb);
  plan.phases.clear();
  plan.pops.clear();
  plan.pcoef.clear();
  size_t ncoef = 0;
  auto push_coef = [&](cd v) {
    if (f64) {
      double c[2] = {v.real(), v.imag()};
      plan.pcoef.insert(plan.pcoef.end(), (unsigned char*)c, (unsigned char*)c + sizeof(c));
    } else {
      float c[2] = {(float)v.real(), (float)v.imag()};
      plan.pcoef.insert(plan.pcoef.end(), (unsigned char*)c, (unsigned char*)c + sizeof(c));
    }
    ncoef++;
  };
  auto form_of = [](const cd* m, int k) -> uint8_t {
    int d = 1 << k;
    bool real = true;
    for (int e = 0; e < d * d; e++) real &= m[e].imag() == 0.0;
    if (real) return PD_REAL;
    if (k == 1 && m[0].imag() == 0.0 && m[3].imag() == 0.0 && m[1].real() == 0.0 && m[2].real() == 0.0) return PD_XROT;
    return PD_GEN;
  };
  // FP64 plans whose sweeps all run in register phases defer the cos factor of
  // X-rotations (|tan| <= 1) into a global scalar: the rotation keeps a unit
  // diagonal (2 FP64 instructions per element instead of 4) and the scalar is
  // folded into the next diagonal operator (free), or applied as a
  // one-coefficient diagonal when its binary exponent leaves [-200, 200]
  // ([-60, 60] for double-word plans, whose values have float exponents) and
  // at the end of the plan.
  bool defer = f64;
  const double scalar_range = plan.dw ? 60.0 : 200.0;
  for (const SweepDesc& sd : plan.sweeps) {
    if (sd.nops == 0) continue;
    bool ok = sd.T >= RB;
    for (int s = 0; s < sd.nops && ok; s++) {
      const BitOp& op = ops[order[sd.op0 + s]];
      ok = is_diagonal(op) || op.k <= 2;
    }
    defer &= ok;
  }
  cd gscale = 1.0;
  double saved = 0.0;  // FP instructions per element removed by the deferral
  auto push_scalar = [&]() {  // one-coefficient diagonal: every element times gscale
    PhaseOp po;
    std::memset(&po, 0, sizeof(po));
    po.cls = PO_DIAG;
    po.coef = (uint32_t)ncoef;
    po.code = 0;
    push_coef(gscale);
    plan.pops.push_back(po);
    gscale = 1.0;
    saved -= 4.0;
  };
  for (SweepDesc& sd : plan.sweeps) {
    sd.prb = (uint8_t)RB;
    sd.ph0 = (uint32_t)plan.phases.size();
    sd.pop0 = (uint32_t)plan.pops.size();
    sd.pc0 = (uint32_t)ncoef;
    bool ok = sd.T >= RB;  // register groups need RB tile bits
    for (int s = 0; s < sd.nops && ok; s++) {
      const BitOp& op = ops[order[sd.op0 + s]];
      ok = is_diagonal(op) || op.k <= 2;  // register operators act on at most 2 bits
    }
    if (!ok) {  // the row kernel runs this sweep
      sd.nph = sd.npop = sd.npc = 0;
      continue;
    }
    int local[64];
    for (int b = 0; b < 64; b++) local[b] = -1;
    for (int b = 0; b < sd.m; b++) local[b] = b;
    for (int i = 0; i < sd.h; i++) local[sd.hpos[i]] = sd.m + i;
    std::vector<std::pair<uint32_t, std::vector<int>>> groups;  // (U mask, op indices)
    uint32_t U = 0;
    std::vector<int> cur;
    for (int s = 0; s < sd.nops; s++) {
      const BitOp& op = ops[order[sd.op0 + s]];
      if (!is_diagonal(op)) {
        uint32_t bm = 0;
        for (int t = 0; t < op.k; t++) bm |= 1u << local[op.bits[t]];
        if (__builtin_popcount(U | bm) > RB) {
          groups.push_back({U, cur});
          U = 0;
          cur.clear();
        }
        U |= bm;
      }
      cur.push_back(order[sd.op0 + s]);
    }
    if (!cur.empty()) groups.push_back({U, cur});
    for (auto& gr : groups) {
      uint32_t Um = gr.first;
      // fill to RB register bits from the highest tile bits (the low bits stay
      // with the lanes of a warp)
      for (int b = sd.T - 1; b >= 0 && __builtin_popcount(Um) < RB; b--) Um |= 1u << b;
      PhaseDesc pd;
      std::memset(&pd, 0, sizeof(pd));
      int upos[4] = {0, 0, 0, 0}, nu = 0;
      for (int b = 0; b < sd.T; b++)
        if ((Um >> b) & 1) upos[nu++] = b;
      for (int p = 0; p < RB; p++) pd.u[p] = (uint8_t)upos[p];
      pd.op0 = (uint32_t)plan.pops.size();
      auto rpos = [&](int lb) {
        for (int q = 0; q < RB; q++)
          if (upos[q] == lb) return q;
        return -1;
      };

      // ---- pending macro-operators
      PDiag dg;          // dg.k == 0: none
      bool kron_any = false;
      cd kron[4][4];     // per register bit: 2x2 (identity when absent)
      uint8_t kron_mask = 0;
      auto flush_diag = [&]() {
        if (dg.k == 0) return;
        PhaseOp po;
        std::memset(&po, 0, sizeof(po));
        po.cls = PO_DIAG;
        po.k = (uint8_t)dg.k;
        po.coef = (uint32_t)ncoef;
        int upos_of[8], outt[8], nout = 0;
        uint8_t SU = 0;
        for (int t = 0; t < dg.k; t++) {
          upos_of[t] = rpos(dg.lbits[t]);
          if (upos_of[t] < 0) {
            outt[nout] = t;
            po.dpos[nout++] = (uint8_t)dg.lbits[t];
          } else {
            SU |= (uint8_t)(1u << upos_of[t]);
          }
        }
        int kU = __builtin_popcount(SU);
        po.mask = SU;
        po.dnu = (uint8_t)nout;
        po.code = SU;
        int dim = 1 << dg.k;
        if (gscale != cd(1.0)) {  // the deferred scalar rides on this diagonal
          for (cd& f : dg.f) f *= gscale;
          gscale = 1.0;
        }
        for (int nidx = 0; nidx < dim; nidx++) {
          int uval = nidx & ((1 << kU) - 1), oval = nidx >> kU, old = 0, c = 0;
          for (int q = 0; q < RB; q++)
            if ((SU >> q) & 1) {
              if ((uval >> c) & 1)
                for (int t = 0; t < dg.k; t++)
                  if (upos_of[t] == q) old |= 1 << t;
              c++;
            }
          for (int o2 = 0; o2 < nout; o2++)
            if ((oval >> o2) & 1) old |= 1 << outt[o2];
          push_coef(dg.f[old]);
        }
        plan.pops.push_back(po);
        dg = PDiag();
      };
      auto flush_kron = [&]() {
        if (!kron_any) return;
        PhaseOp po;
        std::memset(&po, 0, sizeof(po));
        po.cls = PO_KRON;
        po.k = 1;
        po.coef = (uint32_t)ncoef;
        po.mask = kron_mask;
        po.code = PCODE_KRON;
        for (int p = 0; p < RB; p++) {
          uint8_t f = form_of(kron[p], 1);
          const cd c0 = kron[p][0];
          if (defer && ((kron_mask >> p) & 1) && f == PD_XROT && c0 == kron[p][3] && c0.real() != 0.0 &&
              std::abs(kron[p][1]) <= std::abs(c0) && std::abs(kron[p][2]) <= std::abs(c0)) {
            f = PD_XROTU;
            push_coef(1.0);
            push_coef(kron[p][1] / c0);
            push_coef(kron[p][2] / c0);
            push_coef(1.0);
            gscale *= c0;
            saved += 2.0;
          } else {
            for (int e = 0; e < 4; e++) push_coef(kron[p][e]);
          }
          po.form |= (uint8_t)(f << (2 * p));
        }
        plan.pops.push_back(po);
        kron_any = false;
        kron_mask = 0;
        if (std::fabs(std::log2(std::abs(gscale))) > scalar_range) push_scalar();  // keep the state's scale in range
      };
      auto kron_reset = [&]() {
        for (int p = 0; p < 4; p++) {
          kron[p][0] = 1; kron[p][1] = 0; kron[p][2] = 0; kron[p][3] = 1;
        }
      };
      kron_reset();
      for (int oi : gr.second) {
        const BitOp& op = ops[oi];
        int dim = 1 << op.k;
        if (is_diagonal(op)) {
          flush_kron();
          kron_reset();
          // union of bits with the pending diagonal
          int ub[8], nub = dg.k;
          for (int t = 0; t < dg.k; t++) ub[t] = dg.lbits[t];
          for (int t = 0; t < op.k; t++) {
            int lb = local[op.bits[t]];
            bool have = false;
            for (int u = 0; u < nub; u++) have |= ub[u] == lb;
            if (!have) {
              if (nub == 8) {
                nub = 9;
                break;
              }
              ub[nub++] = lb;
            }
          }
          if (nub > 8) {
            flush_diag();
            nub = 0;
            for (int t = 0; t < op.k; t++) ub[nub++] = local[op.bits[t]];
          }
          PDiag nd;
          nd.k = nub;
          for (int u = 0; u < nub; u++) nd.lbits[u] = ub[u];
          nd.f.assign((size_t)1 << nub, cd(1.0));
          for (int idx = 0; idx < (1 << nub); idx++) {
            cd v = 1.0;
            if (dg.k) {  // pending factor
              int sub = 0;
              for (int t = 0; t < dg.k; t++)
                for (int u = 0; u < nub; u++)
                  if (ub[u] == dg.lbits[t] && ((idx >> u) & 1)) sub |= 1 << t;
              v *= dg.f[sub];
            }
            int sub = 0;
            for (int t = 0; t < op.k; t++)
              for (int u = 0; u < nub; u++)
                if (ub[u] == local[op.bits[t]] && ((idx >> u) & 1)) sub |= 1 << t;
            v *= op.m[(size_t)sub * dim + sub];
            nd.f[idx] = v;
          }
          dg = nd;
          continue;
        }
        flush_diag();
        if (op.k == 1) {  // one-bit dense or permutation: into the KRON group
          int p = rpos(local[op.bits[0]]);
          if ((kron_mask >> p) & 1) {
            flush_kron();
            kron_reset();
          }
          for (int e = 0; e < 4; e++) kron[p][e] = op.m[e];
          kron_mask |= (uint8_t)(1u << p);
          kron_any = true;
          continue;
        }
        flush_kron();
        kron_reset();
        // two-bit dense / permutation: operator bits in ascending register order
        PhaseOp po;
        std::memset(&po, 0, sizeof(po));
        po.k = (uint8_t)op.k;
        po.coef = (uint32_t)ncoef;
        int rp[4];
        for (int t = 0; t < op.k; t++) rp[t] = rpos(local[op.bits[t]]);
        int ord[4];
        for (int t = 0; t < op.k; t++) ord[t] = t;
        std::sort(ord, ord + op.k, [&](int a, int b) { return rp[a] < rp[b]; });
        uint8_t mask = 0;
        for (int t = 0; t < op.k; t++) mask |= (uint8_t)(1u << rp[t]);
        po.mask = mask;
        auto remap = [&](int inew) {
          int iold = 0;
          for (int t = 0; t < op.k; t++) iold |= ((inew >> t) & 1) << ord[t];
          return iold;
        };
        if (is_signed_perm(op)) {
          po.cls = PO_PERM;
          for (int i = 0; i < dim; i++)
            for (int j = 0; j < dim; j++) {
              cd v = op.m[(size_t)remap(i) * dim + remap(j)];
              if (v != cd(0.0)) po.perm[i] = (uint8_t)(j | (v.real() < 0 ? 0x80 : 0));
            }
          po.code = (uint8_t)(16 + mask);
        } else {
          po.cls = PO_DENSE;
          std::vector<cd> mm((size_t)dim * dim);
          for (int i = 0; i < dim; i++)
            for (int j = 0; j < dim; j++) mm[(size_t)i * dim + j] = op.m[(size_t)remap(i) * dim + remap(j)];
          po.form = form_of(mm.data(), op.k);
          for (auto& v : mm) push_coef(v);
          po.code = (uint8_t)(32 + 16 * po.form + mask);
        }
        plan.pops.push_back(po);
      }
      flush_diag();
      flush_kron();
      pd.nops = (uint32_t)plan.pops.size() - pd.op0;
      plan.phases.push_back(pd);
    }
    sd.nph = (uint32_t)plan.phases.size() - sd.ph0;
    sd.npop = (uint32_t)plan.pops.size() - sd.pop0;
    sd.npc = (uint32_t)ncoef - sd.pc0;
  }
  if (defer && gscale != cd(1.0)) {  // what no diagonal absorbed: onto the last phase of the plan
    for (size_t s = plan.sweeps.size(); s-- > 0;) {
      SweepDesc& sd = plan.sweeps[s];
      if (sd.nph == 0) continue;
      push_scalar();
      plan.phases.back().nops++;
      sd.npop++;
      sd.npc++;
      break;
    }
  }
  plan.fma_per_elem -= saved;
}

// ------------------------------------------------------------------ sweeps
void build_plan(std::vector<BitOp>& ops, const PlanOptions& opt, Plan& plan) {
  const bool cplx = plan.is_complex;
  if (opt.merge && !opt.plain) {
    merge_ops(ops, cplx, opt.max_merge_bits);
    // complex: a second pass joins diagonal operators that became adjacent
    if (cplx) merge_ops(ops, cplx, opt.max_merge_bits);
  }
  // per-qubit scale limit: FP64 storage 2^-40; FP32 storage and double-word
  // plans (float exponents) 2^-6, so 16 qubits stay below 2^96
  if (!cplx && opt.rescale_qubits > 0)
    rescale_dm(ops, opt.rescale_qubits, plan.dtype == NWQ_F64 && !plan.dw ? 0x1p-40 : 0x1p-6);

  const int B = plan.B;
  const int T = std::min(opt.tile_bits, B);
  const uint64_t full = B == 64 ? ~0ull : ((1ull << B) - 1);
  const uint64_t low = (1ull << std::min(opt.min_low, T)) - 1;

  size_t nops = ops.size();
  std::vector<char> done(nops, 0);
  std::vector<int> order;
  order.reserve(nops);
  plan.sweeps.clear();
  std::vector<uint64_t> sweep_tiles;
  size_t pos = 0;
  // With opt.commute (complex plans), a diagonal operator may move ahead of a
  // skipped diagonal operator (diagonal matrices commute): skipped diagonal
  // operators block only non-diagonal ones (blocked_nd), every other skipped
  // operator blocks everything on its bits (blocked).
  std::vector<char> diag(nops, 0);
  if (opt.commute && cplx)
    for (size_t i = 0; i < nops; i++) diag[i] = is_diagonal(ops[i]);
  while (pos < nops) {
    uint64_t R = low, blocked = 0, blocked_nd = 0;
    int first = (int)order.size();
    int scanned = 0;
    for (size_t i = pos; i < nops && scanned < opt.lookahead; i++) {
      if (done[i]) continue;
      scanned++;
      uint64_t m = op_mask(ops[i]);
      if ((m & blocked) || (!diag[i] && (m & blocked_nd))) {
        (diag[i] ? blocked_nd : blocked) |= m;
      } else if (__builtin_popcountll(R | m) <= T) {
        R |= m;
        done[i] = 1;
        order.push_back((int)i);
        if (opt.plain) break;
        if (opt.max_sweep_ops && (int)order.size() - first >= opt.max_sweep_ops) break;
      } else {
        (diag[i] ? blocked_nd : blocked) |= m;
      }
      if ((full & ~blocked) == 0) break;
    }
    while (pos < nops && done[pos]) pos++;
    // fill the tile with the lowest free bits (longer contiguous runs)
    for (int b = 0; b < B && __builtin_popcountll(R) < T; b++) R |= 1ull << b;
    SweepDesc sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.T = T;
    int m = 0;
    while (m < B && ((R >> m) & 1)) m++;
    sd.m = m;
    int h = 0;
    for (int b = m; b < B; b++)
      if ((R >> b) & 1) sd.hpos[h++] = (uint8_t)b;
    sd.h = h;
    sd.hmask = R & ~((1ull << m) - 1ull);
    sd.fmask = full & ~R;
    sd.nops = (int)order.size() - first;
    sd.op0 = (uint32_t)first;
    plan.sweeps.push_back(sd);
  }

  // device tables
  plan.ops.clear();
  plan.ents.clear();
  plan.op_gate0.clear();
  plan.op_ngates.clear();
  plan.fma_per_elem = 0;
  const size_t esz = plan.ent_bytes;
  const bool f64 = plan.dtype == NWQ_F64;
  size_t nent = 0;
  for (SweepDesc& sd : plan.sweeps) {
    int local[64];
    for (int b = 0; b < 64; b++) local[b] = -1;
    for (int b = 0; b < sd.m; b++) local[b] = b;
    for (int i = 0; i < sd.h; i++) local[sd.hpos[i]] = sd.m + i;
    const size_t sweep_ent0 = nent;
    for (int s = 0; s < sd.nops; s++) {
      const BitOp& op = ops[order[sd.op0 + s]];
      plan.fma_per_elem += op_cost(op, cplx);
      plan.op_gate0.push_back(op.gate0);
      plan.op_ngates.push_back(op.ngates);
      DevOp d;
      std::memset(&d, 0, sizeof(d));
      d.k = (uint8_t)op.k;
      for (int t = 0; t < op.k; t++) d.lb[t] = (uint8_t)local[op.bits[t]];
      for (int t = 0; t < op.k; t++) d.slb[t] = d.lb[t];
      std::sort(d.slb, d.slb + op.k);
      d.ent = (uint32_t)nent;
      int dim = 1 << op.k;
      uint32_t offs[16];
      for (int i = 0; i < dim; i++) {
        uint32_t o = 0;
        for (int t = 0; t < op.k; t++) o |= (uint32_t)((i >> t) & 1) << d.lb[t];
        offs[i] = o;
      }
      for (int i = 0; i < dim; i++) {
        RowMeta& rm = d.row[i];
        rm.out = (uint16_t)offs[i];
        std::vector<int> cols;
        for (int j = 0; j < dim; j++)
          if (op.m[(size_t)i * dim + j] != cd(0.0)) cols.push_back(j);
        if (cols.size() == 1 && cols[0] == i && op.m[(size_t)i * dim + i] == cd(1.0)) {
          rm.kind = ROW_ID;
          continue;
        }
        int bj = -1;
        for (int j : cols)
          if (is_unit(op.m[(size_t)i * dim + j])) {
            bj = j;
            break;
          }
        if (bj >= 0) {
          rm.base = op.m[(size_t)i * dim + bj].real() > 0 ? 1 : 2;
          rm.boff = (uint16_t)offs[bj];
        }
        std::vector<int> rest;
        for (int j : cols)
          if (j != bj) rest.push_back(j);
        rm.kind = (rest.empty() && bj >= 0) ? ROW_MOVE : ROW_GEN;
        rm.beg = (uint16_t)(nent - d.ent);
        auto ckind = [&](int j) {
          cd v = op.m[(size_t)i * dim + j];
          return v.imag() == 0.0 ? CE_RE : (v.real() == 0.0 ? CE_IM : CE_GEN);
        };
        if (cplx) std::stable_sort(rest.begin(), rest.end(), [&](int a, int b) { return ckind(a) < ckind(b); });
        for (int j : rest) {
          cd v = op.m[(size_t)i * dim + j];
          unsigned char rec[32];
          std::memset(rec, 0, sizeof(rec));
          if (!cplx) {
            rm.cnt[0]++;
            if (f64) {
              EntR<double> e{v.real(), offs[j]};
              std::memcpy(rec, &e, sizeof(e));
            } else {
              EntR<float> e{(float)v.real(), offs[j]};
              std::memcpy(rec, &e, sizeof(e));
            }
          } else {
            uint32_t kind = ckind(j);
            rm.cnt[kind]++;
            if (f64) {
              EntC<double> e{v.real(), v.imag(), offs[j], kind};
              std::memcpy(rec, &e, sizeof(e));
            } else {
              EntC<float> e{(float)v.real(), (float)v.imag(), offs[j], kind};
              std::memcpy(rec, &e, sizeof(e));
            }
          }
          plan.ents.insert(plan.ents.end(), rec, rec + esz);
          nent++;
        }
      }
      plan.ops.push_back(d);
    }
    sd.ent0 = (uint32_t)sweep_ent0;
    sd.nent = (uint32_t)(nent - sweep_ent0);
  }
  if (cplx) build_phases(ops, order, plan, opt.register_bits);
  double state_bytes = (double)plan.elem_bytes * (double)(1ull << B);
  plan.bytes = 2.0 * state_bytes * (double)plan.sweeps.size();
  // the operators in execution order, moved (not copied): the caller's list is spent
  plan.exec_ops.clear();
  plan.exec_ops.reserve(order.size());
  for (int i : order) plan.exec_ops.push_back(std::move(ops[i]));
}

}  // namespace nwq
