/*
 * nwq_oracle.c -- plain, slow FP64 reference simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  It is called by the tests, by the smoke check
 * and by the CPU-baseline leg of the benchmark; the product path never links
 * or calls it.  It shares no code, header, table or constant with the CUDA
 * library: gate matrices, noise channels and reductions are re-derived here
 * from their textbook definitions.
 *
 * What it computes (paper Sec. II and Sec. III; the paper prints no formulas,
 * so each definition below is the standard one and the readings of the
 * conventions are listed in the design notes):
 *   - state-vector simulation: psi <- U psi, gate after gate (SV-Sim, Sec. II)
 *   - density-matrix simulation: rho <- U rho U^dag, and noise channels in
 *     Kraus form rho <- sum_k K_k rho K_k^dag (DM-Sim, Sec. II), with the
 *     device noise model of Sec. III: depolarising after every gate, then
 *     thermal relaxation, and measurement (readout) noise on the outcome
 *     distribution.
 *   - expectation values <P> = <psi|P|psi> and Tr(rho P) of Pauli strings.
 *
 * Conventions: qubit q is bit q of the basis index.  A two-qubit matrix acts
 * in the local basis j = b(q0) + 2 b(q1).  rho is stored row-major:
 * rho[r * N + c] = <r|rho|c>.  Pauli string (x, z) means
 * i^{|x & z|} X^x Z^z (Z applied first), which is Hermitian.
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cx;

/* Gate kinds understood by the oracle (numbering private to this file and
 * its Python loader). */
enum {
  OG_ID = 0, OG_X, OG_Y, OG_Z, OG_H, OG_S, OG_SDG, OG_T, OG_TDG, OG_SX,
  OG_RX, OG_RY, OG_RZ, OG_P, OG_U3, OG_MAT1,
  OG_CX = 32, OG_CZ, OG_SWAP, OG_RZZ, OG_MAT2
};

static int is_two_qubit(int kind) { return kind >= 32; }

/* ------------------------------------------------------------------ matrices
 * One-qubit matrices written from the Pauli matrices:
 *   rotations R_P(theta) = exp(-i theta P / 2) = cos(theta/2) I - i sin(theta/2) P
 *   P(lambda) = diag(1, e^{i lambda});  S = P(pi/2);  T = P(pi/4)
 *   H = (X + Z)/sqrt(2);  SX = sqrt(X) = ((1+i) I + (1-i) X)/2
 *   U3(t, p, l) = [[cos(t/2), -e^{il} sin(t/2)], [e^{ip} sin(t/2), e^{i(p+l)} cos(t/2)]]
 */
static const cx PI_[4] = {1, 0, 0, 1};
static const cx PX_[4] = {0, 1, 1, 0};
static const cx PY_[4] = {0, -I, I, 0};
static const cx PZ_[4] = {1, 0, 0, -1};

static void lin2(cx out[4], cx a, const cx A[4], cx b, const cx B[4]) {
  for (int k = 0; k < 4; k++) out[k] = a * A[k] + b * B[k];
}

static void diag2(cx out[4], cx d0, cx d1) {
  out[0] = d0; out[1] = 0; out[2] = 0; out[3] = d1;
}

/* Fill U (row-major, dim 2 or 4).  Returns the number of qubits (1 or 2). */
static int gate_matrix(int kind, const double *th, const double *mat, cx *U) {
  double c, s;
  switch (kind) {
    case OG_ID: lin2(U, 1, PI_, 0, PI_); return 1;
    case OG_X: lin2(U, 1, PX_, 0, PI_); return 1;
    case OG_Y: lin2(U, 1, PY_, 0, PI_); return 1;
    case OG_Z: lin2(U, 1, PZ_, 0, PI_); return 1;
    case OG_H: lin2(U, 1 / sqrt(2.0), PX_, 1 / sqrt(2.0), PZ_); return 1;
    case OG_S: diag2(U, 1, cexp(I * M_PI / 2)); return 1;
    case OG_SDG: diag2(U, 1, cexp(-I * M_PI / 2)); return 1;
    case OG_T: diag2(U, 1, cexp(I * M_PI / 4)); return 1;
    case OG_TDG: diag2(U, 1, cexp(-I * M_PI / 4)); return 1;
    case OG_SX: lin2(U, (1 + I) / 2, PI_, (1 - I) / 2, PX_); return 1;
    case OG_RX: c = cos(th[0] / 2); s = sin(th[0] / 2); lin2(U, c, PI_, -I * s, PX_); return 1;
    case OG_RY: c = cos(th[0] / 2); s = sin(th[0] / 2); lin2(U, c, PI_, -I * s, PY_); return 1;
    case OG_RZ: c = cos(th[0] / 2); s = sin(th[0] / 2); lin2(U, c, PI_, -I * s, PZ_); return 1;
    case OG_P: diag2(U, 1, cexp(I * th[0])); return 1;
    case OG_U3:
      c = cos(th[0] / 2); s = sin(th[0] / 2);
      U[0] = c; U[1] = -cexp(I * th[2]) * s;
      U[2] = cexp(I * th[1]) * s; U[3] = cexp(I * (th[1] + th[2])) * c;
      return 1;
    case OG_MAT1:
      for (int k = 0; k < 4; k++) U[k] = mat[2 * k] + I * mat[2 * k + 1];
      return 1;
    case OG_CX: /* flips q1 when q0 = 1: |j=1> <-> |j=3> */
      memset(U, 0, 16 * sizeof(cx));
      U[0 * 4 + 0] = 1; U[2 * 4 + 2] = 1; U[3 * 4 + 1] = 1; U[1 * 4 + 3] = 1;
      return 2;
    case OG_CZ:
      memset(U, 0, 16 * sizeof(cx));
      U[0] = 1; U[5] = 1; U[10] = 1; U[15] = -1;
      return 2;
    case OG_SWAP:
      memset(U, 0, 16 * sizeof(cx));
      U[0] = 1; U[2 * 4 + 1] = 1; U[1 * 4 + 2] = 1; U[15] = 1;
      return 2;
    case OG_RZZ: { /* cos(t/2) I(x)I - i sin(t/2) Z(x)Z, built as a Kronecker product */
      c = cos(th[0] / 2); s = sin(th[0] / 2);
      for (int r = 0; r < 4; r++)
        for (int k = 0; k < 4; k++) {
          /* (A (x) B)[r][k] with A on q1 (high local bit), B on q0 (low local bit) */
          int r0 = r & 1, r1 = r >> 1, k0 = k & 1, k1 = k >> 1;
          cx ii = PI_[r1 * 2 + k1] * PI_[r0 * 2 + k0];
          cx zz = PZ_[r1 * 2 + k1] * PZ_[r0 * 2 + k0];
          U[r * 4 + k] = c * ii - I * s * zz;
        }
      return 2;
    }
    case OG_MAT2:
      for (int k = 0; k < 16; k++) U[k] = mat[2 * k] + I * mat[2 * k + 1];
      return 2;
  }
  return 0;
}

int oracle_gate_matrix(int kind, const double *th, const double *mat, double *out_reim) {
  cx U[16];
  int nq = gate_matrix(kind, th, mat, U);
  int d = nq == 2 ? 16 : 4;
  for (int k = 0; k < d; k++) { out_reim[2 * k] = creal(U[k]); out_reim[2 * k + 1] = cimag(U[k]); }
  return nq;
}

/* ------------------------------------------------------------------ vector action
 * Apply a k-qubit matrix (k = 1, 2) to a vector of N = 2^n entries with the
 * given stride: v[base + stride * idx].  Used on the state vector (stride 1)
 * and on the rows / columns of a density matrix. */
static void apply_vec(cx *v, int n, size_t stride, int k, const int *q, const cx *U) {
  size_t N = (size_t)1 << n;
  size_t m0 = (size_t)1 << q[0];
  size_t m1 = k == 2 ? ((size_t)1 << q[1]) : 0;
  int d = 1 << k;
  for (size_t b = 0; b < N; b++) {
    if (b & (m0 | m1)) continue;
    size_t idx[4];
    cx in[4], out[4];
    for (int j = 0; j < d; j++) {
      idx[j] = b | ((j & 1) ? m0 : 0) | ((j & 2) ? m1 : 0);
      in[j] = v[idx[j] * stride];
    }
    for (int r = 0; r < d; r++) {
      cx acc = 0;
      for (int j = 0; j < d; j++) acc += U[r * d + j] * in[j];
      out[r] = acc;
    }
    for (int j = 0; j < d; j++) v[idx[j] * stride] = out[j];
  }
}

/* The same action on a state vector (stride 1), amplitude groups split over
 * OpenMP threads (independent: each group's indices are disjoint). */
static void apply_vec_par(cx *v, int n, int k, const int *q, const cx *U) {
  size_t N = (size_t)1 << n;
  size_t m0 = (size_t)1 << q[0];
  size_t m1 = k == 2 ? ((size_t)1 << q[1]) : 0;
  int d = 1 << k;
#pragma omp parallel for schedule(static) if (n >= 16)
  for (long bb = 0; bb < (long)N; bb++) {
    size_t b = (size_t)bb;
    if (b & (m0 | m1)) continue;
    size_t idx[4];
    cx in[4], out[4];
    for (int j = 0; j < d; j++) {
      idx[j] = b | ((j & 1) ? m0 : 0) | ((j & 2) ? m1 : 0);
      in[j] = v[idx[j]];
    }
    for (int r = 0; r < d; r++) {
      cx acc = 0;
      for (int j = 0; j < d; j++) acc += U[r * d + j] * in[j];
      out[r] = acc;
    }
    for (int j = 0; j < d; j++) v[idx[j]] = out[j];
  }
}

/* Thread count of the OpenMP loops (benchmark baselines time 1 and all). */
void oracle_set_threads(int t) { omp_set_num_threads(t > 0 ? t : 1); }
int oracle_max_threads(void) { return omp_get_max_threads(); }

/* psi <- U psi */
void oracle_sv_apply(double *psi_reim, int n, int k, const int *q, const double *U_reim) {
  cx U[16];
  for (int j = 0; j < (1 << (2 * k)); j++) U[j] = U_reim[2 * j] + I * U_reim[2 * j + 1];
  apply_vec((cx *)psi_reim, n, 1, k, q, U);
}

/* Apply a whole circuit to psi (in place). kinds[g], qs[2g..2g+1], th[3g..3g+2],
 * mats[32g..] (re/im interleaved 4x4 or 2x2, used by MAT1/MAT2 only). */
int oracle_sv_run(double *psi_reim, int n, int ng, const int *kinds, const int *qs,
                  const double *th, const double *mats) {
  cx *psi = (cx *)psi_reim;
  for (int g = 0; g < ng; g++) {
    cx U[16];
    int k = gate_matrix(kinds[g], th + 3 * g, mats + 32 * g, U);
    if (!k) return -1;
    apply_vec_par(psi, n, k, qs + 2 * g, U);
  }
  return 0;
}

/* ------------------------------------------------------------------ density matrix
 * rho <- A rho        : A acts on the row index  (each column is a vector)
 * rho <- rho A^dag    : conj(A) acts on the column index (each row is a vector)
 */
static void left_mul(cx *rho, int n, int k, const int *q, const cx *A) {
  size_t N = (size_t)1 << n;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < (long)N; c++) apply_vec(rho + c, n, N, k, q, A);
}

static void right_mul_dag(cx *rho, int n, int k, const int *q, const cx *A) {
  size_t N = (size_t)1 << n;
  int d = 1 << k;
  cx Ac[16];
  for (int j = 0; j < d * d; j++) Ac[j] = conj(A[j]);
#pragma omp parallel for schedule(static)
  for (long r = 0; r < (long)N; r++) apply_vec(rho + (size_t)r * N, n, 1, k, q, Ac);
}

static void dm_unitary(cx *rho, int n, int k, const int *q, const cx *U) {
  left_mul(rho, n, k, q, U);
  right_mul_dag(rho, n, k, q, U);
}

/* rho <- sum_j K_j rho K_j^dag */
static void dm_kraus(cx *rho, int n, int k, const int *q, int nk, const cx *K) {
  size_t N = (size_t)1 << n, NN = N * N;
  int dd = 1 << (2 * k);
  cx *acc = calloc(NN, sizeof(cx));
  cx *tmp = malloc(NN * sizeof(cx));
  for (int j = 0; j < nk; j++) {
    memcpy(tmp, rho, NN * sizeof(cx));
    left_mul(tmp, n, k, q, K + j * dd);
    right_mul_dag(tmp, n, k, q, K + j * dd);
#pragma omp parallel for schedule(static)
    for (long e = 0; e < (long)NN; e++) acc[e] += tmp[e];
  }
  memcpy(rho, acc, NN * sizeof(cx));
  free(acc);
  free(tmp);
}

/* Depolarising channel on k qubits (k = 1, 2) in the "depolarising
 * parameter" form  E(rho) = (1 - p) rho + p Tr_S(rho) (x) I / 2^k,
 * written as Kraus operators: sqrt(1 - (4^k - 1) p / 4^k) on the identity
 * string and sqrt(p / 4^k) on each of the other 4^k - 1 Pauli strings
 * (the Pauli twirl identity sum_P P rho P = 2^k Tr_S(rho) (x) I). */
static void dm_depolarize(cx *rho, int n, int k, const int *q, double p) {
  const cx *P1[4] = {PI_, PX_, PY_, PZ_};
  int np = 1 << (2 * k), d = 1 << k;
  cx *K = malloc((size_t)np * d * d * sizeof(cx));
  for (int s = 0; s < np; s++) {
    double w = s == 0 ? sqrt(1.0 - (np - 1) * p / np) : sqrt(p / np);
    if (k == 1) {
      for (int e = 0; e < 4; e++) K[s * 4 + e] = w * P1[s][e];
    } else {
      const cx *A = P1[s & 3];  /* on q0 (low local bit) */
      const cx *B = P1[s >> 2]; /* on q1 (high local bit) */
      for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++)
          K[s * 16 + r * 4 + c] = w * B[(r >> 1) * 2 + (c >> 1)] * A[(r & 1) * 2 + (c & 1)];
    }
  }
  dm_kraus(rho, n, k, q, np, K);
  free(K);
}

/* Thermal relaxation toward |0> for a duration t: amplitude damping with
 * gamma = 1 - exp(-t/T1) followed by pure dephasing chosen so that the total
 * coherence factor is eta = exp(-t/T2):  sqrt(1-gamma) sqrt(1-lambda) = eta.
 * Valid (CPTP in this split form) when T2 <= 2 T1.  Returns -1 otherwise. */
static int dm_relax(cx *rho, int n, int q, double t_ns, double T1_us, double T2_us) {
  double gamma = 1.0 - exp(-t_ns / (T1_us * 1e3));
  double eta = exp(-t_ns / (T2_us * 1e3));
  double one_minus_lambda = eta * eta / (1.0 - gamma);
  if (one_minus_lambda > 1.0 + 1e-15) return -1;
  if (one_minus_lambda > 1.0) one_minus_lambda = 1.0;
  cx AD[8] = {1, 0, 0, sqrt(1.0 - gamma), /* K0 */ 0, sqrt(gamma), 0, 0 /* K1 */};
  cx PD[8] = {1, 0, 0, sqrt(one_minus_lambda), 0, 0, 0, sqrt(1.0 - one_minus_lambda)};
  dm_kraus(rho, n, 1, &q, 2, AD);
  dm_kraus(rho, n, 1, &q, 2, PD);
  return 0;
}

/* The same relaxation written as its direct action on each 2x2 block of
 * qubit q: rho00 += gamma rho11, rho11 *= (1 - gamma), rho01, rho10 *= eta.
 * Valid for any T1, T2 > 0 (no Kraus split needed). */
void oracle_dm_relax_direct(double *rho_reim, int n, int q, double t_ns, double T1_us, double T2_us) {
  cx *rho = (cx *)rho_reim;
  size_t N = (size_t)1 << n, m = (size_t)1 << q;
  double gamma = 1.0 - exp(-t_ns / (T1_us * 1e3));
  double eta = exp(-t_ns / (T2_us * 1e3));
  for (size_t r = 0; r < N; r++) {
    if (r & m) continue;
    for (size_t c = 0; c < N; c++) {
      if (c & m) continue;
      cx *a = &rho[r * N + c], *b = &rho[r * N + (c | m)];
      cx *d = &rho[(r | m) * N + c], *e = &rho[(r | m) * N + (c | m)];
      *a += gamma * *e;
      *e *= (1.0 - gamma);
      *b *= eta;
      *d *= eta;
    }
  }
}

int oracle_dm_relax_kraus(double *rho_reim, int n, int q, double t_ns, double T1_us, double T2_us) {
  return dm_relax((cx *)rho_reim, n, q, t_ns, T1_us, T2_us);
}

void oracle_dm_depolarize(double *rho_reim, int n, int k, const int *q, double p) {
  dm_depolarize((cx *)rho_reim, n, k, q, p);
}

void oracle_dm_unitary(double *rho_reim, int n, int k, const int *q, const double *U_reim) {
  cx U[16];
  for (int j = 0; j < (1 << (2 * k)); j++) U[j] = U_reim[2 * j] + I * U_reim[2 * j + 1];
  dm_unitary((cx *)rho_reim, n, k, q, U);
}

/* Noisy circuit on rho (in place).  Noise model (Sec. III): after every gate,
 * depolarising on the gate's qubits (p1 for one-qubit gates, p2 for two-qubit
 * gates), then thermal relaxation on each of the gate's qubits for the gate's
 * duration (t1q_ns / t2q_ns).  flags bit 0: RZ is virtual (noise-free, 0 ns).
 * flags bit 1: depolarising probability given in the Pauli form (p spread
 * as p/(4^k-1) on each non-identity Pauli), converted here to the
 * depolarising parameter p_dep = p 4^k / (4^k - 1).
 * With nm == 0 (noise off) it is a plain unitary simulation. */
int oracle_dm_run(double *rho_reim, int n, int ng, const int *kinds, const int *qs,
                  const double *th, const double *mats, int noisy, const double *T1_us,
                  const double *T2_us, double t1q_ns, double t2q_ns, double p1, double p2,
                  unsigned flags) {
  cx *rho = (cx *)rho_reim;
  for (int g = 0; g < ng; g++) {
    cx U[16];
    int k = gate_matrix(kinds[g], th + 3 * g, mats + 32 * g, U);
    if (!k) return -1;
    const int *q = qs + 2 * g;
    dm_unitary(rho, n, k, q, U);
    if (!noisy) continue;
    if ((flags & 1u) && kinds[g] == OG_RZ) continue;
    double p = k == 2 ? p2 : p1;
    if (flags & 2u) p = p * (1 << (2 * k)) / ((1 << (2 * k)) - 1.0);
    if (p > 0) dm_depolarize(rho, n, k, q, p);
    double t = k == 2 ? t2q_ns : t1q_ns;
    if (t > 0)
      for (int j = 0; j < k; j++)
        if (dm_relax(rho, n, q[j], t, T1_us[q[j]], T2_us[q[j]])) return -2;
  }
  return 0;
}

/* ------------------------------------------------------------------ quantum trajectories
 * One trajectory of the Monte-Carlo unravelling of the same noise model on a
 * state vector (its average over trajectories is the density matrix of
 * oracle_dm_run).  The random draws are inputs: u[] holds uniforms in [0, 1),
 * consumed in this order, gate by gate, after the gate is applied:
 *   - depolarising with parameter p on the gate's k qubits (if p > 0), one
 *     draw: each of the 4^k - 1 non-identity Pauli strings has probability
 *     p / 4^k; string s = 1 + floor(u 4^k / p) (at most 4^k - 1) is applied
 *     when u < (4^k - 1) p / 4^k, else none.  s & 3 is the Pauli on q0 and
 *     s >> 2 the Pauli on q1 (0 I, 1 X, 2 Y, 3 Z).
 *   - thermal relaxation on each gate qubit q (if t > 0), two draws: amplitude
 *     damping (gamma) then phase damping (lambda, with sqrt(1-gamma)
 *     sqrt(1-lambda) = eta).  With P1 = the probability of q = 1 in the
 *     current state, the jump operator (|0><1| resp. |1><1|) is applied when
 *     u < gamma P1 (resp. lambda P1), else diag(1, sqrt(1 - gamma)) (resp.
 *     sqrt(1 - lambda)); the state is then renormalised (its norm after the
 *     Kraus operator is the probability of the branch taken).
 * Returns the number of draws consumed, -1 for an unknown gate, -2 when T2 >
 * 2 T1, -3 when more than nu draws would be needed.
 * margin and kind (may be NULL) receive, per draw consumed, how far the draw
 * lay from the nearest value at which its outcome changes, relative to the
 * branch width: depolarising (kind 0): min_j |u - j p/4^k| / (p/4^k) over the
 * sub-interval ends j = 1 .. 4^k - 1; amplitude damping (kind 1) and phase
 * damping (kind 2): |u - rate P1| / (rate P1) (+inf when rate P1 = 0). */
static double prob_one(const cx *psi, int n, int q) {
  size_t N = (size_t)1 << n, m = (size_t)1 << q;
  double s = 0.0;
  for (size_t b = 0; b < N; b++)
    if (b & m) s += creal(psi[b]) * creal(psi[b]) + cimag(psi[b]) * cimag(psi[b]);
  return s;
}

static void scale_vec(cx *psi, int n, double f) {
  size_t N = (size_t)1 << n;
  for (size_t b = 0; b < N; b++) psi[b] *= f;
}

int oracle_traj_run(double *psi_reim, int n, int ng, const int *kinds, const int *qs, const double *th,
                    const double *mats, int noisy, const double *T1_us, const double *T2_us, double t1q_ns,
                    double t2q_ns, double p1, double p2, unsigned flags, const double *u, int nu,
                    double *margin, int *kind) {
  const cx *P1[4] = {PI_, PX_, PY_, PZ_};
  cx *psi = (cx *)psi_reim;
  int used = 0;
  for (int g = 0; g < ng; g++) {
    cx U[16];
    int k = gate_matrix(kinds[g], th + 3 * g, mats + 32 * g, U);
    if (!k) return -1;
    const int *q = qs + 2 * g;
    apply_vec(psi, n, 1, k, q, U);
    if (!noisy) continue;
    if ((flags & 1u) && kinds[g] == OG_RZ) continue;
    int np = 1 << (2 * k);
    double p = k == 2 ? p2 : p1;
    if (flags & 2u) p = p * np / (np - 1.0);
    if (p > 0) {
      if (used >= nu) return -3;
      double x = u[used];
      if (margin) {
        double w = p / np, best = INFINITY;
        for (int j = 1; j < np; j++) best = fmin(best, fabs(x - j * w) / w);
        margin[used] = best;
      }
      if (kind) kind[used] = 0;
      used++;
      if (x < (np - 1) * p / np) {
        int s = 1 + (int)floor(x * np / p);
        if (s > np - 1) s = np - 1;
        for (int w = 0; w < k; w++) {
          int a = (s >> (2 * w)) & 3;
          if (a) apply_vec(psi, n, 1, 1, q + w, P1[a]);
        }
      }
    }
    double t = k == 2 ? t2q_ns : t1q_ns;
    if (t > 0)
      for (int w = 0; w < k; w++) {
        int qq = q[w];
        double gamma = 1.0 - exp(-t / (T1_us[qq] * 1e3));
        double eta = exp(-t / (T2_us[qq] * 1e3));
        double oml = eta * eta / (1.0 - gamma);
        if (oml > 1.0 + 1e-15) return -2;
        if (oml > 1.0) oml = 1.0;
        double rate[2] = {gamma, 1.0 - oml};
        for (int step = 0; step < 2; step++) {  /* amplitude damping, then phase damping */
          if (used >= nu) return -3;
          double x = u[used];
          double pr1 = prob_one(psi, n, qq);
          if (margin) {
            double thr = rate[step] * pr1;
            margin[used] = thr > 0 ? fabs(x - thr) / thr : INFINITY;
          }
          if (kind) kind[used] = 1 + step;
          used++;
          size_t N = (size_t)1 << n, m = (size_t)1 << qq;
          if (x < rate[step] * pr1) {
            for (size_t b = 0; b < N; b++) {
              if (b & m) continue;
              psi[b] = step == 0 ? psi[b | m] : 0.0;  /* |0><1| moves the |1> part down; |1><1| keeps it */
              if (step == 0) psi[b | m] = 0.0;
            }
            scale_vec(psi, n, 1.0 / sqrt(pr1));
          } else {
            double f = sqrt(1.0 - rate[step]);
            for (size_t b = 0; b < N; b++)
              if (b & m) psi[b] *= f;
            scale_vec(psi, n, 1.0 / sqrt(1.0 - rate[step] * pr1));
          }
        }
      }
  }
  return used;
}

/* Draws one trajectory of oracle_traj_run consumes (independent of them). */
int oracle_traj_draws(int ng, const int *kinds, int noisy, double t1q_ns, double t2q_ns, double p1, double p2,
                      unsigned flags) {
  int c = 0;
  for (int g = 0; g < ng; g++) {
    if (!noisy || ((flags & 1u) && kinds[g] == OG_RZ)) continue;
    int k = is_two_qubit(kinds[g]) ? 2 : 1;
    if ((k == 2 ? p2 : p1) > 0) c += 1;
    if ((k == 2 ? t2q_ns : t1q_ns) > 0) c += 2 * k;
  }
  return c;
}

/* ------------------------------------------------------------------ Pauli strings
 * P(x, z) |b> = i^{|x&z|} (-1)^{|b&z|} |b ^ x>. */
static cx pauli_phase(uint64_t x, uint64_t z, uint64_t b) {
  int y = __builtin_popcountll(x & z) & 3;
  static const cx ipow[4] = {1, I, -1, -I};
  cx ph = ipow[y];
  return (__builtin_popcountll(b & z) & 1) ? -ph : ph;
}

/* <psi| P |psi> for each term (real part; P is Hermitian). */
void oracle_sv_expect(const double *psi_reim, int n, int nt, const uint64_t *xm, const uint64_t *zm,
                      double *out) {
  const cx *psi = (const cx *)psi_reim;
  size_t N = (size_t)1 << n;
  for (int t = 0; t < nt; t++) {
    cx acc = 0;
    for (size_t b = 0; b < N; b++) acc += conj(psi[b ^ xm[t]]) * pauli_phase(xm[t], zm[t], b) * psi[b];
    out[t] = creal(acc);
  }
}

/* Tr(rho P) = sum_r <r|rho|r^x> <r^x|P|r>. */
void oracle_dm_expect(const double *rho_reim, int n, int nt, const uint64_t *xm, const uint64_t *zm,
                      double *out) {
  const cx *rho = (const cx *)rho_reim;
  size_t N = (size_t)1 << n;
  for (int t = 0; t < nt; t++) {
    cx acc = 0;
    for (size_t r = 0; r < N; r++) acc += rho[r * N + (r ^ xm[t])] * pauli_phase(xm[t], zm[t], r);
    out[t] = creal(acc);
  }
}

/* Outcome distribution with symmetric readout error e on every bit:
 * p'(b) = sum_{b'} prod_i C(b_i | b'_i) p(b'), C = [[1-e, e], [e, 1-e]],
 * applied one bit at a time. */
static void readout(double *p, int n, double e) {
  size_t N = (size_t)1 << n;
  for (int i = 0; i < n; i++) {
    size_t m = (size_t)1 << i;
    for (size_t b = 0; b < N; b++) {
      if (b & m) continue;
      double a0 = p[b], a1 = p[b | m];
      p[b] = (1 - e) * a0 + e * a1;
      p[b | m] = e * a0 + (1 - e) * a1;
    }
  }
}

void oracle_sv_probs(const double *psi_reim, int n, double e, double *out) {
  const cx *psi = (const cx *)psi_reim;
  size_t N = (size_t)1 << n;
  for (size_t b = 0; b < N; b++) out[b] = creal(psi[b]) * creal(psi[b]) + cimag(psi[b]) * cimag(psi[b]);
  if (e > 0) readout(out, n, e);
}

void oracle_dm_probs(const double *rho_reim, int n, double e, double *out) {
  const cx *rho = (const cx *)rho_reim;
  size_t N = (size_t)1 << n;
  for (size_t b = 0; b < N; b++) out[b] = creal(rho[b * N + b]);
  if (e > 0) readout(out, n, e);
}
