// Batched evaluation of parametrised circuits (the VQE inner loop of paper
// Sec. III): one CTA per job (one parameter set of one circuit template),
// the whole 2^n state resident in shared memory, gates applied in place,
// Pauli-term expectations reduced with FP64 accuracy (FP64 arithmetic, or
// exact products and compensated float-pair sums, added across the CTA in
// FP64), energies written per job.
// Jobs are taken from an atomic work queue (a persistent grid), so templates
// of different qubit counts and depths balance across SMs in one launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <type_traits>

#include "batch.hpp"
#include "dw.cuh"
#include "kernels.hpp"

namespace nwq {

template <class R>
struct C2;
template <>
struct C2<double> {
  using T = double2;
};
template <>
struct C2<float> {
  using T = float2;
};

// Per-job gate matrix: 2x2 complex (or the 4 diagonal phases of a 2q
// diagonal) with its structure class.
template <class R>
struct GateMat {
  typename C2<R>::T m[4];
  int cls;  // BG_* class below
};

enum : int { BG_DENSE = 0, BG_REAL = 1, BG_DIAG = 2, BG_CX = 3, BG_CZ = 4, BG_SWAP = 5, BG_DIAG2 = 6 };

// One-qubit gate g as a full 2x2 matrix in FP64 (FP64 trigonometry) with its
// structure class.
__device__ void gate1_d(const BGate& g, const double* __restrict__ p, double2 (&m)[4], int& cls) {
  if (g.type == BT_FIXED1) {
    for (int k = 0; k < 4; k++) m[k] = make_double2(g.m[2 * k], g.m[2 * k + 1]);
    cls = g.cls;
    return;
  }
  const double th = g.pidx >= 0 ? p[g.pidx] : g.th[0];
  double s, c;
  sincos(0.5 * th, &s, &c);
  m[1] = m[2] = make_double2(0.0, 0.0);
  switch (g.type) {
    case BT_RX:
      m[0] = make_double2(c, 0); m[1] = make_double2(0, -s); m[2] = make_double2(0, -s); m[3] = make_double2(c, 0);
      cls = BG_DENSE;
      break;
    case BT_RY:
      m[0] = make_double2(c, 0); m[1] = make_double2(-s, 0); m[2] = make_double2(s, 0); m[3] = make_double2(c, 0);
      cls = BG_REAL;
      break;
    case BT_RZ:  // diag(e^{-i th/2}, e^{i th/2})
      m[0] = make_double2(c, -s); m[3] = make_double2(c, s);
      cls = BG_DIAG;
      break;
    case BT_P: {  // diag(1, e^{i th})
      double s2, c2;
      sincos(th, &s2, &c2);
      m[0] = make_double2(1, 0); m[3] = make_double2(c2, s2);
      cls = BG_DIAG;
      break;
    }
    default: {  // BT_U3
      double sp, cp, sl, cl, spl, cpl;
      sincos(g.th[1], &sp, &cp);
      sincos(g.th[2], &sl, &cl);
      sincos(g.th[1] + g.th[2], &spl, &cpl);
      m[0] = make_double2(c, 0);
      m[1] = make_double2(-cl * s, -sl * s);
      m[2] = make_double2(cp * s, sp * s);
      m[3] = make_double2(cpl * c, spl * c);
      cls = BG_DENSE;
    }
  }
}

// Matrix of gate g for parameter vector p (FP64 trigonometry and, for fused
// runs, FP64 products; stored in R).
template <class R>
__device__ void make_gate(const BGate& g, const BGate* __restrict__ all, const double* __restrict__ p,
                          GateMat<R>& out) {
  using C = typename C2<R>::T;
  if (g.type == BT_CX) { out.cls = BG_CX; return; }
  if (g.type == BT_CZ) { out.cls = BG_CZ; return; }
  if (g.type == BT_SWAP) { out.cls = BG_SWAP; return; }
  if (g.type == BT_RZZ) {  // phases e^{-i th/2} on even parity, e^{+i th/2} on odd
    const double th = g.pidx >= 0 ? p[g.pidx] : g.th[0];
    double s, c;
    sincos(0.5 * th, &s, &c);
    out.m[0] = C{(R)c, (R)-s}; out.m[1] = C{(R)c, (R)s};
    out.cls = BG_DIAG2;
    return;
  }
  double2 m[4];
  int cls;
  if (g.type == BT_FUSED) {  // M = G_last ... G_first
    gate1_d(all[g.pidx], p, m, cls);
    bool diag = cls == BG_DIAG, real = cls == BG_REAL;
    for (int k = 1; k < g.cls; k++) {
      double2 a[4];
      int ca;
      gate1_d(all[g.pidx + k], p, a, ca);
      diag &= ca == BG_DIAG;
      real &= ca == BG_REAL;
      double2 r[4];
      for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
          const double2 x = a[2 * i], y = m[j], u = a[2 * i + 1], v = m[2 + j];
          r[2 * i + j] = make_double2(fma(x.x, y.x, fma(-x.y, y.y, fma(u.x, v.x, -u.y * v.y))),
                                      fma(x.x, y.y, fma(x.y, y.x, fma(u.x, v.y, u.y * v.x))));
        }
      for (int e = 0; e < 4; e++) m[e] = r[e];
    }
    cls = diag ? BG_DIAG : (real ? BG_REAL : BG_DENSE);
  } else {
    gate1_d(g, p, m, cls);
  }
  for (int k = 0; k < 4; k++) out.m[k] = C{(R)m[k].x, (R)m[k].y};
  out.cls = cls;
}

template <class C, class R>
__device__ __forceinline__ C cmul(C a, C b) {
  return C{fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)};
}

template <class R>
__device__ void apply_gate(typename C2<R>::T* __restrict__ psi, int n, const BGate& g, const GateMat<R>& G) {
  using C = typename C2<R>::T;
  const uint32_t half = 1u << (n - 1);
  const uint32_t q0 = g.q0, q1 = g.q1;
  const uint32_t m0 = 1u << q0, m1 = 1u << q1;
  switch (G.cls) {
    case BG_CX:
    case BG_CZ:
    case BG_SWAP: {
      // quarter of the state: indices with both bits 0
      const uint32_t lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
      for (uint32_t t = threadIdx.x; t < (half >> 1); t += blockDim.x) {
        uint32_t b = t;
        b = ((b >> lo) << (lo + 1)) | (b & ((1u << lo) - 1));
        b = ((b >> hi) << (hi + 1)) | (b & ((1u << hi) - 1));
        if (G.cls == BG_CX) {  // swap |c=1,t=0> and |c=1,t=1>
          C a = psi[b | m0], d = psi[b | m0 | m1];
          psi[b | m0] = d;
          psi[b | m0 | m1] = a;
        } else if (G.cls == BG_CZ) {
          C a = psi[b | m0 | m1];
          psi[b | m0 | m1] = C{-a.x, -a.y};
        } else {
          C a = psi[b | m0], d = psi[b | m1];
          psi[b | m0] = d;
          psi[b | m1] = a;
        }
      }
      return;
    }
    case BG_DIAG2:  // parity phases
      for (uint32_t b = threadIdx.x; b < 2 * half; b += blockDim.x) {
        uint32_t par = ((b >> q0) ^ (b >> q1)) & 1u;
        psi[b] = cmul<C, R>(G.m[par], psi[b]);
      }
      return;
    case BG_DIAG:
      for (uint32_t b = threadIdx.x; b < 2 * half; b += blockDim.x) psi[b] = cmul<C, R>(G.m[(b >> q0) & 1u ? 3 : 0], psi[b]);
      return;
    default:
      break;
  }
  for (uint32_t t = threadIdx.x; t < half; t += blockDim.x) {
    uint32_t i0 = ((t >> q0) << (q0 + 1)) | (t & (m0 - 1));
    uint32_t i1 = i0 | m0;
    C a = psi[i0], d = psi[i1];
    C o0, o1;
    if (G.cls == BG_REAL) {
      o0 = C{fma(G.m[0].x, a.x, G.m[1].x * d.x), fma(G.m[0].x, a.y, G.m[1].x * d.y)};
      o1 = C{fma(G.m[2].x, a.x, G.m[3].x * d.x), fma(G.m[2].x, a.y, G.m[3].x * d.y)};
    } else {
      C x0 = cmul<C, R>(G.m[0], a), x1 = cmul<C, R>(G.m[1], d);
      C y0 = cmul<C, R>(G.m[2], a), y1 = cmul<C, R>(G.m[3], d);
      o0 = C{x0.x + x1.x, x0.y + x1.y};
      o1 = C{y0.x + y1.x, y0.y + y1.y};
    }
    psi[i0] = o0;
    psi[i1] = o1;
  }
}

// Block-wide FP64 sum; every thread gets the result.
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0;
  for (int w = 0; w < nw; w++) s += red[w];
  return s;
}

// ------------------------------------------------------------------ double words
// FP64 batches and trajectories in double-word arithmetic (the default; the
// FP64-pipe kernels run on request): the state in shared memory as float
// pairs (re.h, re.l, im.h, im.l: 16 bytes per amplitude, as complex128),
// gate matrices built in FP64 and split into float pairs, every gate, norm
// and term product in double words on the FP32 pipe (dw.cuh), each thread's
// sums kept as compensated float pairs and added across the block in FP64.
struct GateMatDw {
  float4 m[4];  // (re.h, re.l, im.h, im.l) per entry
  int cls;
};
static_assert(sizeof(GateMatDw) <= sizeof(GateMat<double>), "the FP64 kernel's shared-memory layout");

__device__ __forceinline__ float4 pack_dw(Dw re, Dw im) { return make_float4(re.h, re.l, im.h, im.l); }

// a b (complex)
__device__ __forceinline__ float4 cmul_dw(float4 a, float4 b) {
  const Dw ar{a.x, a.y}, ai{a.z, a.w}, br{b.x, b.y}, bi{b.z, b.w};
  return pack_dw(dw_fma(ar, br, dw_mul(dw_neg(ai), bi)), dw_fma(ar, bi, dw_mul(ai, br)));
}

// a x + b y (complex)
__device__ __forceinline__ float4 cmul2_dw(float4 a, float4 x, float4 b, float4 y) {
  const Dw ar{a.x, a.y}, ai{a.z, a.w}, br{b.x, b.y}, bi{b.z, b.w};
  const Dw xr{x.x, x.y}, xi{x.z, x.w}, yr{y.x, y.y}, yi{y.z, y.w};
  return pack_dw(dw_fma(ar, xr, dw_fma(dw_neg(ai), xi, dw_fma(br, yr, dw_mul(dw_neg(bi), yi)))),
                 dw_fma(ar, xi, dw_fma(ai, xr, dw_fma(br, yi, dw_mul(bi, yr)))));
}

__device__ void apply_gate_dw(float4* __restrict__ psi, int n, const BGate& g, const GateMatDw& G) {
  const uint32_t half = 1u << (n - 1);
  const uint32_t q0 = g.q0, q1 = g.q1;
  const uint32_t m0 = 1u << q0, m1 = 1u << q1;
  switch (G.cls) {
    case BG_CX:
    case BG_CZ:
    case BG_SWAP: {
      const uint32_t lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
      for (uint32_t t = threadIdx.x; t < (half >> 1); t += blockDim.x) {
        uint32_t b = t;
        b = ((b >> lo) << (lo + 1)) | (b & ((1u << lo) - 1));
        b = ((b >> hi) << (hi + 1)) | (b & ((1u << hi) - 1));
        if (G.cls == BG_CX) {
          const float4 a = psi[b | m0], d = psi[b | m0 | m1];
          psi[b | m0] = d;
          psi[b | m0 | m1] = a;
        } else if (G.cls == BG_CZ) {
          const float4 a = psi[b | m0 | m1];
          psi[b | m0 | m1] = make_float4(-a.x, -a.y, -a.z, -a.w);
        } else {
          const float4 a = psi[b | m0], d = psi[b | m1];
          psi[b | m0] = d;
          psi[b | m1] = a;
        }
      }
      return;
    }
    case BG_DIAG2:
      for (uint32_t b = threadIdx.x; b < 2 * half; b += blockDim.x) {
        const uint32_t par = ((b >> q0) ^ (b >> q1)) & 1u;
        psi[b] = cmul_dw(G.m[par], psi[b]);
      }
      return;
    case BG_DIAG:
      for (uint32_t b = threadIdx.x; b < 2 * half; b += blockDim.x) psi[b] = cmul_dw(G.m[(b >> q0) & 1u ? 3 : 0], psi[b]);
      return;
    default:
      break;
  }
  for (uint32_t t = threadIdx.x; t < half; t += blockDim.x) {
    const uint32_t i0 = ((t >> q0) << (q0 + 1)) | (t & (m0 - 1)), i1 = i0 | m0;
    const float4 a = psi[i0], d = psi[i1];
    float4 o0, o1;
    if (G.cls == BG_REAL) {
      const Dw r0{G.m[0].x, G.m[0].y}, r1{G.m[1].x, G.m[1].y}, r2{G.m[2].x, G.m[2].y}, r3{G.m[3].x, G.m[3].y};
      const Dw ar{a.x, a.y}, ai{a.z, a.w}, dr{d.x, d.y}, di{d.z, d.w};
      o0 = pack_dw(dw_fma(r0, ar, dw_mul(r1, dr)), dw_fma(r0, ai, dw_mul(r1, di)));
      o1 = pack_dw(dw_fma(r2, ar, dw_mul(r3, dr)), dw_fma(r2, ai, dw_mul(r3, di)));
    } else {
      o0 = cmul2_dw(G.m[0], a, G.m[1], d);
      o1 = cmul2_dw(G.m[2], a, G.m[3], d);
    }
    psi[i0] = o0;
    psi[i1] = o1;
  }
}

// ------------------------------------------------------------------ precision modes
// The batched and trajectory kernels run in one of three modes: 0 FP32
// (float2 amplitudes), 1 FP64 on the FP64 pipe (double2), 2 FP64 in double
// words (float4: re.h, re.l, im.h, im.l).  The helpers below are overloaded
// on the amplitude type.
template <int M>
struct Mode;

__device__ __forceinline__ void put_real(float2& v, float x) { v = make_float2(x, 0.f); }
__device__ __forceinline__ void put_real(double2& v, float x) { v = make_double2(x, 0.0); }
__device__ __forceinline__ void put_real(float4& v, float x) { v = make_float4(x, 0.f, 0.f, 0.f); }

__device__ __forceinline__ void build_mat(const BGate& g, const BGate* all, const double* p, GateMat<float>& out) {
  make_gate<float>(g, all, p, out);
}
__device__ __forceinline__ void build_mat(const BGate& g, const BGate* all, const double* p, GateMat<double>& out) {
  make_gate<double>(g, all, p, out);
}
__device__ __forceinline__ void build_mat(const BGate& g, const BGate* all, const double* p, GateMatDw& out) {
  GateMat<double> m;
  make_gate<double>(g, all, p, m);
  for (int e = 0; e < 4; e++) out.m[e] = pack_dw(dw_split(m.m[e].x), dw_split(m.m[e].y));
  out.cls = m.cls;
}

__device__ __forceinline__ void apply_m(float2* psi, int n, const BGate& g, const GateMat<float>& G) {
  apply_gate<float>(psi, n, g, G);
}
__device__ __forceinline__ void apply_m(double2* psi, int n, const BGate& g, const GateMat<double>& G) {
  apply_gate<double>(psi, n, g, G);
}
__device__ __forceinline__ void apply_m(float4* psi, int n, const BGate& g, const GateMatDw& G) {
  apply_gate_dw(psi, n, g, G);
}

// -i v and -v
__device__ __forceinline__ float2 mul_mi(float2 v) { return make_float2(v.y, -v.x); }
__device__ __forceinline__ double2 mul_mi(double2 v) { return make_double2(v.y, -v.x); }
__device__ __forceinline__ float4 mul_mi(float4 v) { return make_float4(v.z, v.w, -v.x, -v.y); }
__device__ __forceinline__ float2 neg(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ double2 neg(double2 v) { return make_double2(-v.x, -v.y); }
__device__ __forceinline__ float4 neg(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }

// v f for an FP64 factor f: FP64 product (double2); float pair f = fh + fl with
// one FMA, x fl + x fh (float2); double-word product (float4)
struct Factor {
  double d;
  float h, l;
  Dw w;
  __device__ explicit Factor(double f) : d(f), h((float)f), l((float)(f - (double)(float)f)), w(dw_split(f)) {}
};
__device__ __forceinline__ float2 scale(float2 v, const Factor& f) {
  return make_float2(__fmaf_rn(v.x, f.l, __fmul_rn(v.x, f.h)), __fmaf_rn(v.y, f.l, __fmul_rn(v.y, f.h)));
}
__device__ __forceinline__ double2 scale(double2 v, const Factor& f) { return make_double2(v.x * f.d, v.y * f.d); }
__device__ __forceinline__ float4 scale(float4 v, const Factor& f) {
  return pack_dw(dw_mul(Dw{v.x, v.y}, f.w), dw_mul(Dw{v.z, v.w}, f.w));
}

// Per-thread sums of |v|^2 and of the term values Re / Im conj(q) p with a
// sign: FP64 arithmetic (FP64 mode); compensated float pairs with exact
// products (FP32: TwoProduct) or double-word products (double words).
struct AccF64 {
  double s = 0.0;
  __device__ void abs2(double2 v) { s = fma(v.x, v.x, fma(v.y, v.y, s)); }
  __device__ void term(double2 q, double2 p, bool imag, bool neg) {
    const double v = imag ? fma(q.x, p.y, -q.y * p.x) : fma(q.x, p.x, q.y * p.y);
    s += neg ? -v : v;
  }
  __device__ double value() const { return s; }
};
struct AccPair {
  float s = 0.f, c = 0.f;
  __device__ void abs2(float2 v) {
    dw_acc(s, c, two_prod(v.x, v.x), 0u);
    dw_acc(s, c, two_prod(v.y, v.y), 0u);
  }
  __device__ void abs2(float4 v) {
    const Dw re{v.x, v.y}, im{v.z, v.w};
    dw_acc(s, c, dw_fma(re, re, dw_mul(im, im)), 0u);
  }
  __device__ void term(float2 q, float2 p, bool imag, bool neg) {  // qr pr + qi pi, or qr pi - qi pr
    const uint32_t sg = neg ? 0x80000000u : 0u;
    dw_acc(s, c, two_prod(q.x, imag ? p.y : p.x), sg);
    dw_acc(s, c, two_prod(q.y, imag ? p.x : p.y), imag ? sg ^ 0x80000000u : sg);
  }
  __device__ void term(float4 q, float4 p, bool imag, bool neg) {
    const Dw pr{p.x, p.y}, pi{p.z, p.w}, qr{q.x, q.y}, qi{q.z, q.w};
    const Dw v = imag ? dw_fma(qr, pi, dw_mul(dw_neg(qi), pr)) : dw_fma(qr, pr, dw_mul(qi, pi));
    dw_acc(s, c, v, neg ? 0x80000000u : 0u);
  }
  __device__ double value() const { return (double)s + (double)c; }
};

template <>
struct Mode<0> {
  using E = float2;
  using Mat = GateMat<float>;
  using Acc = AccPair;
};
template <>
struct Mode<1> {
  using E = double2;
  using Mat = GateMat<double>;
  using Acc = AccF64;
};
template <>
struct Mode<2> {
  using E = float4;
  using Mat = GateMatDw;
  using Acc = AccPair;
};
static_assert(sizeof(GateMatDw) == sizeof(GateMat<double>), "FP64 modes share one shared-memory layout");

// Norm and per-term values <P_t> / norm of the state in shared memory (vals[t],
// written by thread 0; the caller synchronises before reading them).
template <int M>
__device__ double norm_and_terms(const typename Mode<M>::E* __restrict__ psi, uint32_t N,
                                 const BTerm* __restrict__ terms, int nt, double* red, double* vals) {
  using Acc = typename Mode<M>::Acc;
  Acc an;
  for (uint32_t b = threadIdx.x; b < N; b += blockDim.x) an.abs2(psi[b]);
  const double nrm = block_sum(an.value(), red);
  for (int t = 0; t < nt; t++) {
    const BTerm tm = terms[t];
    const bool imag = tm.y & 1, neg0 = tm.y == 1 || tm.y == 2;
    Acc at;
    for (uint32_t b = threadIdx.x; b < N; b += blockDim.x) {
      const auto pv = psi[b];
      const auto qv = tm.x ? psi[b ^ tm.x] : pv;
      at.term(qv, pv, imag, neg0 ^ (bool)(__popc(b & tm.z) & 1));
    }
    const double acc = block_sum(at.value(), red);
    if (threadIdx.x == 0) vals[t] = acc / nrm;
  }
  return nrm;
}

template <int M, int TH>
__global__ void __launch_bounds__(TH) batch_kernel(BatchArgs a) {
  using E = typename Mode<M>::E;
  using Mat = typename Mode<M>::Mat;
  extern __shared__ __align__(16) unsigned char smem[];
  E* psi = reinterpret_cast<E*>(smem);
  Mat* mats = reinterpret_cast<Mat*>(smem + (sizeof(E) << a.max_n));
  double* red = reinterpret_cast<double*>(mats + a.max_gates);  // 32 doubles
  double* vals = red + 32;                                       // max_terms + 1 doubles
  __shared__ int s_job;
  for (int iter = 0; iter < a.njobs; iter++) {  // bounded: at most njobs jobs per CTA
    if (threadIdx.x == 0) s_job = atomicAdd(a.counter, 1);
    __syncthreads();
    const int job = s_job;
    __syncthreads();
    if (job >= a.njobs) break;
    const int tid = a.job_template ? a.job_template[job] : 0;
    if (tid < 0 || tid >= a.ntemplates) {  // invalid template index: NaN energies
      for (int e = threadIdx.x; e < a.out_stride; e += blockDim.x) a.out[(size_t)job * a.out_stride + e] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    const BTemplate T = a.templates[tid];
    const double* p = a.params + (size_t)job * a.nparams;
    const int n = T.n;
    const uint32_t N = 1u << n;
    // |0..0>
    for (uint32_t b = threadIdx.x; b < N; b += blockDim.x) put_real(psi[b], b == 0 ? 1.f : 0.f);
    // per-job gate matrices (each thread builds different gates)
    for (int k = threadIdx.x; k < T.ng; k += blockDim.x) build_mat(a.gates[T.g0 + k], a.gates, p, mats[k]);
    __syncthreads();
    for (int k = 0; k < T.ng; k++) {
      apply_m(psi, n, a.gates[T.g0 + k], mats[k]);
      __syncthreads();
    }
    const double nrm = norm_and_terms<M>(psi, N, a.terms + T.t0, T.nt, red, vals);
    __syncthreads();
    for (int e = threadIdx.x; e < T.ne; e += blockDim.x) {
      double s = 0;
      for (int t = 0; t < T.nt; t++) s = fma(a.coeffs[T.c0 + e * T.nt + t], vals[t], s);
      a.out[(size_t)job * a.out_stride + e] = s;
    }
    if (a.norms && threadIdx.x == 0) a.norms[job] = nrm;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ quantum trajectories
// Noisy state vectors by Monte-Carlo unravelling of the device noise model
// (the stochastic alternative to the density matrix of paper Sec. II/III):
// one CTA per trajectory, the state in shared memory.  After each gate, with
// the trajectory's draws u (inputs, consumed in order):
//   depolarising p on k qubits: one draw x; if x < (4^k - 1) p / 4^k the
//     Pauli string s = 1 + floor(x 4^k / p) (<= 4^k - 1) is applied,
//     s & 3 on q0 and s >> 2 on q1 (0 I, 1 X, 2 Y, 3 Z);
//   relaxation on each gate qubit: amplitude damping (gamma) then phase
//     damping (lambda), one draw x each: with P1 = prob(q = 1) (a block sum
//     with FP64 accuracy), the jump |0><1| (resp. |1><1|) when x < rate P1,
//     else diag(1, sqrt(1 - rate)); the state is renormalised by FP64 factors.
// Every thread reads the same draw and the same P1, so branches are uniform.
template <class E>
__device__ void apply_pauli(E* __restrict__ psi, int n, int q, int a) {
  const uint32_t half = 1u << (n - 1), m = 1u << q;
  for (uint32_t t = threadIdx.x; t < half; t += blockDim.x) {
    const uint32_t b0 = ((t >> q) << (q + 1)) | (t & (m - 1)), b1 = b0 | m;
    const E x0 = psi[b0], x1 = psi[b1];
    if (a == 1) {  // X
      psi[b0] = x1;
      psi[b1] = x0;
    } else if (a == 2) {  // Y: (x0, x1) -> (-i x1, i x0)
      psi[b0] = mul_mi(x1);
      psi[b1] = neg(mul_mi(x0));
    } else {  // Z
      psi[b1] = neg(x1);
    }
  }
}

template <int M>
__global__ void __launch_bounds__(256) traj_kernel(TrajArgs a) {
  using E = typename Mode<M>::E;
  using Mat = typename Mode<M>::Mat;
  using Acc = typename Mode<M>::Acc;
  extern __shared__ __align__(16) unsigned char smem[];
  E* psi = reinterpret_cast<E*>(smem);
  Mat* mats = reinterpret_cast<Mat*>(smem + (sizeof(E) << a.n));
  double* red = reinterpret_cast<double*>(mats + a.ng);  // 32 doubles
  double* vals = red + 32;                                // nt doubles
  __shared__ int s_job;
  const int n = a.n;
  const uint32_t N = 1u << n, half = N >> 1;
  // fixed circuit: gate matrices once per CTA
  for (int k = threadIdx.x; k < a.ng; k += blockDim.x) build_mat(a.gates[k], a.gates, nullptr, mats[k]);
  __syncthreads();
  for (int iter = 0; iter < a.ntraj; iter++) {  // bounded: at most ntraj trajectories per CTA
    if (threadIdx.x == 0) s_job = atomicAdd(a.counter, 1);
    __syncthreads();
    const int job = s_job;
    __syncthreads();
    if (job >= a.ntraj) break;
    const double* u = a.u + (size_t)job * a.draws;
    int used = 0;
    for (uint32_t b = threadIdx.x; b < N; b += blockDim.x) put_real(psi[b], b == 0 ? 1.f : 0.f);
    __syncthreads();
    for (int g = 0; g < a.ng; g++) {
      const BGate& G = a.gates[g];
      apply_m(psi, n, G, mats[g]);
      __syncthreads();
      const TNoise& T = a.noise[g];
      if (T.pdep > 0) {
        const double x = u[used++];
        const int np = 1 << (2 * T.k);
        if (x < (np - 1) * T.pdep / np) {
          int s = 1 + (int)floor(x * np / T.pdep);
          if (s > np - 1) s = np - 1;
          for (int w = 0; w < T.k; w++) {
            const int pa = (s >> (2 * w)) & 3;
            if (pa) {
              apply_pauli(psi, n, w == 0 ? G.q0 : G.q1, pa);
              __syncthreads();
            }
          }
        }
      }
      if (!T.relax) continue;
      for (int w = 0; w < T.k; w++) {
        const int q = w == 0 ? G.q0 : G.q1;
        const uint32_t m = 1u << q;
        for (int step = 0; step < 2; step++) {
          const double rate = step == 0 ? T.gamma[w] : T.lambda[w];
          const double x = u[used++];
          Acc ap;
          for (uint32_t t = threadIdx.x; t < half; t += blockDim.x) ap.abs2(psi[((t >> q) << (q + 1)) | (t & (m - 1)) | m]);
          const double p1 = block_sum(ap.value(), red);
          const bool jump = x < rate * p1;
          const double f0 = jump ? 0.0 : 1.0 / sqrt(1.0 - rate * p1);  // |0> part
          const Factor F0(f0), F1(jump ? 1.0 / sqrt(p1) : sqrt(1.0 - rate) * f0);
          for (uint32_t t = threadIdx.x; t < half; t += blockDim.x) {
            const uint32_t b0 = ((t >> q) << (q + 1)) | (t & (m - 1)), b1 = b0 | m;
            const E x0 = psi[b0], x1 = psi[b1];
            if (jump && step == 0) {  // |0><1|: the |1> part moves down
              psi[b0] = scale(x1, F1);
              put_real(psi[b1], 0.f);
            } else if (jump) {  // |1><1|: the |0> part vanishes
              put_real(psi[b0], 0.f);
              psi[b1] = scale(x1, F1);
            } else {
              psi[b0] = scale(x0, F0);
              psi[b1] = scale(x1, F1);
            }
          }
          __syncthreads();
        }
      }
    }
    // energies of the (normalised) final state
    norm_and_terms<M>(psi, N, a.terms, a.nt, red, vals);
    __syncthreads();
    for (int e = threadIdx.x; e < a.ne; e += blockDim.x) {
      double s = 0;
      for (int t = 0; t < a.nt; t++) s = fma(a.coeffs[e * a.nt + t], vals[t], s);
      a.out[(size_t)job * a.ne + e] = s;
    }
    __syncthreads();
  }
}

size_t traj_smem_bytes(bool f64, int n, int ng, int nt) {
  size_t c = f64 ? 16 : 8;
  size_t gm = f64 ? sizeof(GateMat<double>) : sizeof(GateMat<float>);
  return (c << n) + gm * (size_t)(ng > 0 ? ng : 1) + 8 * (32 + (size_t)nt + 1);
}

template <int M>
static cudaError_t launch_traj_t(const TrajArgs& a, size_t smem, int sm_count, cudaStream_t s) {
  static int attr_dev = -1;
  static std::mutex attr_mu;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaError_t e = cudaSuccess;
  {
    std::lock_guard<std::mutex> lk(attr_mu);
    if (attr_dev != dev) {
      e = cudaFuncSetAttribute(traj_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchMaxSmem);
      if (e == cudaSuccess) attr_dev = dev;
    }
  }
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, traj_kernel<M>, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = sm_count * per_sm;
  if (grid > a.ntraj) grid = a.ntraj;
  e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  traj_kernel<M><<<grid, 256, smem, s>>>(a);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_traj(bool f64, const TrajArgs& a, int sm_count, cudaStream_t s) {
  const size_t smem = traj_smem_bytes(f64, a.n, a.ng, a.nt);
  if (smem > (size_t)kBatchMaxSmem || a.ntraj < 1) return cudaErrorInvalidValue;
  if (!f64) return launch_traj_t<0>(a, smem, sm_count, s);
  return a.dw ? launch_traj_t<2>(a, smem, sm_count, s) : launch_traj_t<1>(a, smem, sm_count, s);
}

size_t batch_smem_bytes(bool f64, int max_n, int max_gates, int max_terms) {
  size_t c = f64 ? 16 : 8;
  size_t gm = f64 ? sizeof(GateMat<double>) : sizeof(GateMat<float>);
  return (c << max_n) + gm * (size_t)max_gates + 8 * (32 + (size_t)max_terms + 1);
}

// Batched kernel of a precision mode: 0 FP32, 1 FP64 on the FP64 pipe, 2 FP64
// in double words.
template <int MODE, int TH>
static void (*batch_fn())(BatchArgs) {
  return batch_kernel<MODE, TH>;
}

template <int MODE, int TH>
static cudaError_t launch_batch_t(const BatchArgs& a, size_t smem, int sm_count, cudaStream_t s) {
  void (*fn)(BatchArgs) = batch_fn<MODE, TH>();
  // The attribute is a per-function maximum shared by every caller (several
  // host threads may launch concurrently): set it once to the largest size any
  // batch may use, never per call.
  static int attr_dev = -1;
  static std::mutex attr_mu;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaError_t e = cudaSuccess;
  {
    std::lock_guard<std::mutex> lk(attr_mu);
    if (attr_dev != dev) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchMaxSmem);
      if (e == cudaSuccess) attr_dev = dev;
    }
  }
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TH, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = sm_count * per_sm;
  if (grid > a.njobs) grid = a.njobs;
  e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  fn<<<grid, TH, smem, s>>>(a);
  g_launches += 1;
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_batch_m(const BatchArgs& a, size_t smem, int sm_count, cudaStream_t s) {
  switch (a.threads) {
    case 128: return launch_batch_t<MODE, 128>(a, smem, sm_count, s);
    case 256: return launch_batch_t<MODE, 256>(a, smem, sm_count, s);
    case 512: return launch_batch_t<MODE, 512>(a, smem, sm_count, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch(bool f64, const BatchArgs& a, int sm_count, cudaStream_t s) {
  const size_t smem = batch_smem_bytes(f64, a.max_n, a.max_gates, a.max_terms);
  if (smem > (size_t)kBatchMaxSmem) return cudaErrorInvalidValue;
  if (!f64) return launch_batch_m<0>(a, smem, sm_count, s);
  return a.dw ? launch_batch_m<2>(a, smem, sm_count, s) : launch_batch_m<1>(a, smem, sm_count, s);
}

}  // namespace nwq
