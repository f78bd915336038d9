// Device kernels of the simulator (sm_103a).
//
// sweep_kernel: the hot path.  One sweep = stage a tile of 2^T state elements
// (2^m contiguous elements x 2^h strided chunks) in shared memory with 16-byte
// vector loads, apply the sweep's operators in order (each operator acts on
// k <= 4 tile-local bits; __syncthreads between operators), write the tile
// back.  The grid is persistent over tiles (grid = SMs x resident CTAs).
//
// Paper Sec. II: SV-Sim applies gates to the 2^n-amplitude state vector;
// DM-Sim applies gates and noise channels to the density matrix.  Here the
// density matrix is held as its 4^n real Pauli coefficients and every gate
// plus its noise is one real Pauli-transfer matrix on bits (q, q+n), so the
// same engine serves both (complex elements for SV, real for DM).
#include <cstring>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "nwq_internal.h"
#include "kernels.hpp"
#include "device_util.cuh"

namespace nwq {

std::atomic<unsigned long long> g_launches{0};

// Insert a zero bit at each position of `pos` (ascending) into g.
template <int K>
__device__ __forceinline__ uint32_t insert_zeros(uint32_t g, const uint8_t* sorted_pos) {
#pragma unroll
  for (int t = 0; t < K; t++) {
    uint32_t p = sorted_pos[t];
    uint32_t lowm = (1u << p) - 1u;
    g = ((g & ~lowm) << 1) | (g & lowm);
  }
  return g;
}

// Signed copy of x (base = 1: +x, 2: -x) or +0 (base = 0), with integer
// operations only: the FP64 pipe is the scarce unit on this GPU, so no
// floating-point instruction is spent on unit coefficients.
__device__ __forceinline__ double signed_base(double x, int base) {
  long long b = __double_as_longlong(x) ^ (base == 2 ? (long long)0x8000000000000000ull : 0ll);
  return __longlong_as_double(base ? b : 0ll);
}
__device__ __forceinline__ float signed_base(float x, int base) {
  int b = __float_as_int(x) ^ (base == 2 ? (int)0x80000000u : 0);
  return __int_as_float(base ? b : 0);
}
__device__ __forceinline__ double2 signed_base(double2 v, int base) {
  return make_double2(signed_base(v.x, base), signed_base(v.y, base));
}
__device__ __forceinline__ float2 signed_base(float2 v, int base) {
  return make_float2(signed_base(v.x, base), signed_base(v.y, base));
}

// ------------------------------------------------------------------ operator application
// Each operator is applied out of place, src tile -> dst tile (ping-pong in
// shared memory), one output row at a time: a warp takes one row i of the
// operator and 32*G of its 2^(T-k) groups (lane l handles groups
// c0 + u*32 + l, u < G, so the lanes of a warp touch consecutive shared
// memory words).  The row's entries are warp-uniform; each entry feeds G
// independent FMA chains.  Rows are either copies (identity / +-unit entry,
// integer operations only) or a unit-entry start plus one FMA per remaining
// entry; entry loops stay rolled so no predicated-off FP64 instruction
// occupies the FP64 pipe, the unit this GPU has least of.
constexpr int kILP = 4;

template <int K>
__device__ __forceinline__ void group_bases(uint32_t c0, uint32_t ngroups, const uint8_t* slb, uint32_t (&b)[kILP],
                                            bool (&valid)[kILP]) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int u = 0; u < kILP; u++) {
    uint32_t g = c0 + (uint32_t)u * 32u + lane;
    valid[u] = g < ngroups;
    b[u] = insert_zeros<K>(valid[u] ? g : 0u, slb);
  }
}

template <int K, class R>
__device__ __forceinline__ void apply_real(const R* __restrict__ src, R* __restrict__ dst, int T, const DevOp& op,
                                           const EntR<R>* __restrict__ e0) {
  constexpr int D = 1 << K;
  const uint32_t ngroups = 1u << (T - K);
  const uint32_t per = 32u * kILP;
  const uint32_t nchunk = (ngroups + per - 1) / per;
  const uint32_t nitems = (uint32_t)D * nchunk;
  for (uint32_t item = threadIdx.x >> 5; item < nitems; item += kSweepThreads / 32) {
    const uint32_t i = item / nchunk, c0 = (item % nchunk) * per;
    const RowMeta rm = op.row[i];
    uint32_t b[kILP];
    bool valid[kILP];
    group_bases<K>(c0, ngroups, op.slb, b, valid);
    R acc[kILP];
    if (rm.kind == ROW_ID) {
#pragma unroll
      for (int u = 0; u < kILP; u++) acc[u] = src[b[u] + rm.out];
    } else {
#pragma unroll
      for (int u = 0; u < kILP; u++) acc[u] = signed_base(src[b[u] + rm.boff], rm.base);
      if (rm.kind == ROW_GEN) {
        const EntR<R>* e = e0 + rm.beg;
        const int cnt = rm.cnt[0];
#pragma unroll 1
        for (int c = 0; c < cnt; c++) {
          const R cf = e[c].c;
          const uint32_t off = e[c].off;
#pragma unroll
          for (int u = 0; u < kILP; u++) acc[u] = fma(cf, src[b[u] + off], acc[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kILP; u++)
      if (valid[u]) dst[b[u] + rm.out] = acc[u];
  }
}

template <int K, class R>
__device__ __forceinline__ void apply_cplx(const typename Cplx<R>::T* __restrict__ src, typename Cplx<R>::T* __restrict__ dst,
                                           int T, const DevOp& op, const EntC<R>* __restrict__ e0) {
  using C = typename Cplx<R>::T;
  constexpr int D = 1 << K;
  const uint32_t ngroups = 1u << (T - K);
  const uint32_t per = 32u * kILP;
  const uint32_t nchunk = (ngroups + per - 1) / per;
  const uint32_t nitems = (uint32_t)D * nchunk;
  for (uint32_t item = threadIdx.x >> 5; item < nitems; item += kSweepThreads / 32) {
    const uint32_t i = item / nchunk, c0 = (item % nchunk) * per;
    const RowMeta rm = op.row[i];
    uint32_t b[kILP];
    bool valid[kILP];
    group_bases<K>(c0, ngroups, op.slb, b, valid);
    C acc[kILP];
    if (rm.kind == ROW_ID) {
#pragma unroll
      for (int u = 0; u < kILP; u++) acc[u] = src[b[u] + rm.out];
    } else {
#pragma unroll
      for (int u = 0; u < kILP; u++) acc[u] = signed_base(src[b[u] + rm.boff], rm.base);
      if (rm.kind == ROW_GEN) {
        const EntC<R>* e = e0 + rm.beg;
        const int c0n = rm.cnt[0], c1n = c0n + rm.cnt[1], c2n = c1n + rm.cnt[2];
        int c = 0;
#pragma unroll 1
        for (; c < c0n; c++) {
          const R re = e[c].re;
          const uint32_t off = e[c].off;
#pragma unroll
          for (int u = 0; u < kILP; u++) {
            const C x = src[b[u] + off];
            acc[u].x = fma(re, x.x, acc[u].x);
            acc[u].y = fma(re, x.y, acc[u].y);
          }
        }
#pragma unroll 1
        for (; c < c1n; c++) {
          const R im = e[c].im;
          const uint32_t off = e[c].off;
#pragma unroll
          for (int u = 0; u < kILP; u++) {
            const C x = src[b[u] + off];
            acc[u].x = fma(-im, x.y, acc[u].x);
            acc[u].y = fma(im, x.x, acc[u].y);
          }
        }
#pragma unroll 1
        for (; c < c2n; c++) {
          const R re = e[c].re, im = e[c].im;
          const uint32_t off = e[c].off;
#pragma unroll
          for (int u = 0; u < kILP; u++) {
            const C x = src[b[u] + off];
            acc[u].x = fma(re, x.x, fma(-im, x.y, acc[u].x));
            acc[u].y = fma(re, x.y, fma(im, x.x, acc[u].y));
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kILP; u++)
      if (valid[u]) dst[b[u] + rm.out] = acc[u];
  }
}

// ------------------------------------------------------------------ sweep kernel
// Padded tile layout: one 16-byte pad after every 128 bytes of elements, so
// lanes whose indices differ by multiples of 128 bytes fall on different
// banks.  pad(a | b) = pad(a) + pad(b) for indices with disjoint bits, which
// lets a phase precompute per-register offsets (an element address is then
// one add) and keeps 16-byte vectors contiguous and aligned.
template <class C>
__device__ __forceinline__ uint32_t swz(uint32_t l) {
  if constexpr (sizeof(C) == 16) return l + (l >> 3);       // 8 complex128 + 1 pad
  else return l + ((l >> 4) << 1);                          // 16 complex64 + 2 pad
}
template <class C>
__host__ __device__ constexpr size_t padded_elems(int T) {
  return sizeof(C) == 16 ? ((size_t)1 << T) + ((size_t)1 << T) / 8 : ((size_t)1 << T) + ((size_t)1 << T) / 8;
}

// Byte offset of the chunk-offset table in shared memory: after the tile(s)
// (tile_bytes_per_elem << T) and, when the tables are staged, after them.
__host__ __device__ inline size_t hoff_offset(const SweepDesc& sd, size_t tile_bytes_per_elem, bool tbl,
                                              size_t table_bytes) {
  size_t o = (tile_bytes_per_elem << sd.T) + (tbl ? table_bytes : 0);
  return (o + 15) & ~(size_t)15;
}

template <class C>
__host__ __device__ inline size_t phase_hoff_offset(const SweepDesc& sd, bool tbl) {
  size_t o = 2 * sizeof(C) * padded_elems<C>(sd.T);
  if (tbl) o += sizeof(PhaseDesc) * sd.nph + sizeof(PhaseOp) * sd.npop + sizeof(C) * sd.npc;
  return (o + 15) & ~(size_t)15;
}

template <class R, bool CPLX>
using ElemT = typename std::conditional<CPLX, typename Cplx<R>::T, R>::type;
template <class R, bool CPLX>
using EntT = typename std::conditional<CPLX, EntC<R>, EntR<R>>::type;

// Shared memory: tile A | tile B | the sweep's operators | their entries (when
// TBL; otherwise the tables are read from global memory through L1).
template <class R, bool CPLX, bool TBL>
__global__ void __launch_bounds__(kSweepThreads) sweep_kernel(void* __restrict__ state_v, uint64_t ntiles, SweepDesc sd,
                                                              const DevOp* __restrict__ ops_g,
                                                              const void* __restrict__ ents_v) {
  using E = ElemT<R, CPLX>;
  using Ent = EntT<R, CPLX>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int T = sd.T;
  E* tileA = reinterpret_cast<E*>(smem_raw);
  E* tileB = tileA + (1u << T);
  const DevOp* ops = ops_g + sd.op0;
  const Ent* ents = reinterpret_cast<const Ent*>(ents_v) + sd.ent0;  // entry e of the sweep at ents[e - ent0]
  if constexpr (TBL) {
    DevOp* sops = reinterpret_cast<DevOp*>(tileB + (1u << T));
    Ent* sents = reinterpret_cast<Ent*>(sops + sd.nops);
    const uint4* s1 = reinterpret_cast<const uint4*>(ops_g + sd.op0);
    uint4* d1 = reinterpret_cast<uint4*>(sops);
    for (uint32_t v = threadIdx.x; v < sd.nops * (sizeof(DevOp) / 16); v += kSweepThreads) d1[v] = s1[v];
    const uint32_t* s2 = reinterpret_cast<const uint32_t*>(reinterpret_cast<const Ent*>(ents_v) + sd.ent0);
    uint32_t* d2 = reinterpret_cast<uint32_t*>(sents);
    for (uint32_t v = threadIdx.x; v < sd.nent * (sizeof(Ent) / 4); v += kSweepThreads) d2[v] = s2[v];
    ops = sops;
    ents = sents;
  }
  E* state = reinterpret_cast<E*>(state_v);
  constexpr int VPE = 16 / sizeof(E);  // elements per 16-byte vector
  const uint32_t nvec = (1u << T) / VPE;
  const int lvpc = sd.m - __ffs(VPE) + 1;  // log2(vectors per contiguous chunk)
  const uint32_t vpc_mask = (1u << lvpc) - 1u;
  // global offset of each strided chunk of the tile, computed once per CTA
  uint64_t* hoff = reinterpret_cast<uint64_t*>(smem_raw + hoff_offset(sd, 2 * sizeof(E), TBL,
                                                                     sizeof(DevOp) * sd.nops + sizeof(Ent) * sd.nent));
  for (uint32_t j = threadIdx.x; j < (1u << sd.h); j += kSweepThreads) hoff[j] = deposit(j, sd.hmask);
  __syncthreads();

  for (uint64_t tileid = blockIdx.x; tileid < ntiles; tileid += gridDim.x) {
    // base = tile id scattered onto the non-tile bits
    const uint64_t base = deposit(tileid, sd.fmask);
    for (uint32_t v = threadIdx.x; v < nvec; v += kSweepThreads) {
      uint64_t off = base + hoff[v >> lvpc] + (uint64_t)(v & vpc_mask) * VPE;
      reinterpret_cast<uint4*>(tileA)[v] = __ldg(reinterpret_cast<const uint4*>(state + off));
    }
    __syncthreads();
    E* src = tileA;
    E* dst = tileB;
    for (int o = 0; o < sd.nops; o++) {
      const DevOp& op = ops[o];
      const Ent* e0 = ents + (op.ent - sd.ent0);
      if constexpr (CPLX) {
        switch (op.k) {
          case 1: apply_cplx<1, R>(src, dst, T, op, e0); break;
          case 2: apply_cplx<2, R>(src, dst, T, op, e0); break;
          case 3: apply_cplx<3, R>(src, dst, T, op, e0); break;
          default: apply_cplx<4, R>(src, dst, T, op, e0); break;
        }
      } else {
        switch (op.k) {
          case 1: apply_real<1, R>(src, dst, T, op, e0); break;
          case 2: apply_real<2, R>(src, dst, T, op, e0); break;
          case 3: apply_real<3, R>(src, dst, T, op, e0); break;
          default: apply_real<4, R>(src, dst, T, op, e0); break;
        }
      }
      __syncthreads();
      E* t = src;
      src = dst;
      dst = t;
    }
    for (uint32_t v = threadIdx.x; v < nvec; v += kSweepThreads) {
      uint64_t off = base + hoff[v >> lvpc] + (uint64_t)(v & vpc_mask) * VPE;
      reinterpret_cast<uint4*>(state + off)[0] = reinterpret_cast<const uint4*>(src)[v];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ register-phase kernel (complex)
// One shared-memory tile per CTA (XOR-swizzled so that lanes differing only in
// higher index bits hit different banks).  Per phase every thread loads the
// 16 elements of a group (all values of the phase's 4 register bits) into
// registers, applies the phase's operators there and stores them back.
__host__ __device__ constexpr int dep4(int v, int mask) {  // deposit v's low bits on mask's set bits
  int out = 0, bit = 0;
  for (int p = 0; p < 4; p++)
    if ((mask >> p) & 1) {
      if ((v >> bit) & 1) out |= 1 << p;
      bit++;
    }
  return out;
}
__host__ __device__ constexpr int popc4(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1); }

template <class R>
__device__ __forceinline__ typename Cplx<R>::T cfma(typename Cplx<R>::T c, typename Cplx<R>::T x, typename Cplx<R>::T acc) {
  acc.x = fma(c.x, x.x, fma(-c.y, x.y, acc.x));
  acc.y = fma(c.x, x.y, fma(c.y, x.x, acc.y));
  return acc;
}

// Dense operator on register bits MASK (k <= 2) of NR-element groups, with the
// arithmetic fixed by its structure form: general complex (4 FMA per entry),
// real (2 FMA per entry) or X-rotation [[a, i b], [i c, d]] (2 FMA per entry).
template <int NR, int MASK, int FORM, class R>
__device__ __forceinline__ void phase_dense(typename Cplx<R>::T (&r)[NR], const typename Cplx<R>::T* __restrict__ c) {
  using C = typename Cplx<R>::T;
  constexpr int K = popc4(MASK), D = 1 << K;
  C m[D * D];
#pragma unroll
  for (int e = 0; e < D * D; e++) m[e] = c[e];
#pragma unroll
  for (int o = 0; o < NR; o++) {
    if (o & MASK) continue;
    C in[D];
#pragma unroll
    for (int j = 0; j < D; j++) in[j] = r[o | dep4(j, MASK)];
    if constexpr (FORM == PD_XROT) {  // K == 1
      const C a = in[0], b = in[1];
      r[o] = C{fma(m[0].x, a.x, -m[1].y * b.y), fma(m[0].x, a.y, m[1].y * b.x)};
      r[o | MASK] = C{fma(m[3].x, b.x, -m[2].y * a.y), fma(m[3].x, b.y, m[2].y * a.x)};
    } else if constexpr (FORM == PD_XROTU) {  // K == 1, unit diagonal
      const C a = in[0], b = in[1];
      r[o] = C{fma(-m[1].y, b.y, a.x), fma(m[1].y, b.x, a.y)};
      r[o | MASK] = C{fma(-m[2].y, a.y, b.x), fma(m[2].y, a.x, b.y)};
    } else {
#pragma unroll
      for (int i = 0; i < D; i++) {
        C acc{R(0), R(0)};
#pragma unroll
        for (int j = 0; j < D; j++) {
          if constexpr (FORM == PD_REAL) {
            acc.x = fma(m[i * D + j].x, in[j].x, acc.x);
            acc.y = fma(m[i * D + j].x, in[j].y, acc.y);
          } else {
            acc = cfma<R>(m[i * D + j], in[j], acc);
          }
        }
        r[o | dep4(i, MASK)] = acc;
      }
    }
  }
}

// KRON operator: register bit P carries its own 2x2 matrix (cf + 4P) when
// bit P of mask is set; its arithmetic form is 2 bits of `form`.
template <int NR, int P, class R>
__device__ __forceinline__ void kron_bit(typename Cplx<R>::T (&r)[NR], const typename Cplx<R>::T* cf, int mask,
                                         int form) {
  if constexpr ((1 << P) < NR) {
    if ((mask >> P) & 1) {
      const typename Cplx<R>::T* m = cf + 4 * P;
      const int f = (form >> (2 * P)) & 3;
      if (f == PD_XROT) phase_dense<NR, 1 << P, PD_XROT, R>(r, m);
      else if (f == PD_XROTU) phase_dense<NR, 1 << P, PD_XROTU, R>(r, m);
      else if (f == PD_REAL) phase_dense<NR, 1 << P, PD_REAL, R>(r, m);
      else phase_dense<NR, 1 << P, PD_GEN, R>(r, m);
    }
  }
}

__host__ __device__ constexpr int pext4(int v, int mask) {  // gather v's bits at mask positions
  int out = 0, bit = 0;
  for (int p = 0; p < 4; p++)
    if ((mask >> p) & 1) {
      if ((v >> p) & 1) out |= 1 << bit;
      bit++;
    }
  return out;
}

// Diagonal operator whose register-bit part is SU: factor of register
// element i is dg[pext(i, SU)] (compile-time offset; no integer work).
template <int NR, int SU, class R>
__device__ __forceinline__ void phase_diag(typename Cplx<R>::T (&r)[NR], const typename Cplx<R>::T* __restrict__ dg) {
  using C = typename Cplx<R>::T;
#pragma unroll
  for (int i = 0; i < NR; i++) {
    const C f = dg[pext4(i, SU)];
    r[i] = C{fma(f.x, r[i].x, -f.y * r[i].y), fma(f.x, r[i].y, f.y * r[i].x)};
  }
}

// Signed permutation on register bits MASK (k <= 2): integer moves only.
template <int NR, int MASK, class R>
__device__ __forceinline__ void phase_perm(typename Cplx<R>::T (&r)[NR], const uint8_t* perm) {
  using C = typename Cplx<R>::T;
  constexpr int K = popc4(MASK), D = 1 << K;
  uint8_t pm[D];
#pragma unroll
  for (int i = 0; i < D; i++) pm[i] = perm[i];
#pragma unroll
  for (int o = 0; o < NR; o++) {
    if (o & MASK) continue;
    C in[D];
#pragma unroll
    for (int j = 0; j < D; j++) in[j] = r[o | dep4(j, MASK)];
#pragma unroll
    for (int i = 0; i < D; i++) {
      C v = in[0];
#pragma unroll
      for (int j = 1; j < D; j++) v = ((pm[i] & 15) == j) ? in[j] : v;
      r[o | dep4(i, MASK)] = signed_base(v, (pm[i] & 0x80) ? 2 : 1);
    }
  }
}


template <class R, int RB, bool TBL>
__global__ void __launch_bounds__(kSweepThreads) phase_kernel(void* __restrict__ state_v, uint64_t ntiles, SweepDesc sd,
                                                              const PhaseDesc* __restrict__ ph_g,
                                                              const PhaseOp* __restrict__ po_g,
                                                              const void* __restrict__ pc_v) {
  using C = typename Cplx<R>::T;
  constexpr int NR = 1 << RB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int T = sd.T;
  const uint32_t PE = (uint32_t)padded_elems<C>(T);
  C* tile = reinterpret_cast<C*>(smem_raw);    // current tile (padded layout)
  C* ntile = tile + PE;                         // next tile, filled asynchronously
  const PhaseDesc* phases = ph_g + sd.ph0;
  const PhaseOp* pops = po_g + sd.pop0;
  const C* coefs = reinterpret_cast<const C*>(pc_v) + sd.pc0;
  if constexpr (TBL) {
    PhaseDesc* sph = reinterpret_cast<PhaseDesc*>(tile + 2 * PE);
    PhaseOp* spo = reinterpret_cast<PhaseOp*>(sph + sd.nph);  // 16-byte records: stays aligned
    C* sc = reinterpret_cast<C*>(spo + sd.npop);
    const uint4* a1 = reinterpret_cast<const uint4*>(phases);
    uint4* b1 = reinterpret_cast<uint4*>(sph);
    for (uint32_t v = threadIdx.x; v < sd.nph * (sizeof(PhaseDesc) / 16); v += kSweepThreads) b1[v] = a1[v];
    const uint4* a2 = reinterpret_cast<const uint4*>(pops);
    uint4* b2 = reinterpret_cast<uint4*>(spo);
    for (uint32_t v = threadIdx.x; v < sd.npop * (sizeof(PhaseOp) / 16); v += kSweepThreads) b2[v] = a2[v];
    for (uint32_t v = threadIdx.x; v < sd.npc; v += kSweepThreads) sc[v] = coefs[v];
    phases = sph;
    pops = spo;
    coefs = sc;
  }
  C* state = reinterpret_cast<C*>(state_v);
  constexpr int VPE = 16 / sizeof(C);
  const uint32_t nvec = (1u << T) / VPE;
  const int lvpc = sd.m - __ffs(VPE) + 1;
  const uint32_t vpc_mask = (1u << lvpc) - 1u;
  const uint32_t ngroups = 1u << (T - RB);
  // global offset of each strided chunk of the tile, computed once per CTA
  uint64_t* hoff = reinterpret_cast<uint64_t*>(smem_raw + phase_hoff_offset<C>(sd, TBL));
  for (uint32_t j = threadIdx.x; j < (1u << sd.h); j += kSweepThreads) hoff[j] = deposit(j, sd.hmask);
  __syncthreads();

  auto prefetch = [&](uint64_t tid, C* dst) {
    const uint64_t b = deposit(tid, sd.fmask);
    for (uint32_t v = threadIdx.x; v < nvec; v += kSweepThreads)
      cp_async16(dst + swz<C>(v * VPE), state + b + hoff[v >> lvpc] + (uint64_t)(v & vpc_mask) * VPE);
    cp_async_commit();
  };
  if (blockIdx.x < ntiles) prefetch(blockIdx.x, tile);
  for (uint64_t tileid = blockIdx.x; tileid < ntiles; tileid += gridDim.x) {
    const uint64_t base = deposit(tileid, sd.fmask);
    const uint64_t next = tileid + gridDim.x;
    if (next < ntiles) {
      prefetch(next, ntile);  // overlaps with the phases below
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    for (uint32_t ph = 0; ph < sd.nph; ph++) {
      const PhaseDesc P = phases[ph];
      uint32_t roff[NR];  // padded offset of register element i inside its group
#pragma unroll
      for (int i = 0; i < NR; i++) {
        uint32_t l = 0;
#pragma unroll
        for (int p = 0; p < RB; p++)
          if ((i >> p) & 1) l |= 1u << P.u[p];
        roff[i] = swz<C>(l);
      }
      const PhaseOp* pop = pops + (P.op0 - sd.pop0);
      for (uint32_t g = threadIdx.x; g < ngroups; g += kSweepThreads) {
        const uint32_t gb = insert_zeros<RB>(g, P.u);
        const C* gt = tile + swz<C>(gb);
        C r[NR];
#pragma unroll
        for (int i = 0; i < NR; i++) r[i] = gt[roff[i]];
        for (uint32_t q = 0; q < P.nops; q++) {
          const PhaseOp& o = pop[q];
          const C* cf = coefs + (o.coef - sd.pc0);
          const int code = o.code;
          if (code < 16) {  // diagonal: factor table offset by the out-of-register bits
            uint32_t ig = 0;
            const int dn = o.dnu;
            for (int t = 0; t < dn; t++) ig |= ((gb >> o.dpos[t]) & 1u) << t;
            cf += ig << popc4(code);
          }
          switch (code) {
#define NWQ_D(M) case M: if constexpr (M < NR) phase_diag<NR, M, R>(r, cf); break;
#define NWQ_P(M) case 16 + M: if constexpr (M < NR) phase_perm<NR, M, R>(r, o.perm); break;
#define NWQ_G(M) case 32 + M: if constexpr (M < NR) phase_dense<NR, M, PD_GEN, R>(r, cf); break;
#define NWQ_R(M) case 48 + M: if constexpr (M < NR) phase_dense<NR, M, PD_REAL, R>(r, cf); break;
#define NWQ_X(M) case 64 + M: if constexpr (M < NR) phase_dense<NR, M, PD_XROT, R>(r, cf); break;
            case PCODE_KRON:
              kron_bit<NR, 0, R>(r, cf, o.mask, o.form);
              kron_bit<NR, 1, R>(r, cf, o.mask, o.form);
              kron_bit<NR, 2, R>(r, cf, o.mask, o.form);
              kron_bit<NR, 3, R>(r, cf, o.mask, o.form);
              break;
            NWQ_D(0) NWQ_D(1) NWQ_D(2) NWQ_D(3) NWQ_D(4) NWQ_D(5) NWQ_D(6) NWQ_D(7)
            NWQ_D(8) NWQ_D(9) NWQ_D(10) NWQ_D(11) NWQ_D(12) NWQ_D(13) NWQ_D(14) NWQ_D(15)
            NWQ_P(1) NWQ_P(2) NWQ_P(4) NWQ_P(8) NWQ_P(3) NWQ_P(5) NWQ_P(6) NWQ_P(9) NWQ_P(10) NWQ_P(12)
            NWQ_G(1) NWQ_G(2) NWQ_G(4) NWQ_G(8) NWQ_G(3) NWQ_G(5) NWQ_G(6) NWQ_G(9) NWQ_G(10) NWQ_G(12)
            NWQ_R(1) NWQ_R(2) NWQ_R(4) NWQ_R(8) NWQ_R(3) NWQ_R(5) NWQ_R(6) NWQ_R(9) NWQ_R(10) NWQ_R(12)
            NWQ_X(1) NWQ_X(2) NWQ_X(4) NWQ_X(8)
#undef NWQ_D
#undef NWQ_P
#undef NWQ_G
#undef NWQ_R
#undef NWQ_X
            default: break;
          }
        }
        C* gw = tile + swz<C>(gb);
#pragma unroll
        for (int i = 0; i < NR; i++) gw[roff[i]] = r[i];
      }
      __syncthreads();
    }
    for (uint32_t v = threadIdx.x; v < nvec; v += kSweepThreads) {
      uint64_t off = base + hoff[v >> lvpc] + (uint64_t)(v & vpc_mask) * VPE;
      *reinterpret_cast<uint4*>(state + off) = *reinterpret_cast<const uint4*>(tile + swz<C>(v * VPE));
    }
    __syncthreads();  // the current tile is refilled by the prefetch of the next iteration
    C* t = tile;
    tile = ntile;
    ntile = t;
  }
  cp_async_wait<0>();
}

template <class R, int RB>
static cudaError_t launch_phase_t(void* state, int B, const SweepDesc& sd, const PhaseTables& pt, int sm_count,
                                  cudaStream_t s) {
  using C = typename Cplx<R>::T;
  size_t tile = 2 * sizeof(C) * padded_elems<C>(sd.T);  // current + prefetched tile
  size_t table = sd.nph * sizeof(PhaseDesc) + sd.npop * sizeof(PhaseOp) + sd.npc * sizeof(C);
  const bool tbl = tile + table <= (size_t)kTableSmemLimit;
  size_t smem = (tbl ? phase_hoff_offset<C>(sd, true) : phase_hoff_offset<C>(sd, false)) + ((size_t)8 << sd.h);
  static std::atomic<int> attr_dev[2] = {-1, -1};  // setting the same maximum twice is harmless
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev[tbl].load() != dev) {
    cudaError_t e = tbl ? cudaFuncSetAttribute(phase_kernel<R, RB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem)
                        : cudaFuncSetAttribute(phase_kernel<R, RB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e != cudaSuccess) return e;
    attr_dev[tbl] = dev;
  }
  uint64_t ntiles = 1ull << (B - sd.T);
  int per_sm = 0;
  cudaError_t e = tbl ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, phase_kernel<R, RB, true>, kSweepThreads, smem)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, phase_kernel<R, RB, false>, kSweepThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t grid = (uint64_t)sm_count * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (tbl) phase_kernel<R, RB, true><<<(unsigned)grid, kSweepThreads, smem, s>>>(state, ntiles, sd, pt.ph, pt.po, pt.pc);
  else phase_kernel<R, RB, false><<<(unsigned)grid, kSweepThreads, smem, s>>>(state, ntiles, sd, pt.ph, pt.po, pt.pc);
  g_launches += 1;
  return cudaGetLastError();
}

template <class R, bool CPLX, bool TBL>
static cudaError_t launch_sweep_tt(void* state, int B, const SweepDesc& sd, const DevOp* ops, const void* ents,
                                   size_t smem, int sm_count, cudaStream_t s) {
  static std::atomic<int> attr_dev{-1};  // per instantiation: the attribute is set once per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev.load() != dev) {
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<R, CPLX, TBL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxDynSmem);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  uint64_t ntiles = 1ull << (B - sd.T);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<R, CPLX, TBL>, kSweepThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t grid = (uint64_t)sm_count * per_sm;
  if (grid > ntiles) grid = ntiles;
  sweep_kernel<R, CPLX, TBL><<<(unsigned)grid, kSweepThreads, smem, s>>>(state, ntiles, sd, ops, ents);
  g_launches += 1;
  return cudaGetLastError();
}

template <class R, bool CPLX>
static cudaError_t launch_sweep_t(void* state, int B, const SweepDesc& sd, const DevOp* ops, const void* ents,
                                  int sm_count, cudaStream_t s) {
  using E = ElemT<R, CPLX>;
  using Ent = EntT<R, CPLX>;
  size_t tiles = 2 * (sizeof(E) << sd.T);
  size_t table = sd.nops * sizeof(DevOp) + sd.nent * sizeof(Ent);
  size_t hbytes = (size_t)8 << sd.h;
  if (tiles + table <= (size_t)kTableSmemLimit)
    return launch_sweep_tt<R, CPLX, true>(state, B, sd, ops, ents,
                                          hoff_offset(sd, 2 * sizeof(E), true, table) + hbytes, sm_count, s);
  return launch_sweep_tt<R, CPLX, false>(state, B, sd, ops, ents, hoff_offset(sd, 2 * sizeof(E), false, 0) + hbytes,
                                         sm_count, s);
}

cudaError_t launch_sweep(bool cplx, bool f64, void* state, int B, const SweepDesc& sd, const DevOp* ops,
                         const void* ents, const PhaseTables* pt, int sm_count, cudaStream_t s) {
  if (cplx && pt && sd.nph > 0) {  // the register-group width is fixed by the plan (SweepDesc::prb)
    if (f64) return sd.prb == 4 ? launch_phase_t<double, 4>(state, B, sd, *pt, sm_count, s)
                                : launch_phase_t<double, 3>(state, B, sd, *pt, sm_count, s);
    return sd.prb == 3 ? launch_phase_t<float, 3>(state, B, sd, *pt, sm_count, s)
                       : launch_phase_t<float, 4>(state, B, sd, *pt, sm_count, s);
  }
  if (cplx) {
    if (f64) return launch_sweep_t<double, true>(state, B, sd, ops, ents, sm_count, s);
    return launch_sweep_t<float, true>(state, B, sd, ops, ents, sm_count, s);
  }
  if (f64) return launch_sweep_t<double, false>(state, B, sd, ops, ents, sm_count, s);
  return launch_sweep_t<float, false>(state, B, sd, ops, ents, sm_count, s);
}

// ------------------------------------------------------------------ init
// SV: psi = |0..0>.  DM (Pauli basis): r[x + 2^n z] = Tr(|0><0| P(x,z)) = [x == 0].
template <class R>
__global__ void init_kernel(R* __restrict__ s, uint64_t count, uint64_t xmask, int cplx, R one) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    R v = 0;
    if (cplx) {
      v = (i == 0) ? one : R(0);
    } else {
      v = ((i & xmask) == 0) ? one : R(0);
    }
    s[i] = v;
  }
}

cudaError_t launch_init(bool cplx, bool f64, void* state, int n, int sm_count, cudaStream_t s, bool dw) {
  // SV: 2^n complex = 2^(n+1) reals, only real[0] = 1.  DM: 4^n reals, 1 where x = 0.  dw
  // (FP64): the double-word layout, each 1 as the float pair (1, 0) in its 8 bytes.
  uint64_t count = cplx ? (2ull << n) : (1ull << (2 * n));
  uint64_t xmask = (1ull << n) - 1;
  unsigned grid = (unsigned)std::min<uint64_t>((count + 255) / 256, (uint64_t)sm_count * 8);
  uint64_t one_bits = 0x3ff0000000000000ull;  // 1.0
  if (dw) one_bits = 0x3f800000ull;  // h = 1.0f (IEEE bits), l = 0
  double one;
  std::memcpy(&one, &one_bits, 8);
  if (f64) init_kernel<double><<<grid, 256, 0, s>>>((double*)state, count, xmask, cplx, one);
  else init_kernel<float><<<grid, 256, 0, s>>>((float*)state, count, xmask, cplx, 1.0f);
  g_launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ double words
// In place, pairs of doubles: to_dw turns each double v into the float pair
// (h, l) in the same 8 bytes by integer operations (GB300 runs FP64 <-> FP32
// conversions on its FP64 pipe): h keeps the top 24 significant bits of v,
// l the next 23, rounded, so |v - h - l| <= 2^-47 |v|; magnitudes below
// 2^-103 become 0.  Back, each pair becomes the double h + l.
__device__ __forceinline__ float2 dw_split_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
  const unsigned e = (hi32 >> 20) & 0x7ffu;  // biased exponent
  // h: exponent rebiased 1023 -> 127, the top 23 fraction bits
  const unsigned hb = (hi32 & 0x80000000u) | (__funnelshift_l(lo32, hi32 - (896u << 20), 3) & 0x7fffffffu);
  // l: the other 29 fraction bits r (value r 2^(E-52)) as (2^(E-23) + q 2^(E-46)) - 2^(E-23),
  // q = r / 64 rounded (at most 2^23), exact by Sterbenz's lemma
  const unsigned mb = (hb & 0xff800000u) - (23u << 23);
  const unsigned q = ((lo32 & 0x1fffffffu) + 32u) >> 6;
  const float l = __fsub_rn(__int_as_float((int)(mb + q)), __int_as_float((int)mb));
  if (e < 920u) return make_float2(0.f, 0.f);  // |x| < 2^-103
  if (e > 1150u) return make_float2(__int_as_float((int)((hi32 & 0x80000000u) | 0x7f800000u)), 0.f);
  return make_float2(__int_as_float((int)hb), l);
}

// mode 1: FP64 -> double words; 0: back; 2: double words renormalised in place
// (TwoSum of each pair, exact: the sweeps' multiply-adds leave the low parts
// unnormalised, and a state kept in the double-word layout over several runs
// is renormalised before the next one).
__device__ __forceinline__ float2 dw_renorm_pair(float h, float l) {
  const float s = __fadd_rn(h, l);
  const float v = __fsub_rn(s, h);
  return make_float2(s, __fadd_rn(__fsub_rn(h, __fsub_rn(s, v)), __fsub_rn(l, v)));
}

__global__ void dw_convert_kernel(void* __restrict__ data, uint64_t npairs, int to_dw) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < npairs; i += (uint64_t)gridDim.x * blockDim.x) {
    if (to_dw == 2) {
      const float4 f = reinterpret_cast<const float4*>(data)[i];
      const float2 a = dw_renorm_pair(f.x, f.y), c = dw_renorm_pair(f.z, f.w);
      reinterpret_cast<float4*>(data)[i] = make_float4(a.x, a.y, c.x, c.y);
    } else if (to_dw) {
      const double2 d = reinterpret_cast<const double2*>(data)[i];
      const float2 a = dw_split_bits(d.x), c = dw_split_bits(d.y);
      reinterpret_cast<float4*>(data)[i] = make_float4(a.x, a.y, c.x, c.y);
    } else {
      const float4 f = reinterpret_cast<const float4*>(data)[i];
      reinterpret_cast<double2*>(data)[i] = make_double2((double)f.x + (double)f.y, (double)f.z + (double)f.w);
    }
  }
}

cudaError_t launch_dw_renormalize(void* data, uint64_t ndouble, int sm_count, cudaStream_t s) {
  const uint64_t npairs = ndouble / 2;
  unsigned grid = (unsigned)std::min<uint64_t>((npairs + 255) / 256, (uint64_t)sm_count * 8);
  if (grid == 0) return cudaSuccess;
  dw_convert_kernel<<<grid, 256, 0, s>>>(data, npairs, 2);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_dw_convert(void* data, uint64_t ndouble, bool to_dw, int sm_count, cudaStream_t s) {
  const uint64_t npairs = ndouble / 2;
  unsigned grid = (unsigned)std::min<uint64_t>((npairs + 255) / 256, (uint64_t)sm_count * 8);
  if (grid == 0) return cudaSuccess;
  dw_convert_kernel<<<grid, 256, 0, s>>>(data, npairs, to_dw ? 1 : 0);
  g_launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ conversions
// Pauli reals -> complex (imag 0) and complex -> real parts.
template <class R>
__global__ void real_to_cplx(const R* __restrict__ in, typename Cplx<R>::T* __restrict__ out, uint64_t count) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = typename Cplx<R>::T{in[i], R(0)};
}
template <class R>
__global__ void cplx_to_real(const typename Cplx<R>::T* __restrict__ in, R* __restrict__ out, uint64_t count) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = in[i].x;
}

cudaError_t launch_real_to_cplx(bool f64, const void* in, void* out, uint64_t count, int sm_count, cudaStream_t s) {
  unsigned grid = (unsigned)std::min<uint64_t>((count + 255) / 256, (uint64_t)sm_count * 8);
  if (f64) real_to_cplx<double><<<grid, 256, 0, s>>>((const double*)in, (double2*)out, count);
  else real_to_cplx<float><<<grid, 256, 0, s>>>((const float*)in, (float2*)out, count);
  g_launches += 1;
  return cudaGetLastError();
}
cudaError_t launch_cplx_to_real(bool f64, const void* in, void* out, uint64_t count, int sm_count, cudaStream_t s) {
  unsigned grid = (unsigned)std::min<uint64_t>((count + 255) / 256, (uint64_t)sm_count * 8);
  if (f64) cplx_to_real<double><<<grid, 256, 0, s>>>((const double2*)in, (double*)out, count);
  else cplx_to_real<float><<<grid, 256, 0, s>>>((const float2*)in, (float*)out, count);
  g_launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ probabilities
// SV: p[b] = |psi_b|^2 in FP64.
template <class R>
__global__ void sv_abs2(const typename Cplx<R>::T* __restrict__ psi, double* __restrict__ p, uint64_t count) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    double re = psi[i].x, im = psi[i].y;
    p[i] = fma(re, re, im * im);
  }
}
// Pauli coefficient i as FP64: from FP64 / FP32 storage, or (DW) from the float
// pair h + l of a density matrix left in the double-word layout.
template <class R, bool DW>
__device__ __forceinline__ double coef_at(const R* __restrict__ r, uint64_t i) {
  if constexpr (DW) {
    const float2 v = reinterpret_cast<const float2*>(r)[i];
    return (double)v.x + (double)v.y;
  } else {
    return (double)r[i];
  }
}

// DM: g[z] = r[z << n] (1 - 2e)^{|z|} / 2^n ; a Walsh-Hadamard transform of g
// over n bits then gives the outcome distribution with readout error e.
template <class R, bool DW>
__global__ void dm_diag_gather(const R* __restrict__ r, double* __restrict__ g, int n, double one_m_2e) {
  uint64_t N = 1ull << n;
  double scale = ldexp(1.0, -n);
  for (uint64_t z = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; z < N; z += (uint64_t)gridDim.x * blockDim.x) {
    int w = __popcll(z);
    double f = scale;
    double b = one_m_2e;
    // (1-2e)^w by binary powering in FP64 (w <= 16)
    while (w) {
      if (w & 1) f *= b;
      b *= b;
      w >>= 1;
    }
    g[z] = coef_at<R, DW>(r, z << n) * f;
  }
}

cudaError_t launch_sv_abs2(bool f64, const void* psi, double* p, uint64_t count, int sm_count, cudaStream_t s) {
  unsigned grid = (unsigned)std::min<uint64_t>((count + 255) / 256, (uint64_t)sm_count * 8);
  if (f64) sv_abs2<double><<<grid, 256, 0, s>>>((const double2*)psi, p, count);
  else sv_abs2<float><<<grid, 256, 0, s>>>((const float2*)psi, p, count);
  g_launches += 1;
  return cudaGetLastError();
}
cudaError_t launch_dm_diag(bool f64, const void* r, double* g, int n, double e, int sm_count, cudaStream_t s, bool dw) {
  uint64_t count = 1ull << n;
  unsigned grid = (unsigned)std::min<uint64_t>((count + 255) / 256, (uint64_t)sm_count * 8);
  if (f64 && dw) dm_diag_gather<double, true><<<grid, 256, 0, s>>>((const double*)r, g, n, 1.0 - 2.0 * e);
  else if (f64) dm_diag_gather<double, false><<<grid, 256, 0, s>>>((const double*)r, g, n, 1.0 - 2.0 * e);
  else dm_diag_gather<float, false><<<grid, 256, 0, s>>>((const float*)r, g, n, 1.0 - 2.0 * e);
  g_launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ DM expectations
template <class R, bool DW>
__global__ void dm_expect_gather(const R* __restrict__ r, int n, const uint64_t* __restrict__ xm,
                                 const uint64_t* __restrict__ zm, const double* __restrict__ coef, int nt,
                                 double* __restrict__ out, int sum, int normalize) {
  const double tr = normalize ? coef_at<R, DW>(r, 0) : 1.0;  // Tr(rho) = coefficient of the identity string
  if (sum) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      double acc = 0;
      for (int t = 0; t < nt; t++) acc = fma(coef[t], coef_at<R, DW>(r, xm[t] | (zm[t] << n)), acc);
      out[0] = acc / tr;
    }
    return;
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x)
    out[t] = coef_at<R, DW>(r, xm[t] | (zm[t] << n)) / tr;
}

__global__ void weighted_sum(const double* __restrict__ v, const double* __restrict__ coef, int nt,
                             double* __restrict__ out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double acc = 0;
    for (int t = 0; t < nt; t++) acc = fma(coef[t], v[t], acc);
    out[0] = acc;
  }
}

cudaError_t launch_dm_expect(bool f64, const void* r, int n, const uint64_t* xm, const uint64_t* zm,
                             const double* coef, int nt, double* out, int sum, int normalize, cudaStream_t s, bool dw) {
  int grid = sum ? 1 : (nt + 255) / 256;
  if (f64 && dw)
    dm_expect_gather<double, true><<<grid, 256, 0, s>>>((const double*)r, n, xm, zm, coef, nt, out, sum, normalize);
  else if (f64)
    dm_expect_gather<double, false><<<grid, 256, 0, s>>>((const double*)r, n, xm, zm, coef, nt, out, sum, normalize);
  else
    dm_expect_gather<float, false><<<grid, 256, 0, s>>>((const float*)r, n, xm, zm, coef, nt, out, sum, normalize);
  g_launches += 1;
  return cudaGetLastError();
}

__global__ void scale_values(double* __restrict__ v, int nt, const double* __restrict__ denom) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nt) v[t] = v[t] / denom[0];
}

cudaError_t launch_scale(double* v, int nt, const double* denom, cudaStream_t s) {
  scale_values<<<(nt + 127) / 128, 128, 0, s>>>(v, nt, denom);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_weighted_sum(const double* v, const double* coef, int nt, double* out, cudaStream_t s) {
  weighted_sum<<<1, 32, 0, s>>>(v, coef, nt, out);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace nwq
