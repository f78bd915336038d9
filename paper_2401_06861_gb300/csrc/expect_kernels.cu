// Pauli-string expectations of a state vector (paper Sec. III: VQE energies
// and observables are weighted sums of Pauli-string expectations).
//
//   <psi| P(x, z) |psi> = sum_b Re( conj(psi[b ^ x]) i^y (-1)^{|b & z|} psi[b] ),
//   y = |x & z| mod 4 (one factor i per Y).
//
// sv_expect_tiled: one launch per pass.  A pass stages tiles of 2^T
// amplitudes (2^m contiguous elements x 2^(T-m) strided chunks at the pass's
// high bit positions) in shared memory, and evaluates every term whose X
// support lies inside the tile's bits: the partner psi[b ^ x] of each element
// is then in the same tile, so one read of the state serves all those terms.
// Each thread keeps |psi|^2 of its E = 2^T / 128 elements in registers for the
// diagonal (Z-type) terms; off-diagonal terms read both amplitudes from shared
// memory.  The sign of element j is bit j of a per-term word built with one
// warp ballot, so the inner loops carry no population counts.
//
// Precision: products and sums over one warp's 32 x E elements are taken in
// the state's precision, everything above (per warp across tiles, per block,
// across blocks) in FP64.  Per-block sums go to part[block * ncols + column];
// reduce_partials adds the blocks in order, so results are deterministic.
//
// sv_expect_group: the general kernel for terms whose X support does not fit
// a tile: one pass per group of at most kExpectChunk terms sharing x, each
// thread reading psi[b] and psi[b ^ x] from global memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>

#include "dw.cuh"
#include "nwq_internal.h"
#include "kernels.hpp"
#include "device_util.cuh"

namespace nwq {

namespace {

// Flip the sign of v when s = 0x80000000 (s = 0: unchanged).
__device__ __forceinline__ float flip_sign(float v, uint32_t s) { return __int_as_float(__float_as_int(v) ^ (int)s); }
__device__ __forceinline__ double flip_sign(double v, uint32_t s) {
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)((unsigned long long)s << 32));
}

template <class R, int E>
__global__ void __launch_bounds__(kExpThreads) sv_expect_tiled(const typename Cplx<R>::T* __restrict__ psi,
                                                               uint64_t ntiles, ExpPass P,
                                                               const ExpTerm* __restrict__ terms,
                                                               double* __restrict__ part, int ncols) {
  using C = typename Cplx<R>::T;
  constexpr int VPE = 16 / sizeof(C);  // elements per 16-byte vector
  constexpr int kLogVPE = VPE == 2 ? 1 : 0;
  constexpr int kWarps = kExpThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t nel = 1u << P.T;
  C* tile = reinterpret_cast<C*>(smem_raw);
  uint64_t* hoff = reinterpret_cast<uint64_t*>(smem_raw + sizeof(C) * (size_t)nel);
  ExpTerm* st = reinterpret_cast<ExpTerm*>(hoff + (1u << P.h));
  double* red = reinterpret_cast<double*>(st + P.nk);  // [warp][term] FP64 sums
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int i = tid; i < P.nk; i += kExpThreads) st[i] = terms[P.k0 + i];
  for (uint32_t j = tid; j < (1u << P.h); j += kExpThreads) hoff[j] = deposit(j, P.hmask);
  for (int i = tid; i < kWarps * P.nk; i += kExpThreads) red[i] = 0.0;
  const uint32_t lowmask = (1u << P.m) - 1u;

  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = deposit(t, P.fmask);
    __syncthreads();  // tables staged; previous tile consumed
    if (P.m >= kLogVPE) {  // 16-byte vectors along the contiguous low bits
      for (uint32_t v = tid; v < nel / VPE; v += kExpThreads) {
        const uint32_t l = v * VPE;
        cp_async16(tile + l, psi + base + hoff[l >> P.m] + (l & lowmask));
      }
      cp_async_commit();
      cp_async_wait<0>();
    } else {
      for (uint32_t l = tid; l < nel; l += kExpThreads) tile[l] = psi[base + hoff[l >> P.m] + (l & lowmask)];
    }
    __syncthreads();

    R p[E];
#pragma unroll
    for (int j = 0; j < E; j++) {
      const uint32_t l = tid + kExpThreads * j;
      C a = tile[l < nel ? l : 0];
      p[j] = (l < nel) ? a.x * a.x + a.y * a.y : R(0);
    }
    for (int k = 0; k < P.nk; k++) {
      const ExpTerm tm = st[k];
      // bit j of W: sign of element tid + 128 j, i.e. parity of its bits in
      // z (tile-local and the tile's base) plus the sign of i^y (y = 1, 2).
      const uint32_t hi = (uint32_t)__popc((uint32_t)lane & (tm.zl >> 7)) & 1u;
      uint32_t W = __ballot_sync(0xffffffffu, hi);
      const uint32_t flip = ((uint32_t)__popc((uint32_t)tid & tm.zl & 127u) + (uint32_t)__popcll(base & tm.zh) +
                             (uint32_t)(tm.y == 1 || tm.y == 2)) & 1u;
      W ^= 0u - flip;
      R a = R(0);
      if (tm.xl == 0) {
#pragma unroll
        for (int j = 0; j < E; j++) a += flip_sign(p[j], (W << (31 - j)) & 0x80000000u);
      } else if ((tm.y & 1) == 0) {  // Re(conj(q) s)
#pragma unroll
        for (int j = 0; j < E; j++) {
          const uint32_t l = tid + kExpThreads * j;
          if (E > 1 || l < nel) {
            const C s = tile[l], q = tile[l ^ tm.xl];
            a += flip_sign(fma(q.x, s.x, q.y * s.y), (W << (31 - j)) & 0x80000000u);
          }
        }
      } else {  // Im(conj(q) s)
#pragma unroll
        for (int j = 0; j < E; j++) {
          const uint32_t l = tid + kExpThreads * j;
          if (E > 1 || l < nel) {
            const C s = tile[l], q = tile[l ^ tm.xl];
            a += flip_sign(fma(q.x, s.y, -q.y * s.x), (W << (31 - j)) & 0x80000000u);
          }
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) red[warp * P.nk + k] += (double)a;
    }
  }
  __syncthreads();
  for (int k = tid; k < P.nk; k += kExpThreads) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) v += red[w * P.nk + k];
    part[(size_t)blockIdx.x * ncols + st[k].out] = v;
  }
}

// ------------------------------------------------------------------ double words
// Complex128 passes with full tiles (2^12 amplitudes, 32 per thread): the
// same passes, products and per-warp sums in double-word arithmetic on the
// FP32 pipe (GB300 issues FP32 at 64 times its FP64 rate).  Each thread splits
// its own 32 amplitudes in shared memory into float pairs by integer
// operations (h = the top 24 significant bits, l = the next 23, rounded:
// |x - h - l| <= 2^-47 |x|; magnitudes below 2^-103 become 0), forms each
// product with an exact FMA-based product (Dekker) plus cross terms, and adds
// the signed products into a compensated float pair (Knuth's TwoSum on the
// running sum, the rounding errors and low parts collected separately).  The
// warp's pairs are added the same way across lanes and lane 0 adds the pair,
// converted to FP64, into the FP64 per-warp sums, as in sv_expect_tiled.
template <int E>
__global__ void __launch_bounds__(kExpThreads) sv_expect_tiled_dw(const double2* __restrict__ psi, uint64_t ntiles,
                                                                  ExpPass P, const ExpTerm* __restrict__ terms,
                                                                  double* __restrict__ part, int ncols) {
  constexpr int kWarps = kExpThreads / 32;
  constexpr int kGrp = 8;  // terms per warp reduce-scatter
  static_assert(E == 32, "full 2^12 tiles");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t nel = 1u << P.T;
  double2* tile = reinterpret_cast<double2*>(smem_raw);
  float4* tw = reinterpret_cast<float4*>(smem_raw);  // the same tile as double words (re.h, re.l, im.h, im.l)
  uint64_t* hoff = reinterpret_cast<uint64_t*>(smem_raw + sizeof(double2) * (size_t)nel);
  ExpTerm* st = reinterpret_cast<ExpTerm*>(hoff + (1u << P.h));
  double* red = reinterpret_cast<double*>(st + P.nk);  // [warp][term] FP64 sums
  float2* wht = reinterpret_cast<float2*>(red + kWarps * P.nk);  // [k][thread] transforms (8-byte aligned)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // a pass with a Z-type string (diagonal: read from the probabilities) has the transform
  // buffer; the host sets P.zt exactly when a term of the pass has xl = 0
  const bool zterm = P.zt != 0;
  for (int i = tid; i < P.nk; i += kExpThreads) st[i] = terms[P.k0 + i];
  for (uint32_t j = tid; j < (1u << P.h); j += kExpThreads) hoff[j] = deposit(j, P.hmask);
  for (int i = tid; i < kWarps * P.nk; i += kExpThreads) red[i] = 0.0;
  const uint32_t lowmask = (1u << P.m) - 1u;
  __syncthreads();

  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = deposit(t, P.fmask);
    __syncthreads();  // tables staged; previous tile consumed
    // each thread copies, then splits, its own 32 amplitudes tid + 128 j
#pragma unroll
    for (int j = 0; j < E; j++) {
      const uint32_t l = tid + kExpThreads * j;
      cp_async16(tile + l, psi + base + hoff[l >> P.m] + (l & lowmask));
    }
    cp_async_commit();
    cp_async_wait<0>();
    if (zterm) {
      Dw p[E];
#pragma unroll
      for (int j = 0; j < E; j++) {
        const uint32_t l = tid + kExpThreads * j;
        Dw x, y;
        if (P.dwin) {  // the state already holds float pairs: renormalised (exactly) in place
          const float4 v = tw[l];
          x = dw_norm(v.x, v.y);
          y = dw_norm(v.z, v.w);
          tw[l] = make_float4(x.h, x.l, y.h, y.l);
        } else {
          const double2 a = tile[l];
          x = dw_split(a.x);
          y = dw_split(a.y);
          tw[l] = make_float4(x.h, x.l, y.h, y.l);
        }
        p[j] = dw_fma(y, y, dw_mul(x, x));
      }
      // Z-type strings: element l = tid + 128 j has sign (-1)^{|tid & zl| + |j & (zl >> 7)|}, so a
      // thread's signed sum over its 32 probabilities is +- entry (zl >> 7) of their Walsh-Hadamard
      // transform W[k] = sum_j (-1)^{|j & k|} p_j: one transform serves every Z-type string
#pragma unroll
      for (int b = 1; b < E; b <<= 1) {
#pragma unroll
        for (int j = 0; j < E; j++) {
          if (j & b) continue;
          const Dw a0 = p[j], a1 = p[j | b];
          p[j] = dw_add(a0, a1);
          p[j | b] = dw_add(a0, Dw{-a1.h, -a1.l});
        }
      }
#pragma unroll
      for (int j = 0; j < E; j++) wht[j * kExpThreads + tid] = make_float2(p[j].h, p[j].l);
    } else if (P.dwin) {  // only X-type strings: the resident pairs renormalised in place
#pragma unroll
      for (int j = 0; j < E; j++) {
        const uint32_t l = tid + kExpThreads * j;
        const float4 v = tw[l];
        const Dw x = dw_norm(v.x, v.y), y = dw_norm(v.z, v.w);
        tw[l] = make_float4(x.h, x.l, y.h, y.l);
      }
    } else {  // only X-type strings in this pass: the split amplitudes alone
#pragma unroll
      for (int j = 0; j < E; j++) {
        const uint32_t l = tid + kExpThreads * j;
        const double2 a = tile[l];
        const Dw x = dw_split(a.x), y = dw_split(a.y);
        tw[l] = make_float4(x.h, x.l, y.h, y.l);
      }
    }
    __syncthreads();

    // Terms in groups of kGrp: each thread forms its compensated pair (s, c) for every term of
    // the group, then one reduce-scatter across the warp (halving the values held per lane at
    // lane offsets 16, 8, 4, then two butterfly levels) leaves the warp's sum of term
    // g = (lane >> 2) in lanes 4g .. 4g + 3.
    for (int k0 = 0; k0 < P.nk; k0 += kGrp) {
      float gs[kGrp], gc[kGrp];
#pragma unroll
      for (int g = 0; g < kGrp; g++) {
        float as = 0.f, ac = 0.f;
        if (k0 + g < P.nk) {
          const ExpTerm tm = st[k0 + g];
          const uint32_t flip = ((uint32_t)__popcll(base & tm.zh) + (uint32_t)(tm.y == 1 || tm.y == 2)) & 1u;
          if (tm.xl == 0) {
            if (zterm) {  // always: P.zt covers every Z-type string of the pass
              const float2 w = wht[((tm.zl >> 7) & 31u) * kExpThreads + tid];
              const uint32_t sg = ((((uint32_t)__popc((uint32_t)tid & tm.zl & 127u)) ^ flip) & 1u) << 31;
              as = __int_as_float(__float_as_int(w.x) ^ (int)sg);
              ac = __int_as_float(__float_as_int(w.y) ^ (int)sg);
            }
          } else if (tm.zl == 0 && (tm.xl & (tm.xl - 1)) == 0) {
            // one X qubit in the tile and no Z bit there (so y = 0): every pair (l, l + xl), l
            // with bit xl clear, carries the term's sign, applied once; l = kk with a zero
            // inserted at bit xl, i.e. kk + (kk & ~(xl - 1))
            const uint32_t nlo = ~(tm.xl - 1u);
#pragma unroll 4
            for (int m = 0; m < E / 2; m++) {
              const uint32_t kk = tid + kExpThreads * m;
              const uint32_t l = kk + (kk & nlo);
              const float4 sv = tw[l], qv = tw[l + tm.xl];
              dw_acc_prod2(as, ac, Dw{qv.x, qv.y}, Dw{sv.x, sv.y}, Dw{qv.z, qv.w}, Dw{sv.z, sv.w});
            }
            const int sg = (int)(flip << 31);
            as = __int_as_float(__float_as_int(__fmul_rn(as, 2.f)) ^ sg);  // twice each pair, exact
            ac = __int_as_float(__float_as_int(__fmul_rn(ac, 2.f)) ^ sg);
          } else {
            // each pair (l, l ^ xl) once, l with the lowest bit of xl clear: the partner's
            // product is the same value (Re part for even y, Im part for odd y), so the pair
            // contributes twice the value of its first member
            const int pb = __ffs(tm.xl) - 1;
            const uint32_t lo = (1u << pb) - 1u;
            const bool im = (tm.y & 1) != 0;
#pragma unroll 4
            for (int m = 0; m < E / 2; m++) {
              const uint32_t kk = tid + kExpThreads * m;
              const uint32_t l = ((kk & ~lo) << 1) | (kk & lo);
              const float4 sv = tw[l], qv = tw[l ^ tm.xl];
              // w = a1 b1 + a2 b2: Re (qr sr + qi si) or Im (qr si - qi sr) of conj(q) s, the
              // sign of the term folded into a1 and a2 (exact)
              const uint32_t sg = ((((uint32_t)__popc(l & tm.zl)) ^ flip) & 1u) << 31;
              const uint32_t sg2 = im ? sg ^ 0x80000000u : sg;
              const Dw a1{__int_as_float(__float_as_int(qv.x) ^ (int)sg), __int_as_float(__float_as_int(qv.y) ^ (int)sg)};
              const Dw a2{__int_as_float(__float_as_int(qv.z) ^ (int)sg2), __int_as_float(__float_as_int(qv.w) ^ (int)sg2)};
              const Dw b1 = im ? Dw{sv.z, sv.w} : Dw{sv.x, sv.y}, b2 = im ? Dw{sv.x, sv.y} : Dw{sv.z, sv.w};
              dw_acc_prod2(as, ac, a1, b1, a2, b2);
            }
            as = __fmul_rn(as, 2.f);  // exact
            ac = __fmul_rn(ac, 2.f);
          }
        }
        gs[g] = as;
        gc[g] = ac;
      }
#pragma unroll
      for (int half = kGrp / 2, o = 16; half >= 1; half >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;  // keep the upper half of the values
#pragma unroll
        for (int j = 0; j < half; j++) {
          const float ks = up ? gs[j + half] : gs[j], kc = up ? gc[j + half] : gc[j];
          const float ss = up ? gs[j] : gs[j + half], sc = up ? gc[j] : gc[j + half];
          const float rs = __shfl_xor_sync(0xffffffffu, ss, o), rc = __shfl_xor_sync(0xffffffffu, sc, o);
          gs[j] = ks;
          gc[j] = kc;
          dw_acc(gs[j], gc[j], Dw{rs, rc}, 0u);
        }
      }
#pragma unroll
      for (int o = 2; o; o >>= 1) {
        const float rs = __shfl_xor_sync(0xffffffffu, gs[0], o), rc = __shfl_xor_sync(0xffffffffu, gc[0], o);
        dw_acc(gs[0], gc[0], Dw{rs, rc}, 0u);
      }
      const int k = k0 + (lane >> 2);
      if ((lane & 3) == 0 && k < P.nk) red[warp * P.nk + k] += (double)gs[0] + (double)gc[0];
    }
  }
  __syncthreads();
  for (int k = tid; k < P.nk; k += kExpThreads) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) v += red[w * P.nk + k];
    part[(size_t)blockIdx.x * ncols + st[k].out] = v;
  }
}

// One group of terms sharing x; per-block partial sums to part[block * nt + t].
template <class R>
__global__ void __launch_bounds__(256) sv_expect_group(const typename Cplx<R>::T* __restrict__ psi, uint64_t N,
                                                       uint64_t x, const uint64_t* __restrict__ zm,
                                                       const int* __restrict__ ym, int nt,
                                                       double* __restrict__ part) {
  double acc[kExpectChunk];
#pragma unroll
  for (int t = 0; t < kExpectChunk; t++) acc[t] = 0.0;
  for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < N; b += (uint64_t)gridDim.x * blockDim.x) {
    double pr = psi[b].x, pi = psi[b].y;
    double qr = pr, qi = pi;
    if (x) {
      qr = psi[b ^ x].x;
      qi = psi[b ^ x].y;
    }
    // w = conj(q) * p
    double wr = fma(qr, pr, qi * pi);
    double wi = fma(qr, pi, -qi * pr);
#pragma unroll
    for (int t = 0; t < kExpectChunk; t++) {
      if (t < nt) {
        // Re(i^y w): y=0 wr, y=1 -wi, y=2 -wr, y=3 wi
        int y = ym[t];
        double v = (y & 1) ? wi : wr;
        int neg = ((y == 1) || (y == 2)) ^ (__popcll(b & zm[t]) & 1);
        acc[t] += neg ? -v : v;
      }
    }
  }
  __shared__ double red[kExpectChunk][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < kExpectChunk; t++) {
    if (t >= nt) break;
    double v = acc[t];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[t][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < nt) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[threadIdx.x][w];
    part[(size_t)blockIdx.x * nt + threadIdx.x] = v;
  }
}

// out[idx ? idx[t] : t] = sum over blocks (in order) of part[block * nt + t].
__global__ void reduce_partials(const double* __restrict__ part, int nblocks, int nt, const int* __restrict__ idx,
                                double* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double v = 0;
  for (int b = 0; b < nblocks; b++) v += part[(size_t)b * nt + t];
  out[idx ? idx[t] : t] = v;
}

// A pass launches at most the CTAs that fit on the device at once (its tiles
// are taken by a grid-stride loop), so a pass whose shared memory allows
// fewer CTAs per SM than the call's grid assumes runs no second wave.
int fit_grid(const void* fn, int grid, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kExpThreads, smem) != cudaSuccess || per_sm < 1)
    return grid;
  return std::min(grid, per_sm * sms);
}

template <class R, int E>
cudaError_t launch_tiled_e(const void* psi, uint64_t ntiles, const ExpPass& P, const ExpTerm* terms, double* part,
                           int ncols, int grid, size_t smem, cudaStream_t s) {
  using C = typename Cplx<R>::T;
  static std::atomic<int> attr_dev{-1};  // setting the same maximum twice is harmless
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev.load() != dev) {
    cudaError_t e = cudaFuncSetAttribute(sv_expect_tiled<R, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxDynSmem);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  grid = fit_grid((const void*)sv_expect_tiled<R, E>, grid, smem);
  sv_expect_tiled<R, E><<<grid, kExpThreads, smem, s>>>((const C*)psi, ntiles, P, terms, part, ncols);
  return cudaGetLastError();
}


constexpr size_t kDwWhtBytes = 32 * kExpThreads * sizeof(float2);  // per-thread transforms of sv_expect_tiled_dw

cudaError_t launch_tiled_dw(const void* psi, uint64_t ntiles, const ExpPass& P, const ExpTerm* terms, double* part,
                            int ncols, int grid, size_t smem, cudaStream_t s) {
  if (P.zt) smem += kDwWhtBytes;  // passes of X-type strings only take no transform buffer (3 CTAs per SM)
  static std::atomic<int> attr_dev{-1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev.load() != dev) {
    cudaError_t e = cudaFuncSetAttribute(sv_expect_tiled_dw<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxDynSmem);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  grid = fit_grid((const void*)sv_expect_tiled_dw<32>, grid, smem);
  sv_expect_tiled_dw<32><<<grid, kExpThreads, smem, s>>>((const double2*)psi, ntiles, P, terms, part, ncols);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_tiled_r(const void* psi, uint64_t ntiles, const ExpPass& P, const ExpTerm* terms, double* part,
                           int ncols, int grid, size_t smem, cudaStream_t s) {
  if (sizeof(R) == 8 && P.T == 12 && (P.dwin || !expect_fp64_only()))
    return launch_tiled_dw(psi, ntiles, P, terms, part, ncols, grid, smem, s);
  switch (P.T <= 7 ? 0 : P.T - 7) {
    case 0: return launch_tiled_e<R, 1>(psi, ntiles, P, terms, part, ncols, grid, smem, s);
    case 1: return launch_tiled_e<R, 2>(psi, ntiles, P, terms, part, ncols, grid, smem, s);
    case 2: return launch_tiled_e<R, 4>(psi, ntiles, P, terms, part, ncols, grid, smem, s);
    case 3: return launch_tiled_e<R, 8>(psi, ntiles, P, terms, part, ncols, grid, smem, s);
    case 4: return launch_tiled_e<R, 16>(psi, ntiles, P, terms, part, ncols, grid, smem, s);
    case 5: return launch_tiled_e<R, 32>(psi, ntiles, P, terms, part, ncols, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// NWQ_EXPECT_FP64=1: complex128 passes on the FP64 pipe only (no double words)
bool expect_fp64_only() {
  static const bool on = [] {
    const char* e = std::getenv("NWQ_EXPECT_FP64");
    return e && e[0] == '1';
  }();
  return on;
}

size_t sv_expect_tiled_smem(bool f64, const ExpPass& P) {
  return ((size_t)(f64 ? 16 : 8) << P.T) + ((size_t)8 << P.h) + (size_t)P.nk * sizeof(ExpTerm) +
         (size_t)(kExpThreads / 32) * P.nk * sizeof(double);
}

cudaError_t launch_sv_expect_tiled(bool f64, const void* psi, int n, const ExpPass& P, const ExpTerm* terms,
                                   double* part, int ncols, int grid, cudaStream_t s) {
  // tile bits (low m plus hmask) and tile-index bits (fmask) partition the index bits
  const uint64_t lowmask = (1ull << P.m) - 1;
  if (P.T < 0 || P.T > kExpTileBits || P.m < 0 || P.m + P.h != P.T || P.T > n || P.nk < 1 ||
      P.nk > kExpPassTerms || __builtin_popcountll(P.hmask) != P.h || __builtin_popcountll(P.fmask) != n - P.T ||
      ((P.hmask | P.fmask) & lowmask) || (P.hmask & P.fmask) || ((P.hmask | P.fmask | lowmask) >> n) || grid < 1)
    return cudaErrorInvalidValue;
  const uint64_t ntiles = 1ull << (n - P.T);
  const size_t smem = sv_expect_tiled_smem(f64, P);
  cudaError_t e = f64 ? launch_tiled_r<double>(psi, ntiles, P, terms, part, ncols, grid, smem, s)
                      : launch_tiled_r<float>(psi, ntiles, P, terms, part, ncols, grid, smem, s);
  g_launches += 1;
  return e;
}

cudaError_t launch_sv_expect_group(bool f64, const void* psi, int n, uint64_t x, const uint64_t* zm, const int* ym,
                                   int nt, double* part, int nblocks, const int* idx, double* out, cudaStream_t s) {
  uint64_t N = 1ull << n;
  if (f64) sv_expect_group<double><<<nblocks, 256, 0, s>>>((const double2*)psi, N, x, zm, ym, nt, part);
  else sv_expect_group<float><<<nblocks, 256, 0, s>>>((const float2*)psi, N, x, zm, ym, nt, part);
  cudaError_t e = cudaGetLastError();
  g_launches += 1;
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(part, nblocks, nt, idx, out, s);
}

cudaError_t launch_reduce_partials(const double* part, int nblocks, int nt, const int* idx, double* out,
                                   cudaStream_t s) {
  reduce_partials<<<(nt + 63) / 64, 64, 0, s>>>(part, nblocks, nt, idx, out);
  g_launches += 1;
  return cudaGetLastError();
}

}  // namespace nwq
