// Host side of the state-vector Pauli expectations: pass planning for the
// tiled kernel, table staging and the launch sequence.  Shared by
// nwq_expect_pauli_sum (pooled scratch) and nwq_expect_pauli_sum_noalloc
// (library-owned scratch); every buffer is the caller's, so this file
// allocates nothing itself.
#include "expect_host.hpp"

#include <cstring>

#include "kernels.hpp"

namespace nwq {

namespace {

// Tile-local image of v: bit i is v's bit at the i-th set bit of S (ascending).
uint32_t compress_bits(uint64_t v, uint64_t S) {
  uint32_t out = 0;
  int i = 0;
  for (uint64_t s = S; s; s &= s - 1, i++)
    if (v & s & (~s + 1)) out |= 1u << i;
  return out;
}

}  // namespace

// Pass 0 holds the low T bits of the index and takes every term whose X
// support lies there (all Z-type terms among them) plus, when normalising,
// the identity string.  Each further pass keeps the 16 lowest elements
// contiguous (runs of >= 128 bytes) and gathers T - 4 high bits, chosen
// greedily in term order so that as many of the remaining terms as possible
// have their X support inside the tile; a term whose X support cannot fit a
// tile goes to the general kernel.  Passes take at most kExpPassTerms terms.
void plan_sv_expect(int n, const nwq_pauli_term* terms, size_t nt, bool norm, SvExpectHost& h, SvExpectCounts& c) {
  const int T = n < kExpTileBits ? n : kExpTileBits;
  const int mhi = T < 4 ? T : 4;
  const uint64_t all = n >= 64 ? ~0ull : ((1ull << n) - 1);
  c = SvExpectCounts{};
  auto emit = [&](uint64_t S, const int* idx, int cnt) {
    int m = 0;
    while (m < T && ((S >> m) & 1)) m++;
    for (int c0 = 0; c0 < cnt; c0 += kExpPassTerms) {
      ExpPass P{};
      P.T = T;
      P.m = m;
      P.h = T - m;
      P.hmask = S & ~((1ull << m) - 1);
      P.fmask = all & ~S;
      P.k0 = c.nterms;
      P.nk = cnt - c0 < kExpPassTerms ? cnt - c0 : kExpPassTerms;
      for (int i = 0; i < P.nk; i++) {
        const int t = idx[c0 + i];
        const uint64_t x = t < 0 ? 0 : terms[t].x_mask, z = t < 0 ? 0 : terms[t].z_mask;
        ExpTerm& et = h.eterms[c.nterms++];
        et = ExpTerm{};
        et.xl = compress_bits(x, S);
        et.zl = compress_bits(z & S, S);
        et.zh = z & ~S;
        et.y = __builtin_popcountll(x & z) & 3;
        et.out = t < 0 ? (int)nt : t;
        if (et.xl == 0) P.zt = 1;
      }
      h.passes[c.npass++] = P;
    }
  };
  // work: [0, nt] the current list, [nt + 1, 2 nt + 2) the terms left over
  int* cur = h.work;
  int* left = h.work + nt + 1;
  const uint64_t S0 = (1ull << T) - 1;
  int ncur = 0, nrest = 0;
  for (size_t t = 0; t < nt; t++)
    if (!(terms[t].x_mask & ~S0)) cur[ncur++] = (int)t;
  if (norm) cur[ncur++] = -1;
  if (ncur) emit(S0, cur, ncur);
  for (size_t t = 0; t < nt; t++)
    if (terms[t].x_mask & ~S0) cur[nrest++] = (int)t;
  const uint64_t low = (1ull << mhi) - 1;
  while (nrest) {
    uint64_t H = 0;
    int ntake = 0, nleft = 0;
    // taken terms are compacted to the front of cur, the others go to left
    for (int i = 0; i < nrest; i++) {
      const int t = cur[i];
      const uint64_t need = terms[t].x_mask & ~low;
      if (__builtin_popcountll(H | need) <= T - mhi) {
        H |= need;
        cur[ntake++] = t;
      } else {
        left[nleft++] = t;
      }
    }
    if (!ntake) {  // X support wider than a tile
      h.fb[c.nfb++] = left[0];
      std::memmove(cur, left + 1, sizeof(int) * (size_t)(nleft - 1));
      nrest = nleft - 1;
      continue;
    }
    for (int b = mhi; b < n && __builtin_popcountll(H) < T - mhi; b++) H |= 1ull << b;  // fixed tile size
    emit(low | H, cur, ntake);
    std::memcpy(cur, left, sizeof(int) * (size_t)nleft);
    nrest = nleft;
  }
  // general terms: chunks of at most kExpectChunk sharing x (stable by x)
  for (int i = 1; i < c.nfb; i++) {  // insertion sort by x mask, stable
    const int t = h.fb[i];
    int k = i;
    while (k > 0 && terms[h.fb[k - 1]].x_mask > terms[t].x_mask) {
      h.fb[k] = h.fb[k - 1];
      k--;
    }
    h.fb[k] = t;
  }
  for (int i = 0; i < c.nfb; i++) {
    const uint64_t x = terms[h.fb[i]].x_mask;
    if (c.nchunk == 0 || h.chunks[c.nchunk - 1].x != x || h.chunks[c.nchunk - 1].cnt == kExpectChunk)
      h.chunks[c.nchunk++] = SvChunk{x, i, 0};
    h.chunks[c.nchunk - 1].cnt++;
  }
}

void sv_expect_shape(const nwq_state* st, size_t nt, size_t scratch_limit, int* grid, int* fblocks) {
  const bool f64 = st->dtype == NWQ_F64;
  const uint64_t N = 1ull << st->n;
  uint64_t fb = (N + 255) / 256;
  if (fb > (uint64_t)st->sm_count * 4) fb = (uint64_t)st->sm_count * 4;
  uint64_t g = 1ull << (st->n - (st->n < kExpTileBits ? st->n : kExpTileBits));
  // at most 3 (FP64) / 4 (FP32) CTAs per SM; each pass's launch takes at most
  // as many CTAs as fit on the device at once (launch_sv_expect_tiled)
  if (g > (uint64_t)st->sm_count * (f64 ? 3 : 4)) g = (uint64_t)st->sm_count * (f64 ? 3 : 4);
  if (scratch_limit) {
    if (fb > (uint64_t)kNoallocMaxGeneralBlocks) fb = kNoallocMaxGeneralBlocks;
    while (g > 1 && sv_expect_scratch_bytes(nt, (int)g, (int)fb) > scratch_limit) g--;
  }
  *grid = (int)g;
  *fblocks = (int)fb;
}

cudaError_t state_to_f64(nwq_state* st) {
  if (!st->dw_resident) return cudaSuccess;
  const uint64_t ndouble = (st->kind == NWQ_SV ? 2ull : 1ull) << st->B;
  const cudaError_t e = launch_dw_convert(st->buf, ndouble, false, st->sm_count, st->stream);
  if (e == cudaSuccess) st->dw_resident = false;
  return e;
}

cudaError_t sv_expect_enqueue(nwq_state* st, const nwq_pauli_term* terms, size_t nt, uint32_t flags,
                              double* out_host, const SvExpectHost& h, const SvExpectCounts& c, int grid,
                              int fblocks, unsigned char* stage, unsigned char* dev) {
  const bool sum = (flags & NWQ_EXPECT_SUM) != 0;
  const bool norm = (flags & NWQ_EXPECT_NORMALIZE) != 0;
  const bool f64 = st->dtype == NWQ_F64;
  cudaStream_t s = st->stream;
  const int ncols = (int)nt + 1;  // column nt: <psi|psi>
  // staging / scratch layout: [terms | z | y | idx | coef] then [values | tiled partials | general partials]
  const size_t o_z = sv_expect_up16((nt + 1) * sizeof(ExpTerm));
  const size_t o_y = o_z + sv_expect_up16(nt * 8);
  const size_t o_idx = o_y + sv_expect_up16(nt * 8);
  const size_t o_coef = o_idx + sv_expect_up16(nt * 8);
  const size_t o_vals = o_coef + sv_expect_up16(nt * 8);
  const size_t o_part = o_vals + sv_expect_up16((nt + 2) * 8);
  const size_t o_fpart = o_part + sv_expect_up16((size_t)grid * ncols * 8);
  std::memcpy(stage, h.eterms, (size_t)c.nterms * sizeof(ExpTerm));
  for (int i = 0; i < c.nfb; i++) {
    const nwq_pauli_term& tm = terms[h.fb[i]];
    const uint64_t z = tm.z_mask;
    const int y = __builtin_popcountll(tm.x_mask & tm.z_mask) & 3, id = h.fb[i];
    std::memcpy(stage + o_z + (size_t)i * 8, &z, 8);
    std::memcpy(stage + o_y + (size_t)i * 4, &y, 4);
    std::memcpy(stage + o_idx + (size_t)i * 4, &id, 4);
  }
  for (size_t t = 0; t < nt; t++) std::memcpy(stage + o_coef + t * 8, &terms[t].coeff, 8);
  double* dv = (double*)(dev + o_vals);
  double* dpart = (double*)(dev + o_part);
  // a state in the double-word layout: read as it is by full complex128 tile passes only
  bool dwin = st->dw_resident && c.nchunk == 0 && !expect_fp64_only();
  for (int i = 0; i < c.npass && dwin; i++) dwin = h.passes[i].T == kExpTileBits;
  cudaError_t e = dwin ? cudaSuccess : state_to_f64(st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dev, stage, o_vals, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && c.npass) {
    // columns of general terms (and the norm column when unused) stay zero
    e = cudaMemsetAsync(dpart, 0, (size_t)grid * ncols * 8, s);
    for (int i = 0; i < c.npass && e == cudaSuccess; i++) {
      ExpPass P = h.passes[i];
      P.dwin = dwin ? 1 : 0;
      e = launch_sv_expect_tiled(f64, st->buf, st->n, P, (const ExpTerm*)dev, dpart, ncols, grid, s);
    }
    if (e == cudaSuccess) e = launch_reduce_partials(dpart, grid, ncols, nullptr, dv, s);
  }
  for (int k = 0; k < c.nchunk && e == cudaSuccess; k++) {
    const SvChunk& ch = h.chunks[k];
    e = launch_sv_expect_group(f64, st->buf, st->n, ch.x, (const uint64_t*)(dev + o_z) + ch.off,
                               (const int*)(dev + o_y) + ch.off, ch.cnt, (double*)(dev + o_fpart), fblocks,
                               (const int*)(dev + o_idx) + ch.off, dv, s);
  }
  if (e == cudaSuccess && norm) e = launch_scale(dv, (int)nt, dv + nt, s);
  if (e == cudaSuccess && sum) {
    e = launch_weighted_sum(dv, (const double*)(dev + o_coef), (int)nt, dv + nt + 1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, dv + nt + 1, 8, cudaMemcpyDeviceToHost, s);
  } else if (e == cudaSuccess) {
    e = cudaMemcpyAsync(out_host, dv, nt * 8, cudaMemcpyDeviceToHost, s);
  }
  return e;
}

}  // namespace nwq
