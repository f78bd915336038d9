// nwq_expect_pauli_sum_noalloc: Pauli expectation values with no memory
// allocation of any kind on the device.  The paper has no counterpart; this
// entry point exists for callers that cannot allocate device memory: code
// whose device memory is entirely reserved by another allocator (a
// framework's caching pool, a serving loop that admits work against a fixed
// memory budget) and latency-critical loops that must neither wait for nor
// fail on an allocation.
//
// Its scratch (term tables, per-block partial sums, results) lives in one
// file-scope device array of kScratchBytes bytes.  Every GPU that loads the
// library holds that array until the process exits.  All calls share it and
// it keeps the last call's contents; each call clears or writes every slot
// before reading it.  State vectors take the same passes and kernels as
// nwq_expect_pauli_sum (host tables on the stack) with two launch-shape
// reductions: the general (wide-X) kernel uses at most 256 blocks, and the
// tiled grid is reduced until its per-block partial sums fit the array.  Both
// change only the partition of the FP64 partial sums.  Calls that overlap on
// the GPU (two host threads, or two streams) race on the array and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/nwqgb.h"
#include "expect_host.hpp"
#include "kernels.hpp"
#include "state.hpp"

namespace nwq {
namespace {

constexpr int kMaxTerms = NWQ_NOALLOC_MAX_TERMS;
constexpr size_t kScratchBytes = 192 * 1024;
// DM: term table (x, z, coefficient per term) then the values
constexpr size_t kDmTable = 3 * kMaxTerms * sizeof(uint64_t);
static_assert(kDmTable + (kMaxTerms + 2) * sizeof(double) <= kScratchBytes, "DM scratch");
// SV: the tables and general partials for kMaxTerms terms leave room for the
// tiled partials of at least 32 blocks
static_assert(sv_expect_scratch_bytes(kMaxTerms, 32, kNoallocMaxGeneralBlocks) <= kScratchBytes, "SV scratch");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, looked up once per device (with that device
// current): in host code g_scratch names a host-side stand-in, not device memory.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return set_error(NWQ_EUNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != dev) e = cudaSetDevice(dev);
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_scratch);
    if (cur >= 0 && cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess || !p) return set_error(NWQ_ECUDA, "cudaGetSymbolAddress of the expectation scratch failed");
    g_addr[dev] = p;
  }
  *out = (unsigned char*)g_addr[dev];
  return NWQ_OK;
}

}  // namespace
}  // namespace nwq

using namespace nwq;

extern "C" int nwq_expect_pauli_sum_noalloc(nwq_state* st, const nwq_pauli_term* terms, size_t nt,
                                            double* out_host, uint32_t flags) {
  if (!st || !out_host || (nt && !terms)) return set_error(NWQ_EINVAL, "NULL argument");
  if (nt > (size_t)kMaxTerms)
    return set_error(NWQ_EINVAL, "nwq_expect_pauli_sum_noalloc: more than NWQ_NOALLOC_MAX_TERMS (256) terms");
  const bool sum = (flags & NWQ_EXPECT_SUM) != 0;
  const bool norm = (flags & NWQ_EXPECT_NORMALIZE) != 0;
  if (nt == 0) {
    if (sum) out_host[0] = 0.0;
    return NWQ_OK;
  }
  const uint64_t qmask = (1ull << st->n) - 1;
  for (size_t t = 0; t < nt; t++)
    if ((terms[t].x_mask & ~qmask) || (terms[t].z_mask & ~qmask))
      return set_error(NWQ_EINVAL, "Pauli mask out of range");
  unsigned char* base = nullptr;
  int rc = scratch_address(st->device, &base);
  if (rc) return rc;
  uint64_t* dz = (uint64_t*)base;           // DM term table
  double* dv = (double*)(base + kDmTable);  // DM values
  const bool f64 = st->dtype == NWQ_F64;
  cudaStream_t s = st->stream;
  cudaError_t e = cudaSuccess;

  if (st->kind == NWQ_DM) {
    uint64_t h[3 * kMaxTerms];
    for (size_t t = 0; t < nt; t++) {
      h[t] = terms[t].x_mask;
      h[nt + t] = terms[t].z_mask;
      double c = terms[t].coeff;
      __builtin_memcpy(&h[2 * nt + t], &c, sizeof(double));
    }
    e = cudaMemcpyAsync(dz, h, 3 * nt * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)  // coefficients read as they are, FP64 or double words
      e = launch_dm_expect(f64, st->buf, st->n, dz, dz + nt, (const double*)(dz + 2 * nt), (int)nt, dv, sum, norm, s,
                           st->dw_resident);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, dv, (sum ? 1 : nt) * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    return e == cudaSuccess ? NWQ_OK : set_error(NWQ_ECUDA, cudaGetErrorString(e));
  }

  // SV: the same passes and kernels as nwq_expect_pauli_sum, tables on the
  // stack, scratch in g_scratch; the tiled grid shrinks until its partial sums fit.
  ExpPass passes[kMaxTerms + 1];
  ExpTerm eterms[kMaxTerms + 1];
  int fb[kMaxTerms], work[2 * kMaxTerms + 2];
  SvChunk chunks[kMaxTerms];
  alignas(16) unsigned char stage[sv_expect_stage_bytes(kMaxTerms)];
  SvExpectHost h{passes, eterms, fb, chunks, work};
  SvExpectCounts c{};
  plan_sv_expect(st->n, terms, nt, norm, h, c);
  int grid = 0, fblocks = 0;
  sv_expect_shape(st, nt, kScratchBytes, &grid, &fblocks);
  e = sv_expect_enqueue(st, terms, nt, flags, out_host, h, c, grid, fblocks, stage, base);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return set_error(NWQ_ECUDA, cudaGetErrorString(e));
  return NWQ_OK;
}

extern "C" int nwq_expect_launch_shape(const nwq_state* st, size_t nt, int noalloc, int* grid, int* fblocks) {
  if (!st || !grid || !fblocks) return set_error(NWQ_EINVAL, "NULL argument");
  if (st->kind != NWQ_SV) return set_error(NWQ_EINVAL, "launch shape: state vectors only");
  sv_expect_shape(st, nt, noalloc ? kScratchBytes : 0, grid, fblocks);
  return NWQ_OK;
}
