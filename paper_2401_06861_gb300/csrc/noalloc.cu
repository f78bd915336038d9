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
// it keeps the last call's contents; the kernels below overwrite every slot
// they read, so nothing has to start at zero.  Calls that overlap on the GPU
// (two host threads, or two streams) race on the array and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/nwqgb.h"
#include "kernels.hpp"
#include "state.hpp"

namespace nwq {
namespace {

constexpr int kMaxTerms = NWQ_NOALLOC_MAX_TERMS;
constexpr int kMaxBlocks = 1024;                // partial sums per expectation pass
constexpr int kMaxChunks = kMaxTerms + 1;       // one chunk per term, plus the norm
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kPartBytes = align_up((size_t)kMaxBlocks * kExpectChunk * sizeof(double));
constexpr size_t kValBytes = align_up((kMaxTerms + 2) * sizeof(double));
constexpr size_t kZBytes = align_up((size_t)kMaxChunks * kExpectChunk * sizeof(uint64_t));
constexpr size_t kYBytes = align_up((size_t)kMaxChunks * kExpectChunk * sizeof(int));
constexpr size_t kCoefBytes = align_up(kMaxTerms * sizeof(double));
constexpr size_t kScratchBytes = kPartBytes + kValBytes + kZBytes + kYBytes + kCoefBytes;
static_assert(kScratchBytes <= 192 * 1024, "scratch must stay at most 192 KiB");
static_assert(3 * kMaxTerms * sizeof(uint64_t) <= kZBytes, "DM term table must fit the z region");

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
  double* dpart = (double*)base;
  double* dv = (double*)(base + kPartBytes);  // values; dv[nt] = norm, dv[nt+1] = weighted sum
  uint64_t* dz = (uint64_t*)(base + kPartBytes + kValBytes);
  int* dy = (int*)(base + kPartBytes + kValBytes + kZBytes);
  double* dc = (double*)(base + kPartBytes + kValBytes + kZBytes + kYBytes);
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
    if (e == cudaSuccess)
      e = launch_dm_expect(f64, st->buf, st->n, dz, dz + nt, (const double*)(dz + 2 * nt), (int)nt, dv, sum, norm, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, dv, (sum ? 1 : nt) * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    return e == cudaSuccess ? NWQ_OK : set_error(NWQ_ECUDA, cudaGetErrorString(e));
  }

  // SV: order terms by x mask (insertion sort on a stack array), then chunks
  // of at most kExpectChunk terms sharing x; the norm chunk goes last.
  int idx[kMaxTerms];
  for (size_t t = 0; t < nt; t++) {
    size_t k = t;
    while (k > 0 && terms[idx[k - 1]].x_mask > terms[t].x_mask) {
      idx[k] = idx[k - 1];
      k--;
    }
    idx[k] = (int)t;
  }
  uint64_t hz[kMaxChunks * kExpectChunk];
  int hy[kMaxChunks * kExpectChunk];
  double hc[kMaxTerms];
  uint64_t cx[kMaxChunks];
  int ccnt[kMaxChunks];
  int nchunk = 0;
  for (size_t t = 0; t < nt; t++) {
    const nwq_pauli_term& tm = terms[idx[t]];
    if (nchunk == 0 || cx[nchunk - 1] != tm.x_mask || ccnt[nchunk - 1] == kExpectChunk) {
      cx[nchunk] = tm.x_mask;
      ccnt[nchunk] = 0;
      nchunk++;
    }
    int c = nchunk - 1, j = ccnt[c]++;
    hz[c * kExpectChunk + j] = tm.z_mask;
    hy[c * kExpectChunk + j] = __builtin_popcountll(tm.x_mask & tm.z_mask) & 3;
    hc[t] = tm.coeff;
  }
  if (norm) {  // identity string: <psi|psi>, written to dv[nt]
    cx[nchunk] = 0;
    ccnt[nchunk] = 1;
    hz[nchunk * kExpectChunk] = 0;
    hy[nchunk * kExpectChunk] = 0;
    nchunk++;
  }
  const uint64_t N = 1ull << st->n;
  uint64_t nb = (N + 255) / 256;
  if (nb > (uint64_t)st->sm_count * 4) nb = (uint64_t)st->sm_count * 4;
  if (nb > (uint64_t)kMaxBlocks) nb = kMaxBlocks;
  e = cudaMemcpyAsync(dz, hz, (size_t)nchunk * kExpectChunk * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dy, hy, (size_t)nchunk * kExpectChunk * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dc, hc, nt * sizeof(double), cudaMemcpyHostToDevice, s);
  size_t done = 0;
  for (int c = 0; c < nchunk && e == cudaSuccess; c++) {
    e = launch_sv_expect_group(f64, st->buf, st->n, cx[c], dz + c * kExpectChunk, dy + c * kExpectChunk, ccnt[c],
                               dpart, (int)nb, dv + done, s);
    done += ccnt[c];
  }
  double vals[kMaxTerms];
  if (e == cudaSuccess && norm) e = launch_scale(dv, (int)nt, dv + nt, s);
  if (e == cudaSuccess && sum) {
    e = launch_weighted_sum(dv, dc, (int)nt, dv + nt + 1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, dv + nt + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
  } else if (e == cudaSuccess) {
    e = cudaMemcpyAsync(vals, dv, nt * sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return set_error(NWQ_ECUDA, cudaGetErrorString(e));
  if (!sum)
    for (size_t t = 0; t < nt; t++) out_host[idx[t]] = vals[t];
  return NWQ_OK;
}
