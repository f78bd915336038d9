// C ABI of the simulator: state handles, plans, measurement.  Every device
// step runs in the library's kernels (sweep_kernels.cu, expect_kernels.cu,
// batch_kernels.cu and the run-time specialised sweeps of jit.cpp); this file
// validates arguments, lowers circuits (planner.cpp), uploads operator tables
// and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/nwqgb.h"
#include "expect_host.hpp"
#include "jit.hpp"
#include "nvtx_range.hpp"
#include "kernels.hpp"
#include "planner.hpp"
#include "state.hpp"

using namespace nwq;

static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
static int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return NWQ_ECUDA;
}
#define CK(call, what)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// Error reporting shared with the other translation units of the library.
int nwq::set_error(int code, const char* msg) {
  g_err = msg;
  return code;
}

// ------------------------------------------------------------------ helpers
static bool f64_of(int dtype) { return dtype == NWQ_F64; }

extern "C" size_t nwq_state_bytes(int kind, int n, int dtype) {
  if ((kind != NWQ_SV && kind != NWQ_DM) || (dtype != NWQ_F32 && dtype != NWQ_F64) || n < 1) return 0;
  size_t real = dtype == NWQ_F64 ? 8 : 4;
  if (kind == NWQ_SV) return n > 34 ? 0 : (2 * real) << n;
  return n > 16 ? 0 : real << (2 * n);
}

static void plan_options(int kind, int dtype, uint32_t flags, PlanOptions& o) {
  bool cplx = kind == NWQ_SV;
  size_t esz = (cplx ? 2 : 1) * (dtype == NWQ_F64 ? 8 : 4);
  // ping-pong tiles of 32 KiB (16 KiB for complex128: its FP64-bound phases
  // run faster with 4 resident CTAs per SM than with 2), >= 128 contiguous bytes
  o.tile_bits = esz == 16 ? 10 : esz == 8 ? 12 : 13;
  o.min_low = esz == 16 ? 3 : esz == 8 ? 4 : 5;
  if (const char* tb = std::getenv("NWQ_TILE_BITS")) {
    int v = std::atoi(tb);
    if (v >= 4 && v <= kMaxTileBits && (2 * esz << v) <= (size_t)kMaxDynSmem) o.tile_bits = v;
  }
  o.plain = (flags & NWQ_PLAN_PLAIN) != 0;
  // state vectors: diagonal operators may pass skipped diagonal operators
  // when grouping sweeps, unless NWQ_PLAN_NO_COMMUTE
  o.commute = kind == NWQ_SV && !(flags & NWQ_PLAN_NO_COMMUTE) && !o.plain;
  o.merge = !(flags & (NWQ_PLAN_PLAIN | NWQ_PLAN_NO_MERGE));
}

static void init_plan_meta(Plan& p, int kind, int n, int dtype, int B) {
  p.kind = kind;
  p.n = n;
  p.dtype = dtype;
  p.B = B;
  p.is_complex = kind == NWQ_SV;
  size_t real = dtype == NWQ_F64 ? 8 : 4;
  p.elem_bytes = (p.is_complex ? 2 : 1) * real;
  p.ent_bytes = p.is_complex ? (dtype == NWQ_F64 ? sizeof(EntC<double>) : sizeof(EntC<float>))
                             : (dtype == NWQ_F64 ? sizeof(EntR<double>) : sizeof(EntR<float>));
}

// Upload a plan's tables once (stream-ordered); later runs reuse them.
static int plan_upload(Plan& p, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(p.mu);
  if (p.dev) return NWQ_OK;
  size_t ob = p.ops.size() * sizeof(DevOp);
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t o_ph = al(ob + p.ents.size());
  size_t o_po = al(o_ph + p.phases.size() * sizeof(PhaseDesc));
  size_t o_pc = al(o_po + p.pops.size() * sizeof(PhaseOp));
  size_t o_tc = al(o_pc + p.pcoef.size());
  size_t total = o_tc + p.tctab.size() * sizeof(float) + 16;
  void* d = nullptr;
  if (p.stream_ordered) {
    CK(cudaMallocAsync(&d, total, s), "plan table allocation");
    p.dev_stream = s;
  } else {
    CK(cudaMalloc(&d, total), "plan table allocation");
  }
  if (ob) CK(cudaMemcpyAsync(d, p.ops.data(), ob, cudaMemcpyHostToDevice, s), "plan upload");
  if (!p.ents.empty())
    CK(cudaMemcpyAsync((char*)d + ob, p.ents.data(), p.ents.size(), cudaMemcpyHostToDevice, s), "plan upload");
  if (!p.phases.empty())
    CK(cudaMemcpyAsync((char*)d + o_ph, p.phases.data(), p.phases.size() * sizeof(PhaseDesc), cudaMemcpyHostToDevice, s),
       "plan upload");
  if (!p.pops.empty())
    CK(cudaMemcpyAsync((char*)d + o_po, p.pops.data(), p.pops.size() * sizeof(PhaseOp), cudaMemcpyHostToDevice, s),
       "plan upload");
  if (!p.pcoef.empty())
    CK(cudaMemcpyAsync((char*)d + o_pc, p.pcoef.data(), p.pcoef.size(), cudaMemcpyHostToDevice, s), "plan upload");
  if (!p.tctab.empty())
    CK(cudaMemcpyAsync((char*)d + o_tc, p.tctab.data(), p.tctab.size() * sizeof(float), cudaMemcpyHostToDevice, s),
       "plan upload");
  p.tc_off = o_tc;
  p.pt_off[0] = o_ph;
  p.pt_off[1] = o_po;
  p.pt_off[2] = o_pc;
  CK(cudaStreamSynchronize(s), "plan upload");
  p.dev = d;
  p.dev_bytes = total;
  return NWQ_OK;
}

// st: the state whose buffer data is (NULL for scratch buffers).  A
// double-word run leaves a library-owned state in the double-word layout
// (dw_resident) and starts from it; every other plan needs the FP64 layout.
static int plan_launch(Plan& p, void* data, cudaStream_t s, int sm_count, nwq_state* st = nullptr) {
  NvtxRange range("nwq plan run");
  int rc = plan_upload(p, s);
  if (rc) return rc;
  const bool dw = !p.tc && p.dw && jit_dw_ready(p);
  if (st && !dw) {
    cudaError_t e = state_to_f64(st);
    if (e != cudaSuccess) return cuda_fail(e, "double-word conversion");
  }
  if (p.tc) {  // dense five-qubit blocks on the tensor cores, one pass each
    const float* tab = (const float*)((const char*)p.dev + p.tc_off);
    for (size_t i = 0; i < p.tcg.size(); i++) {
      NvtxRange sweep_range("nwq tc block");
      cudaError_t e = launch_tc_block(data, p.tcg[i], tab + i * kTcMatFloats, sm_count, s);
      if (e != cudaSuccess) return cuda_fail(e, "tensor-core block launch");
    }
    return NWQ_OK;
  }
  const DevOp* ops = (const DevOp*)p.dev;
  const void* ents = (const char*)p.dev + p.ops.size() * sizeof(DevOp);
  PhaseTables pt{(const PhaseDesc*)((const char*)p.dev + p.pt_off[0]), (const PhaseOp*)((const char*)p.dev + p.pt_off[1]),
                 (const char*)p.dev + p.pt_off[2]};
  // double-word plans: the state goes to the double-word layout for the
  // sweeps when every sweep has its double-word kernel (unless it is there
  // already), and back after them unless the library owns it
  p.last_run_dw = dw;
  const uint64_t ndouble = (p.is_complex ? 2ull : 1ull) << p.B;
  if (dw && !(st && st->dw_resident)) {
    cudaError_t e = launch_dw_convert(data, ndouble, true, sm_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "double-word conversion");
  } else if (dw && !st->dw_exact) {  // left by an earlier run: low parts renormalised first
    cudaError_t e = launch_dw_renormalize(data, ndouble, sm_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "double-word renormalisation");
  }
  for (size_t i = 0; i < p.sweeps.size(); i++) {
    const SweepDesc& sd = p.sweeps[i];
    if (sd.nops == 0) continue;
    NvtxRange sweep_range("nwq sweep");
    cudaError_t e = cudaSuccess;
    if (dw) {
      if (!jit_launch_sweep(p, i, pt, data, sm_count, s, &e, true)) e = cudaErrorInvalidValue;  // ready: never
    } else if (!((!p.is_complex || sd.nph > 0) && jit_launch_sweep(p, i, pt, data, sm_count, s, &e))) {
      e = launch_sweep(p.is_complex, p.dtype == NWQ_F64, data, p.B, sd, ops, ents, p.phases.empty() ? nullptr : &pt,
                       sm_count, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
  }
  if (dw && st && st->owned) {
    st->dw_resident = true;
    st->dw_exact = false;
  } else if (dw) {
    if (st) st->dw_resident = false;
    cudaError_t e = launch_dw_convert(data, ndouble, false, sm_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "double-word conversion");
  }
  return NWQ_OK;
}

Plan::~Plan() {
  if (!dev) return;
  if (stream_ordered) cudaFreeAsync(dev, dev_stream);
  else cudaFree(dev);
}

// ------------------------------------------------------------------ states
static int create_state(int kind, int n, int dtype, void* dev_buf, size_t buf_bytes, void* stream, nwq_state** out) {
  if (!out) return fail(NWQ_EINVAL, "out is NULL");
  *out = nullptr;
  size_t need = nwq_state_bytes(kind, n, dtype);
  if (!need) return fail(NWQ_EINVAL, "unsupported qubit count or dtype");
  if (dev_buf && buf_bytes < need) return fail(NWQ_EINVAL, "device buffer too small");
  if (dev_buf && ((uintptr_t)dev_buf & 15)) return fail(NWQ_EINVAL, "device buffer not 16-byte aligned");
  auto st = std::make_unique<nwq_state>();
  st->kind = kind;
  st->n = n;
  st->dtype = dtype;
  st->B = kind == NWQ_SV ? n : 2 * n;
  st->bytes = need;
  st->stream = (cudaStream_t)stream;
  CK(cudaGetDevice(&st->device), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&st->sm_count, cudaDevAttrMultiProcessorCount, st->device), "device query");
  if (dev_buf) {
    st->buf = dev_buf;
  } else {
    cudaError_t e = cudaMallocAsync(&st->buf, need, st->stream);  // stream-ordered, pooled
    if (e != cudaSuccess) return fail(NWQ_ENOMEM, std::string("state allocation: ") + cudaGetErrorString(e));
    st->owned = true;
  }
  cudaError_t e = launch_init(kind == NWQ_SV, f64_of(dtype), st->buf, n, st->sm_count, st->stream);
  if (e != cudaSuccess) {
    if (st->owned) cudaFreeAsync(st->buf, st->stream);
    return cuda_fail(e, "state init");
  }
  *out = st.release();
  return NWQ_OK;
}

extern "C" int nwq_sv_create(int n, int dtype, void* dev_buf, size_t buf_bytes, void* stream, nwq_state** out) {
  return create_state(NWQ_SV, n, dtype, dev_buf, buf_bytes, stream, out);
}
extern "C" int nwq_dm_create(int n, int dtype, void* dev_buf, size_t buf_bytes, void* stream, nwq_state** out) {
  return create_state(NWQ_DM, n, dtype, dev_buf, buf_bytes, stream, out);
}

extern "C" int nwq_state_reset(nwq_state* st) {
  if (!st) return fail(NWQ_EINVAL, "state is NULL");
  // a state left in the double-word layout is reset in that layout (its next
  // double-word run then needs no conversion); anything else in FP64 / FP32
  const bool dw = st->dw_resident;
  cudaError_t e = launch_init(st->kind == NWQ_SV, f64_of(st->dtype), st->buf, st->n, st->sm_count, st->stream, dw);
  st->dw_resident = dw && e == cudaSuccess;
  st->dw_exact = st->dw_resident;  // |0..0> is exact in either layout
  return e == cudaSuccess ? NWQ_OK : cuda_fail(e, "state reset");
}

// The FP64 layout before a reader or writer of the buffer (see dw_resident).
static int state_f64(nwq_state* st) {
  cudaError_t e = state_to_f64(st);
  return e == cudaSuccess ? NWQ_OK : cuda_fail(e, "double-word conversion");
}

extern "C" int nwq_destroy(nwq_state* st) {
  if (!st) return NWQ_OK;
  // stream-ordered release: work already queued on the state's stream finishes first
  if (st->owned && st->buf) cudaFreeAsync(st->buf, st->stream);
  delete st;  // the state's helper plans free their tables on the same stream
  return NWQ_OK;
}

extern "C" int nwq_device_sync(nwq_state* st) {
  if (!st) return fail(NWQ_EINVAL, "state is NULL");
  CK(cudaStreamSynchronize(st->stream), "stream synchronize");
  return NWQ_OK;
}

// Per-qubit basis change between Pauli coefficients and vec(rho) (complex, 2n bits).
static nwq_plan* dm_conv_plan(nwq_state* st, bool to_rho) {
  std::unique_ptr<nwq_plan>& slot = to_rho ? st->p2r : st->r2p;
  if (slot) return slot.get();
  auto pl = std::make_unique<nwq_plan>();
  pl->p.stream_ordered = true;
  init_plan_meta(pl->p, NWQ_SV, st->n, st->dtype, 2 * st->n);  // complex elements over 2n bits
  cd M[16];
  if (to_rho) pauli_to_rho_matrix(M);
  else rho_to_pauli_matrix(M);
  std::vector<BitOp> ops(st->n);
  for (int q = 0; q < st->n; q++) {
    ops[q].k = 2;
    ops[q].bits[0] = q;
    ops[q].bits[1] = q + st->n;
    ops[q].m.assign(M, M + 16);
    ops[q].gate0 = q;
  }
  PlanOptions o;
  plan_options(NWQ_SV, st->dtype, NWQ_PLAN_NO_MERGE, o);
  build_plan(ops, o, pl->p);
  slot = std::move(pl);
  return slot.get();
}

static int dm_to_rho(nwq_state* st, void* dst_dev) {
  bool f64 = f64_of(st->dtype);
  uint64_t count = 1ull << (2 * st->n);
  cudaError_t e = launch_real_to_cplx(f64, st->buf, dst_dev, count, st->sm_count, st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dm convert");
  return plan_launch(dm_conv_plan(st, true)->p, dst_dev, st->stream, st->sm_count);
}

extern "C" int nwq_state_copy(nwq_state* st, void* dst, size_t bytes, int dst_on_device) {
  if (!st || !dst) return fail(NWQ_EINVAL, "NULL argument");
  if (int rc = state_f64(st)) return rc;
  if (st->kind == NWQ_SV) {
    if (bytes < st->bytes) return fail(NWQ_EINVAL, "destination too small");
    CK(cudaMemcpyAsync(dst, st->buf, st->bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       st->stream),
       "state copy");
    CK(cudaStreamSynchronize(st->stream), "state copy");
    return NWQ_OK;
  }
  size_t need = 2 * st->bytes;  // complex vec(rho)
  if (bytes < need) return fail(NWQ_EINVAL, "destination too small");
  void* tmp = dst;
  if (!dst_on_device) CK(cudaMallocAsync(&tmp, need, st->stream), "scratch allocation");
  int rc = dm_to_rho(st, tmp);
  if (!rc && !dst_on_device) {
    cudaError_t e = cudaMemcpyAsync(dst, tmp, need, cudaMemcpyDeviceToHost, st->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "state copy");
  }
  if (!dst_on_device) cudaFreeAsync(tmp, st->stream);
  cudaError_t e = cudaStreamSynchronize(st->stream);
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "state copy");
  return rc;
}

extern "C" int nwq_dm_copy_pauli(nwq_state* st, void* dst, size_t bytes, int dst_on_device) {
  if (!st || !dst) return fail(NWQ_EINVAL, "NULL argument");
  if (st->kind != NWQ_DM) return fail(NWQ_EINVAL, "not a density matrix");
  if (bytes < st->bytes) return fail(NWQ_EINVAL, "destination too small");
  if (int rc = state_f64(st)) return rc;
  CK(cudaMemcpyAsync(dst, st->buf, st->bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     st->stream),
     "copy");
  CK(cudaStreamSynchronize(st->stream), "copy");
  return NWQ_OK;
}

extern "C" int nwq_dm_load_pauli(nwq_state* st, const void* src, size_t bytes, int src_on_device) {
  if (!st || !src) return fail(NWQ_EINVAL, "NULL argument");
  if (st->kind != NWQ_DM) return fail(NWQ_EINVAL, "not a density matrix");
  if (bytes != st->bytes) return fail(NWQ_EINVAL, "size mismatch");
  st->dw_resident = false;  // overwritten in the FP64 layout
  CK(cudaMemcpyAsync(st->buf, src, bytes, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     st->stream),
     "state load");
  CK(cudaStreamSynchronize(st->stream), "state load");
  return NWQ_OK;
}

extern "C" int nwq_state_load(nwq_state* st, const void* src, size_t bytes, int src_on_device) {
  if (!st || !src) return fail(NWQ_EINVAL, "NULL argument");
  cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (st->kind == NWQ_SV) {
    if (bytes != st->bytes) return fail(NWQ_EINVAL, "size mismatch");
    st->dw_resident = false;  // overwritten in the FP64 layout
    CK(cudaMemcpyAsync(st->buf, src, bytes, kind, st->stream), "state load");
    CK(cudaStreamSynchronize(st->stream), "state load");
    return NWQ_OK;
  }
  size_t need = 2 * st->bytes;
  if (bytes != need) return fail(NWQ_EINVAL, "size mismatch");
  st->dw_resident = false;  // overwritten in the FP64 layout
  void* tmp = nullptr;
  CK(cudaMallocAsync(&tmp, need, st->stream), "scratch allocation");
  int rc = NWQ_OK;
  cudaError_t e = cudaMemcpyAsync(tmp, src, need, kind, st->stream);
  if (e != cudaSuccess) rc = cuda_fail(e, "state load");
  if (!rc) rc = plan_launch(dm_conv_plan(st, false)->p, tmp, st->stream, st->sm_count);
  if (!rc) {
    e = launch_cplx_to_real(f64_of(st->dtype), tmp, st->buf, 1ull << (2 * st->n), st->sm_count, st->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "state load");
  }
  cudaFreeAsync(tmp, st->stream);
  e = cudaStreamSynchronize(st->stream);
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "state load");
  return rc;
}

// ------------------------------------------------------------------ plans
extern "C" int nwq_plan_create(int kind, int n, int dtype, const nwq_gate* gates, size_t ng,
                               const nwq_noise_model* nm, uint32_t flags, void* stream, nwq_plan** out) {
  return nwq_plan_create_tuned(kind, n, dtype, gates, ng, nm, flags, nullptr, stream, out);
}

extern "C" int nwq_plan_create_tuned(int kind, int n, int dtype, const nwq_gate* gates, size_t ng,
                                     const nwq_noise_model* nm, uint32_t flags, const nwq_plan_tuning* tuning,
                                     void* stream, nwq_plan** out) {
  (void)stream;
  NvtxRange range("nwq plan create");
  if (!out) return fail(NWQ_EINVAL, "out is NULL");
  *out = nullptr;
  if (!nwq_state_bytes(kind, n, dtype)) return fail(NWQ_EINVAL, "unsupported qubit count or dtype");
  if (ng && !gates) return fail(NWQ_EINVAL, "gates is NULL");
  if (kind == NWQ_SV && nm) return fail(NWQ_EINVAL, "noise model needs a density matrix");
  for (size_t i = 0; i < ng; i++)
    if (gates[i].reserved || gates[i].reserved2) return fail(NWQ_EINVAL, "reserved gate field not 0");
  // NWQ_PLAN=plain|fused|tc|commute|nocommute picks the plan form when the
  // call names none (no PLAIN / TC / COMMUTE / NO_COMMUTE flag, no tuning);
  // tc applies where it is supported; commute (the default) and nocommute to
  // state vectors.
  static const int env_plan = [] {
    const char* e = std::getenv("NWQ_PLAN");
    if (!e) return 0;
    if (!std::strcmp(e, "plain")) return 1;
    if (!std::strcmp(e, "tc")) return 2;
    if (!std::strcmp(e, "commute")) return 3;
    if (!std::strcmp(e, "nocommute")) return 4;
    return 0;
  }();
  if (env_plan && !tuning &&
      !(flags & (NWQ_PLAN_PLAIN | NWQ_PLAN_TC | NWQ_PLAN_COMMUTE | NWQ_PLAN_NO_COMMUTE))) {
    if (env_plan == 1) flags |= NWQ_PLAN_PLAIN;
    else if (env_plan == 3) flags |= NWQ_PLAN_COMMUTE;
    else if (env_plan == 4) flags |= NWQ_PLAN_NO_COMMUTE;
    else if (kind == NWQ_SV && dtype == NWQ_F32 && n >= kTcMinQubits) flags |= NWQ_PLAN_TC;
  }
  auto pl = std::make_unique<nwq_plan>();
  init_plan_meta(pl->p, kind, n, dtype, kind == NWQ_SV ? n : 2 * n);
  std::vector<BitOp> ops;
  std::string err;
  bool ok = kind == NWQ_SV ? lower_sv(gates, ng, n, ops, err) : lower_dm(gates, ng, n, nm, ops, err);
  if (!ok) return fail(NWQ_EINVAL, err);
  if (tuning && tuning->fusion_bits == kTcBits) flags |= NWQ_PLAN_TC;  // shape "5 fused qubits" = tensor-core blocks
  if (flags & NWQ_PLAN_TC) {
    if (kind != NWQ_SV || dtype != NWQ_F32 || n < kTcMinQubits)
      return fail(NWQ_EUNSUPPORTED, "tensor-core plans take complex64 state vectors of at least 12 qubits");
    if (!build_tc_plan(ops, pl->p, err)) return fail(NWQ_EINVAL, err);
    static const bool tc_checks = [] {
      const char* e = std::getenv("NWQ_CHECKS");
      return e && e[0] == '1';
    }();
    if (tc_checks) {
      std::string cerr;
      if (!verify_plan(pl->p, cerr)) return fail(NWQ_EINVAL, cerr);
    }
    *out = pl.release();
    return NWQ_OK;
  }
  PlanOptions o;
  plan_options(kind, dtype, flags, o);
  if (tuning) {
    const size_t esz = pl->p.elem_bytes;
    if (tuning->tile_bits) {
      if (tuning->tile_bits < 4 || tuning->tile_bits > kMaxTileBits ||
          (2 * esz << tuning->tile_bits) > (size_t)kMaxDynSmem)
        return fail(NWQ_EINVAL, "tile_bits out of range for this element size");
      o.tile_bits = tuning->tile_bits;
    }
    if (tuning->fusion_bits) {
      if (tuning->fusion_bits < 2 || tuning->fusion_bits > 4) return fail(NWQ_EINVAL, "fusion_bits must be 2..4 (5: tensor-core blocks, complex64 state vectors)");
      o.max_merge_bits = tuning->fusion_bits;
    }
    if (tuning->register_bits) {
      if (tuning->register_bits != 3 && tuning->register_bits != 4)
        return fail(NWQ_EINVAL, "register_bits must be 3 or 4");
      o.register_bits = tuning->register_bits;
    }
  }
  if (kind == NWQ_DM && !(flags & NWQ_PLAN_NO_RESCALE)) o.rescale_qubits = n;
  // double-word sweeps for FP64 plans unless NWQ_PLAN_FP64; NWQ_DW=1 / 0
  // forces them on / off
  static const int env_dw = [] {
    const char* e = std::getenv("NWQ_DW");
    return !e ? -1 : (e[0] == '1' ? 1 : 0);
  }();
  pl->p.dw = dtype == NWQ_F64 && (env_dw == 1 || (env_dw == -1 && !(flags & NWQ_PLAN_FP64)));
  // double-word complex128 sweeps are FP32-issue bound: tiles of 2^11 give
  // every thread of a 256-thread CTA a register group of 8 amplitudes in each
  // phase (2^10 tiles, sized for the FP64 pipe, leave half of them idle)
  const bool dw_sv = pl->p.dw && kind == NWQ_SV && n >= jit_min_state_bits();  // run by specialised kernels
  if (dw_sv && !(tuning && tuning->tile_bits) && !std::getenv("NWQ_TILE_BITS")) o.tile_bits = 11;
  // and at most 16 operators per sweep: their generated code then stays in the
  // instruction cache (n = 33 depth-10 chain: 30 sweeps instead of 27, plan run
  // 3.68 -> 3.59 s); NWQ_SWEEP_MAX_OPS sets the cap of every plan (0: none)
  if (const char* mo = std::getenv("NWQ_SWEEP_MAX_OPS")) o.max_sweep_ops = std::max(0, std::atoi(mo));
  else if (dw_sv) o.max_sweep_ops = 16;
  build_plan(ops, o, pl->p);
  pl->p.interpreted = (flags & NWQ_PLAN_INTERPRETED) != 0;
  static const bool checks = [] {
    const char* e = std::getenv("NWQ_CHECKS");
    return e && e[0] == '1';
  }();
  if (checks) {
    std::string cerr;
    if (!verify_plan(pl->p, cerr)) return fail(NWQ_EINVAL, cerr);
  }
  *out = pl.release();
  return NWQ_OK;
}

extern "C" int nwq_plan_run(nwq_state* st, const nwq_plan* plan) {
  if (!st || !plan) return fail(NWQ_EINVAL, "NULL argument");
  const Plan& p = plan->p;
  if (p.kind != st->kind || p.n != st->n || p.dtype != st->dtype) return fail(NWQ_EINVAL, "plan does not match state");
  return plan_launch(const_cast<Plan&>(p), st->buf, st->stream, st->sm_count, st);
}

extern "C" int nwq_plan_autotune(nwq_state* st, const nwq_gate* gates, size_t ng, const nwq_noise_model* nm,
                                 uint32_t flags, int reps, nwq_plan_tuning* best, double* best_ms,
                                 nwq_plan_tuning* tried, double* tried_ms, int max_tried, int* ntried) {
  if (!st || !best || (ng && !gates)) return fail(NWQ_EINVAL, "NULL argument");
  if (reps < 1) return fail(NWQ_EINVAL, "reps must be >= 1");
  const size_t esz = (st->kind == NWQ_SV ? 2 : 1) * (st->dtype == NWQ_F64 ? 8 : 4);
  const int t0 = esz == 16 ? 11 : esz == 8 ? 12 : 13;
  std::vector<nwq_plan_tuning> cand;
  for (int dt = -1; dt <= 1; dt++) {
    const int tb = t0 + dt;
    if ((2 * esz << tb) > (size_t)kMaxDynSmem) continue;
    for (int fb : (st->kind == NWQ_DM ? std::vector<int>{2, 4} : std::vector<int>{3, 4}))
      for (int rb : (st->kind == NWQ_SV ? std::vector<int>{3, 4} : std::vector<int>{0})) cand.push_back({tb, fb, rb});
  }
  // complex64 state vectors: also the dense five-qubit blocks on the tensor cores
  if (st->kind == NWQ_SV && st->dtype == NWQ_F32 && st->n >= kTcMinQubits && !(flags & NWQ_PLAN_PLAIN))
    cand.push_back({0, kTcBits, 0});
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a), "event");
  CK(cudaEventCreate(&b), "event");
  double bms = -1.0;
  int nt = 0;
  for (const nwq_plan_tuning& c : cand) {
    double ms = -1.0;
    nwq_plan* pl = nullptr;
    if (nwq_plan_create_tuned(st->kind, st->n, st->dtype, gates, ng, nm, flags, &c, st->stream, &pl) == NWQ_OK) {
      bool ok = nwq_plan_run(st, pl) == NWQ_OK && cudaStreamSynchronize(st->stream) == cudaSuccess;  // warm-up
      if (ok) {
        cudaEventRecord(a, st->stream);
        for (int r = 0; r < reps && ok; r++) ok = nwq_plan_run(st, pl) == NWQ_OK;
        cudaEventRecord(b, st->stream);
        float f = 0.f;
        ok = ok && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&f, a, b) == cudaSuccess;
        if (ok) ms = f / reps;
      }
      nwq_plan_destroy(pl);
    }
    cudaGetLastError();  // a failed candidate leaves no sticky launch error behind
    if (tried && nt < max_tried) {
      tried[nt] = c;
      if (tried_ms) tried_ms[nt] = ms;
    }
    nt++;
    if (ms >= 0 && (bms < 0 || ms < bms)) {
      bms = ms;
      *best = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (ntried) *ntried = nt < max_tried ? nt : max_tried;
  if (best_ms) *best_ms = bms;
  nwq_state_reset(st);
  if (bms < 0) return fail(NWQ_ECUDA, "no candidate plan shape could be run");
  return NWQ_OK;
}

extern "C" int nwq_plan_info(const nwq_plan* plan, int* sweeps, int* ops, double* bytes, double* fma_per_elem,
                             size_t* table_bytes) {
  if (!plan) return fail(NWQ_EINVAL, "plan is NULL");
  int ns = 0;
  for (auto& s : plan->p.sweeps) ns += s.nops > 0;
  if (plan->p.tc) ns = (int)plan->p.tcb.size();
  if (sweeps) *sweeps = ns;
  if (ops) *ops = plan->p.tc ? ns : (int)plan->p.ops.size();
  if (bytes) *bytes = plan->p.bytes;
  if (fma_per_elem) *fma_per_elem = plan->p.fma_per_elem;
  if (table_bytes)
    *table_bytes = plan->p.ops.size() * sizeof(DevOp) + plan->p.ents.size() + plan->p.tctab.size() * sizeof(float);
  return NWQ_OK;
}

extern "C" int nwq_plan_layout(const nwq_plan* plan, int* sweep_nops, int* op_gate, int* op_ngates) {
  if (!plan) return fail(NWQ_EINVAL, "plan is NULL");
  int s = 0;
  for (auto& sd : plan->p.sweeps)
    if (sd.nops > 0 && sweep_nops) sweep_nops[s++] = sd.nops;
  if (plan->p.tc && sweep_nops)
    for (size_t k = 0; k < plan->p.tcb.size(); k++) sweep_nops[k] = 1;
  for (size_t k = 0; k < plan->p.op_gate0.size(); k++) {
    if (op_gate) op_gate[k] = plan->p.op_gate0[k];
    if (op_ngates) op_ngates[k] = plan->p.op_ngates[k];
  }
  return NWQ_OK;
}

extern "C" int nwq_plan_tc_blocks(const nwq_plan* plan, int* qubits, double* mats) {
  if (!plan) return fail(NWQ_EINVAL, "plan is NULL");
  if (!plan->p.tc) return fail(NWQ_EINVAL, "not a tensor-core plan");
  for (size_t b = 0; b < plan->p.tcb.size(); b++) {
    const TcBlock& blk = plan->p.tcb[b];
    if (qubits)
      for (int i = 0; i < kTcBits; i++) qubits[b * kTcBits + i] = blk.q[i];
    if (mats)
      for (size_t e = 0; e < blk.U.size(); e++) {
        mats[(b * 1024 + e) * 2] = blk.U[e].real();
        mats[(b * 1024 + e) * 2 + 1] = blk.U[e].imag();
      }
  }
  return NWQ_OK;
}

extern "C" int nwq_plan_ops(const nwq_plan* plan, int* k, int* bits, double* mats) {
  if (!plan) return fail(NWQ_EINVAL, "plan is NULL");
  const Plan& p = plan->p;
  if (p.tc || p.exec_ops.size() != p.ops.size()) return fail(NWQ_EINVAL, "operators are recorded for sweep plans only");
  for (size_t o = 0; o < p.exec_ops.size(); o++) {
    const BitOp& op = p.exec_ops[o];
    const int d = 1 << op.k;
    if (k) k[o] = op.k;
    if (bits)
      for (int t = 0; t < 4; t++) bits[4 * o + t] = t < op.k ? op.bits[t] : -1;
    if (mats)
      for (int r = 0; r < 16; r++)
        for (int c = 0; c < 16; c++) {
          const cd v = (r < d && c < d) ? op.m[(size_t)r * d + c] : cd(0.0);
          mats[(o * 256 + (size_t)r * 16 + c) * 2] = v.real();
          mats[(o * 256 + (size_t)r * 16 + c) * 2 + 1] = v.imag();
        }
  }
  return NWQ_OK;
}

extern "C" int nwq_expect_plan(int n, const nwq_pauli_term* terms, size_t nt, int normalize, int* npass,
                               uint64_t* tile_masks, int* term_range, uint32_t* xl, uint32_t* zl, uint64_t* zh,
                               int* y, int* out, int* nfb, int* fb) {
  if (n < 1 || n > 34) return fail(NWQ_EINVAL, "n must be 1..34");
  if (nt && !terms) return fail(NWQ_EINVAL, "terms is NULL");
  const uint64_t qmask = (1ull << n) - 1;
  for (size_t t = 0; t < nt; t++)
    if ((terms[t].x_mask & ~qmask) || (terms[t].z_mask & ~qmask)) return fail(NWQ_EINVAL, "Pauli mask out of range");
  std::vector<ExpPass> passes(nt + 1);
  std::vector<ExpTerm> eterms(nt + 1);
  std::vector<int> fbv(nt + 1), work(2 * nt + 2);
  std::vector<SvChunk> chunks(nt + 1);
  SvExpectHost h{passes.data(), eterms.data(), fbv.data(), chunks.data(), work.data()};
  SvExpectCounts c{};
  plan_sv_expect(n, terms, nt, normalize != 0, h, c);
  if (npass) *npass = c.npass;
  if (nfb) *nfb = c.nfb;
  for (int p = 0; p < c.npass; p++) {
    const ExpPass& P = passes[p];
    if (tile_masks) tile_masks[p] = ((1ull << P.m) - 1) | P.hmask;
    if (term_range) {
      term_range[2 * p] = P.k0;
      term_range[2 * p + 1] = P.nk;
    }
  }
  for (int r = 0; r < c.nterms; r++) {
    if (xl) xl[r] = eterms[r].xl;
    if (zl) zl[r] = eterms[r].zl;
    if (zh) zh[r] = eterms[r].zh;
    if (y) y[r] = eterms[r].y;
    if (out) out[r] = eterms[r].out;
  }
  if (fb)
    for (int i = 0; i < c.nfb; i++) fb[i] = fbv[i];
  return NWQ_OK;
}

extern "C" int nwq_tc_wait_test(nwq_state* st, const nwq_plan* plan, int* timeouts) {
  if (!st || !plan || !timeouts) return fail(NWQ_EINVAL, "NULL argument");
  Plan& p = const_cast<Plan&>(plan->p);
  if (!p.tc || p.tcg.empty()) return fail(NWQ_EINVAL, "not a tensor-core plan");
  if (p.kind != st->kind || p.n != st->n || p.dtype != st->dtype) return fail(NWQ_EINVAL, "plan does not match state");
  int rc = plan_upload(p, st->stream);
  if (rc) return rc;
  int before = 0, after = 0;
  CK(cudaStreamSynchronize(st->stream), "wait test");
  CK(tc_timeouts(&before), "tensor-core status read");
  const float* tab = (const float*)((const char*)p.dev + p.tc_off);
  CK(launch_tc_block(st->buf, p.tcg[0], tab, st->sm_count, st->stream, true), "tensor-core wait test launch");
  CK(cudaStreamSynchronize(st->stream), "wait test");
  CK(tc_timeouts(&after), "tensor-core status read");
  *timeouts = after - before;
  return *timeouts > 0 ? fail(NWQ_ETIMEOUT, "tensor-core MMA-completion waits ran out (MMAs withheld)") : NWQ_OK;
}

extern "C" int nwq_tc_timeouts(int* count) {
  if (!count) return fail(NWQ_EINVAL, "count is NULL");
  CK(cudaDeviceSynchronize(), "device synchronize");
  CK(tc_timeouts(count), "tensor-core status read");
  return NWQ_OK;
}

extern "C" int nwq_plan_verify(const nwq_plan* plan) {
  if (!plan) return fail(NWQ_EINVAL, "plan is NULL");
  std::string err;
  return verify_plan(plan->p, err) ? NWQ_OK : fail(NWQ_EINVAL, err);
}

extern "C" int nwq_plan_jit_check(const nwq_plan* plan, int* eligible, int* built) {
  if (!plan || !eligible || !built) return fail(NWQ_EINVAL, "NULL argument");
  std::string log;
  jit_build_check(plan->p, eligible, built, &log);
  if (*built < *eligible) return fail(NWQ_EUNSUPPORTED, log.empty() ? "specialised kernel compilation failed" : log);
  return NWQ_OK;
}

extern "C" int nwq_plan_last_run_dw(const nwq_plan* plan, int* dw) {
  if (!plan || !dw) return fail(NWQ_EINVAL, "NULL argument");
  *dw = plan->p.last_run_dw ? 1 : 0;
  return NWQ_OK;
}

extern "C" int nwq_plan_kernel_arith(const nwq_plan* plan, int dw, double* fma_per_elem, double* mul_per_elem,
                                     double* instr_per_elem, int* sweeps) {
  if (!plan || !fma_per_elem || !mul_per_elem || !instr_per_elem) return fail(NWQ_EINVAL, "NULL argument");
  const int e = jit_plan_arith(plan->p, dw != 0, fma_per_elem, mul_per_elem, instr_per_elem);
  if (sweeps) *sweeps = e;
  return NWQ_OK;
}

extern "C" int nwq_plan_jit_prefetch(const nwq_plan* plan, int* pending) {
  if (!plan) return fail(NWQ_EINVAL, "plan is NULL");
  const int q = jit_prefetch(plan->p);
  if (pending) *pending = q;
  return NWQ_OK;
}

extern "C" int nwq_jit_shutdown(void) {
  jit_shutdown();
  return NWQ_OK;
}

extern "C" int nwq_plan_destroy(nwq_plan* plan) {
  delete plan;
  return NWQ_OK;
}

// One-shot circuit: lower, run, and release the tables stream-ordered (the
// host returns without waiting for the sweeps).
static int apply_once(nwq_state* st, int kind, const nwq_gate* gates, size_t ng, const nwq_noise_model* nm,
                      uint32_t flags) {
  nwq_plan* pl = nullptr;
  int rc = nwq_plan_create(kind, st->n, st->dtype, gates, ng, nm, flags, st->stream, &pl);
  if (rc) return rc;
  pl->p.stream_ordered = true;
  rc = nwq_plan_run(st, pl);
  nwq_plan_destroy(pl);
  return rc;
}

extern "C" int nwq_sv_apply_circuit(nwq_state* st, const nwq_gate* gates, size_t ng, uint32_t flags) {
  if (!st) return fail(NWQ_EINVAL, "state is NULL");
  if (st->kind != NWQ_SV) return fail(NWQ_EINVAL, "not a state vector");
  return apply_once(st, NWQ_SV, gates, ng, nullptr, flags);
}

extern "C" int nwq_dm_apply_circuit_noisy(nwq_state* st, const nwq_gate* gates, size_t ng,
                                          const nwq_noise_model* nm, uint32_t flags) {
  if (!st) return fail(NWQ_EINVAL, "state is NULL");
  if (st->kind != NWQ_DM) return fail(NWQ_EINVAL, "not a density matrix");
  return apply_once(st, NWQ_DM, gates, ng, nm, flags);
}

// ------------------------------------------------------------------ measurement
extern "C" int nwq_expect_pauli_sum(nwq_state* st, const nwq_pauli_term* terms, size_t nt, double* out_host,
                                    uint32_t flags) {
  NvtxRange range("nwq expect");
  if (!st || !out_host || (nt && !terms)) return fail(NWQ_EINVAL, "NULL argument");
  if (nt == 0) {
    if (flags & NWQ_EXPECT_SUM) out_host[0] = 0.0;
    return NWQ_OK;
  }
  const uint64_t qmask = st->n >= 64 ? ~0ull : ((1ull << st->n) - 1);
  for (size_t t = 0; t < nt; t++)
    if ((terms[t].x_mask & ~qmask) || (terms[t].z_mask & ~qmask)) return fail(NWQ_EINVAL, "Pauli mask out of range");
  const bool sum = (flags & NWQ_EXPECT_SUM) != 0;
  const bool norm = (flags & NWQ_EXPECT_NORMALIZE) != 0;
  const bool f64 = f64_of(st->dtype);
  cudaStream_t s = st->stream;

  if (st->kind == NWQ_DM) {  // coefficients read as they are, FP64 or double words
    std::vector<uint64_t> h(3 * nt);
    for (size_t t = 0; t < nt; t++) {
      h[t] = terms[t].x_mask;
      h[nt + t] = terms[t].z_mask;
      std::memcpy(&h[2 * nt + t], &terms[t].coeff, 8);
    }
    void* d = nullptr;
    size_t outn = sum ? 1 : nt;
    CK(cudaMallocAsync(&d, h.size() * 8 + outn * 8, s), "scratch allocation");
    uint64_t* dx = (uint64_t*)d;
    double* dout = (double*)(dx + 3 * nt);
    int rc = NWQ_OK;
    cudaError_t e = cudaMemcpyAsync(d, h.data(), h.size() * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = launch_dm_expect(f64, st->buf, st->n, dx, dx + nt, (const double*)(dx + 2 * nt), (int)nt, dout, sum, norm, s,
                           st->dw_resident);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, dout, outn * 8, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "expectation");
    cudaFreeAsync(d, s);
    e = cudaStreamSynchronize(s);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "expectation");
    return rc;
  }

  // SV: tiled passes, then the general kernel for terms no tile can hold.
  std::vector<ExpPass> passes(nt + 1);
  std::vector<ExpTerm> eterms(nt + 1);
  std::vector<int> fb(nt), work(2 * nt + 2);
  std::vector<SvChunk> chunks(nt);
  SvExpectHost h{passes.data(), eterms.data(), fb.data(), chunks.data(), work.data()};
  SvExpectCounts c{};
  plan_sv_expect(st->n, terms, nt, norm, h, c);
  int grid = 0, fblocks = 0;
  sv_expect_shape(st, nt, 0, &grid, &fblocks);
  std::vector<unsigned char> stage(sv_expect_stage_bytes(nt));
  void* d = nullptr;
  CK(cudaMallocAsync(&d, sv_expect_scratch_bytes(nt, grid, fblocks), s), "scratch allocation");
  int rc = NWQ_OK;
  cudaError_t e = sv_expect_enqueue(st, terms, nt, flags, out_host, h, c, grid, fblocks, stage.data(),
                                    (unsigned char*)d);
  if (e != cudaSuccess) rc = cuda_fail(e, "expectation");
  cudaFreeAsync(d, s);
  e = cudaStreamSynchronize(s);
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "expectation");
  return rc;
}

// Real f64 plan over n bits: readout confusion per bit (SV) or the
// Walsh-Hadamard butterfly (DM diagonal from Z-string coefficients).
static nwq_plan* probs_plan(nwq_state* st, double e, bool wht) {
  double key = wht ? -1.0 - e : e;
  auto it = st->probs.find(key);
  if (it != st->probs.end()) return it->second.get();
  auto pl = std::make_unique<nwq_plan>();
  pl->p.stream_ordered = true;
  init_plan_meta(pl->p, NWQ_DM, st->n, NWQ_F64, st->n);  // real f64 elements over n bits
  std::vector<BitOp> ops(st->n);
  for (int q = 0; q < st->n; q++) {
    ops[q].k = 1;
    ops[q].bits[0] = q;
    if (wht) ops[q].m = {1.0, 1.0, 1.0, -1.0};
    else ops[q].m = {1.0 - e, e, e, 1.0 - e};
    ops[q].gate0 = q;
  }
  PlanOptions o;
  plan_options(NWQ_DM, NWQ_F64, NWQ_PLAN_NO_MERGE, o);
  build_plan(ops, o, pl->p);
  nwq_plan* raw = pl.get();
  st->probs[key] = std::move(pl);
  return raw;
}

extern "C" int nwq_probs(nwq_state* st, double readout_e, double* out_host) {
  NvtxRange range("nwq probs");
  if (!st || !out_host) return fail(NWQ_EINVAL, "NULL argument");
  if (st->n > 30) return fail(NWQ_EUNSUPPORTED, "probabilities limited to n <= 30");
  if (!(readout_e >= 0.0 && readout_e <= 0.5)) return fail(NWQ_EINVAL, "readout error outside [0, 0.5]");
  if (st->kind == NWQ_SV)  // density matrices read their diagonal coefficients in either layout
    if (int rc = state_f64(st)) return rc;
  cudaStream_t s = st->stream;
  uint64_t N = 1ull << st->n;
  double* p = nullptr;
  CK(cudaMallocAsync((void**)&p, N * 8, s), "scratch allocation");
  int rc = NWQ_OK;
  cudaError_t e;
  if (st->kind == NWQ_SV) {
    e = launch_sv_abs2(f64_of(st->dtype), st->buf, p, N, st->sm_count, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "probabilities");
    if (!rc && readout_e > 0) rc = plan_launch(probs_plan(st, readout_e, false)->p, p, s, st->sm_count);
  } else {
    e = launch_dm_diag(f64_of(st->dtype), st->buf, p, st->n, readout_e, st->sm_count, s, st->dw_resident);
    if (e != cudaSuccess) rc = cuda_fail(e, "probabilities");
    if (!rc) rc = plan_launch(probs_plan(st, 0.0, true)->p, p, s, st->sm_count);
  }
  if (!rc) {
    e = cudaMemcpyAsync(out_host, p, N * 8, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "probabilities");
  }
  cudaFreeAsync(p, s);
  e = cudaStreamSynchronize(s);
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "probabilities");
  return rc;
}

extern "C" const char* nwq_last_error(void) { return g_err.c_str(); }

extern "C" uint64_t nwq_launch_count(void) { return (uint64_t)g_launches.load(); }

