// Host side of the batched parametrised-circuit evaluation: validation,
// device tables, launches and CUDA-graph replay for repeated runs (a VQE
// optimiser calls the same batch with new parameters every iteration).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/nwqgb.h"
#include "batch.hpp"
#include "kernels.hpp"
#include "nvtx_range.hpp"
#include "planner.hpp"
#include "state.hpp"

using namespace nwq;

struct nwq_batch {
  int dtype = 0, nparams = 0, ntemplates = 0;
  int max_n = 0, max_gates = 0, max_terms = 0, max_ne = 0;
  int device = 0, sm_count = 1;
  void* dev = nullptr;  // tables + work-queue counter
  const BGate* gates = nullptr;
  const BTemplate* templates = nullptr;
  const BTemplate* templates_fused = nullptr;  // the same templates with one-qubit runs fused
  int threads = kBatchThreads, fusion = 0;      // kernel shape (nwq_batch_set_shape)
  const BTerm* terms = nullptr;
  const double* coeffs = nullptr;
  int* counter = nullptr;
  cudaStream_t stream = nullptr;  // tables are allocated and freed stream-ordered here
  // captured launch for repeated runs with the same pointers and job count
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  BatchArgs cap_args{};
};

static bool lower_batch_gate(const nwq_gate& g, int n, int nparams, BGate& b, std::string& err) {
  std::memset(&b, 0, sizeof(b));
  b.pidx = g.param_idx;
  b.q0 = (uint8_t)g.q[0];
  b.q1 = (uint8_t)g.q[1];
  for (int k = 0; k < 3; k++) b.th[k] = g.theta[k];
  bool two = g.kind >= NWQ_GATE_CX;
  if (g.q[0] < 0 || g.q[0] >= n || (two && (g.q[1] < 0 || g.q[1] >= n || g.q[1] == g.q[0]))) {
    err = "gate qubit out of range";
    return false;
  }
  if (g.param_idx >= nparams || g.param_idx < -1) {
    err = "parameter index out of range";
    return false;
  }
  bool param_ok = true;
  switch (g.kind) {
    case NWQ_GATE_CX: b.type = BT_CX; param_ok = false; break;
    case NWQ_GATE_CZ: b.type = BT_CZ; param_ok = false; break;
    case NWQ_GATE_SWAP: b.type = BT_SWAP; param_ok = false; break;
    case NWQ_GATE_RZZ: b.type = BT_RZZ; break;
    case NWQ_GATE_RX: b.type = BT_RX; break;
    case NWQ_GATE_RY: b.type = BT_RY; break;
    case NWQ_GATE_RZ: b.type = BT_RZ; break;
    case NWQ_GATE_P: b.type = BT_P; break;
    case NWQ_GATE_U3: b.type = BT_U3; break;
    case NWQ_GATE_MAT2:
      err = "MAT2 is not supported in batched evaluation";
      return false;
    default: {
      cd U[16];
      if (gate_matrix(g, g.theta[0], U) != 1) {
        err = "unknown gate kind or missing matrix";
        return false;
      }
      b.type = BT_FIXED1;
      param_ok = false;
      bool real = true, diag = U[1] == cd(0.0) && U[2] == cd(0.0);
      for (int k = 0; k < 4; k++) {
        b.m[2 * k] = U[k].real();
        b.m[2 * k + 1] = U[k].imag();
        real &= U[k].imag() == 0.0;
      }
      b.cls = diag ? 2 : (real ? 1 : 0);  // BG_DIAG / BG_REAL / BG_DENSE
    }
  }
  if (!param_ok && g.param_idx >= 0) {
    err = "parameter index on a gate without an angle";
    return false;
  }
  return true;
}

static bool is_one_qubit(const BGate& g) {
  return g.type == BT_FIXED1 || g.type == BT_RX || g.type == BT_RY || g.type == BT_RZ || g.type == BT_P ||
         g.type == BT_U3;
}

// Fusion of one template's gates g[0, ng): each run of one-qubit gates on a
// qubit, up to the next two-qubit gate touching that qubit, becomes one
// BT_FUSED entry at the position of its first gate (the gates it moves past
// act on other qubits, so the order of operations on every qubit is kept).
// members[i] lists the gates of fused entry i (empty for other entries).
static void fuse_runs(const BGate* g, size_t ng, std::vector<BGate>& out, std::vector<std::vector<BGate>>& members) {
  const size_t first = out.size();
  int open[64];
  for (int& o : open) o = -1;
  for (size_t k = 0; k < ng; k++) {
    const BGate& x = g[k];
    if (is_one_qubit(x)) {
      const int q = x.q0;
      if (open[q] >= 0 && members[open[q]].size() < 255) {
        members[open[q]].push_back(x);
      } else {
        BGate f;
        std::memset(&f, 0, sizeof(f));
        f.type = BT_FUSED;
        f.q0 = f.q1 = x.q0;
        f.pidx = -1;
        out.push_back(f);
        members.push_back({x});
        open[q] = (int)(out.size() - 1);
      }
    } else {
      open[x.q0] = open[x.q1] = -1;
      out.push_back(x);
      members.push_back({});
    }
  }
  for (size_t i = first; i < out.size(); i++)
    if (members[i].size() == 1) {  // a run of one gate stays that gate
      out[i] = members[i][0];
      members[i].clear();
    }
}

extern "C" int nwq_batch_create(int dtype, const nwq_batch_template* t, int ntemplates, int nparams,
                                void* stream, nwq_batch** out) {
  if (!out || !t || ntemplates < 1 || nparams < 0) return set_error(NWQ_EINVAL, "bad batch arguments");
  *out = nullptr;
  if (dtype != NWQ_F32 && dtype != NWQ_F64) return set_error(NWQ_EINVAL, "unsupported dtype");
  const int nmax = dtype == NWQ_F64 ? 13 : 14;
  std::vector<BGate> gates;
  std::vector<BTemplate> tmpl;
  std::vector<BTerm> terms;
  std::vector<double> coeffs;
  auto b = std::make_unique<nwq_batch>();
  for (int k = 0; k < ntemplates; k++) {
    const nwq_batch_template& tk = t[k];
    if (tk.n < 1 || tk.n > nmax) return set_error(NWQ_EINVAL, "batch template qubit count outside [1, 13] (F64) / [1, 14] (F32)");
    if ((tk.ngates && !tk.gates) || (tk.nterms && !tk.terms) || tk.ne < 1 || !tk.coeffs)
      return set_error(NWQ_EINVAL, "batch template with NULL tables or no energies");
    BTemplate bt{};
    bt.n = tk.n;
    bt.g0 = (int)gates.size();
    bt.ng = (int)tk.ngates;
    bt.t0 = (int)terms.size();
    bt.nt = (int)tk.nterms;
    bt.c0 = (int)coeffs.size();
    bt.ne = tk.ne;
    std::string err;
    for (size_t i = 0; i < tk.ngates; i++) {
      BGate g;
      if (tk.gates[i].reserved || tk.gates[i].reserved2) return set_error(NWQ_EINVAL, "reserved gate field not 0");
      if (!lower_batch_gate(tk.gates[i], tk.n, nparams, g, err)) return set_error(NWQ_EINVAL, err.c_str());
      gates.push_back(g);
    }
    const uint64_t qmask = (1ull << tk.n) - 1;
    for (size_t i = 0; i < tk.nterms; i++) {
      const nwq_pauli_term& p = tk.terms[i];
      if ((p.x_mask & ~qmask) || (p.z_mask & ~qmask)) return set_error(NWQ_EINVAL, "Pauli mask out of range");
      terms.push_back(BTerm{(uint32_t)p.x_mask, (uint32_t)p.z_mask, __builtin_popcountll(p.x_mask & p.z_mask) & 3, 0});
    }
    coeffs.insert(coeffs.end(), tk.coeffs, tk.coeffs + (size_t)tk.ne * tk.nterms);
    tmpl.push_back(bt);
    b->max_n = std::max(b->max_n, tk.n);
    b->max_gates = std::max(b->max_gates, (int)tk.ngates);
    b->max_terms = std::max(b->max_terms, (int)tk.nterms);
    b->max_ne = std::max(b->max_ne, tk.ne);
  }
  // fused variant: gates = [plain | fused | members of the fused runs]
  std::vector<BGate> fused;
  std::vector<std::vector<BGate>> members;
  std::vector<BTemplate> tmplf = tmpl;
  for (int k = 0; k < ntemplates; k++) {
    tmplf[k].g0 = (int)(gates.size() + fused.size());
    fuse_runs(gates.data() + tmpl[k].g0, (size_t)tmpl[k].ng, fused, members);
    tmplf[k].ng = (int)(gates.size() + fused.size()) - tmplf[k].g0;
  }
  const size_t nplain = gates.size();
  std::vector<BGate> runs;
  for (size_t i = 0; i < fused.size(); i++) {
    if (members[i].empty()) continue;
    fused[i].pidx = (int32_t)(nplain + fused.size() + runs.size());
    fused[i].cls = (uint8_t)members[i].size();
    runs.insert(runs.end(), members[i].begin(), members[i].end());
  }
  gates.insert(gates.end(), fused.begin(), fused.end());
  gates.insert(gates.end(), runs.begin(), runs.end());
  b->dtype = dtype;
  b->nparams = nparams;
  b->ntemplates = ntemplates;
  if (batch_smem_bytes(dtype == NWQ_F64, b->max_n, std::max(b->max_gates, 1), b->max_terms) > (size_t)kBatchMaxSmem)
    return set_error(NWQ_EUNSUPPORTED, "batch state plus gate tables exceed shared memory");
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) return set_error(NWQ_ECUDA, cudaGetErrorString(e));
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t og = 0, ot = al(og + gates.size() * sizeof(BGate)), otf = al(ot + tmpl.size() * sizeof(BTemplate));
  size_t oterm = al(otf + tmplf.size() * sizeof(BTemplate));
  size_t oc = al(oterm + terms.size() * sizeof(BTerm)), ocnt = al(oc + coeffs.size() * sizeof(double));
  size_t total = ocnt + 256;
  b->stream = (cudaStream_t)stream;
  e = cudaMallocAsync(&b->dev, total, b->stream);
  if (e != cudaSuccess) return set_error(NWQ_ENOMEM, "batch table allocation failed");
  char* d = (char*)b->dev;
  const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
  if (!gates.empty()) e = cudaMemcpyAsync(d + og, gates.data(), gates.size() * sizeof(BGate), h2d, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + ot, tmpl.data(), tmpl.size() * sizeof(BTemplate), h2d, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + otf, tmplf.data(), tmplf.size() * sizeof(BTemplate), h2d, b->stream);
  if (e == cudaSuccess && !terms.empty())
    e = cudaMemcpyAsync(d + oterm, terms.data(), terms.size() * sizeof(BTerm), h2d, b->stream);
  if (e == cudaSuccess && !coeffs.empty())
    e = cudaMemcpyAsync(d + oc, coeffs.data(), coeffs.size() * sizeof(double), h2d, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host tables go out of scope
  if (e != cudaSuccess) {
    cudaFreeAsync(b->dev, b->stream);
    return set_error(NWQ_ECUDA, cudaGetErrorString(e));
  }
  b->gates = (const BGate*)(d + og);
  b->templates = (const BTemplate*)(d + ot);
  b->templates_fused = (const BTemplate*)(d + otf);
  b->terms = (const BTerm*)(d + oterm);
  b->coeffs = (const double*)(d + oc);
  b->counter = (int*)(d + ocnt);
  *out = b.release();
  return NWQ_OK;
}

extern "C" int nwq_batch_run(nwq_batch* b, const double* params, const int32_t* job_template, int njobs,
                             double* out, int out_stride, double* norms, void* stream, uint32_t flags) {
  NvtxRange range("nwq batch run");
  if (!b || (njobs > 0 && (!out || (b->nparams > 0 && !params)))) return set_error(NWQ_EINVAL, "NULL argument");
  if (njobs < 0) return set_error(NWQ_EINVAL, "negative job count");
  if (njobs == 0) return NWQ_OK;
  if (out_stride < b->max_ne) return set_error(NWQ_EINVAL, "output stride below the largest energy count");
  if (b->ntemplates > 1 && !job_template) return set_error(NWQ_EINVAL, "several templates need a job_template array");
  BatchArgs a;
  std::memset(&a, 0, sizeof(a));  // compared bytewise against the captured arguments
  a.gates = b->gates;
  a.templates = b->fusion ? b->templates_fused : b->templates;
  a.threads = b->threads;
  a.terms = b->terms;
  a.coeffs = b->coeffs;
  a.params = params;
  a.job_template = job_template;
  a.out = out;
  a.norms = norms;
  a.counter = b->counter;
  a.njobs = njobs;
  a.nparams = b->nparams;
  a.out_stride = out_stride;
  a.ntemplates = b->ntemplates;
  a.max_n = b->max_n;
  a.max_gates = std::max(b->max_gates, 1);
  a.max_terms = b->max_terms;
  cudaStream_t s = (cudaStream_t)stream;
  const bool f64 = b->dtype == NWQ_F64;
  a.dw = f64 && !(flags & NWQ_BATCH_FP64_PIPE);
  if (!(flags & NWQ_BATCH_GRAPH)) {
    cudaError_t e = launch_batch(f64, a, b->sm_count, s);
    return e == cudaSuccess ? NWQ_OK : set_error(NWQ_ECUDA, cudaGetErrorString(e));
  }
  // Replay a captured graph (work-queue reset + launch); recapture when the
  // pointers or the job count differ from the captured ones.
  if (!b->exec || std::memcmp(&b->cap_args, &a, sizeof(a)) != 0) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!b->cap_stream) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    // one direct launch first: kernel attributes are set outside the capture
    if (e == cudaSuccess) e = launch_batch(f64, a, b->sm_count, b->cap_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap_stream);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t el = launch_batch(f64, a, b->sm_count, b->cap_stream);
      e = cudaStreamEndCapture(b->cap_stream, &g);
      if (e == cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return set_error(NWQ_ECUDA, cudaGetErrorString(e));
    b->cap_args = a;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, s);
  if (e == cudaSuccess) g_launches += 1;
  return e == cudaSuccess ? NWQ_OK : set_error(NWQ_ECUDA, cudaGetErrorString(e));
}

extern "C" int nwq_batch_set_shape(nwq_batch* b, int threads, int fusion) {
  if (!b) return set_error(NWQ_EINVAL, "batch is NULL");
  if (threads != 128 && threads != 256 && threads != 512) return set_error(NWQ_EINVAL, "threads must be 128, 256 or 512");
  if (fusion != 0 && fusion != 1) return set_error(NWQ_EINVAL, "fusion must be 0 or 1");
  b->threads = threads;
  b->fusion = fusion;
  return NWQ_OK;
}

extern "C" int nwq_batch_autotune(nwq_batch* b, const double* params, const int32_t* job_template, int njobs,
                                  double* out, int out_stride, int reps, void* stream, int* best_threads,
                                  int* best_fusion, double* best_ms) {
  if (!b || reps < 1 || njobs < 1) return set_error(NWQ_EINVAL, "bad autotune arguments");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_error(NWQ_ECUDA, "event creation failed");
  double bms = -1.0;
  int bt = b->threads, bf = b->fusion;
  int rc = NWQ_OK;
  for (int f = 0; f <= 1 && !rc; f++)
    for (int th : kBatchThreadChoices) {
      b->threads = th;
      b->fusion = f;
      rc = nwq_batch_run(b, params, job_template, njobs, out, out_stride, nullptr, stream, 0);  // warm-up
      if (rc) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && !rc; r++)
        rc = nwq_batch_run(b, params, job_template, njobs, out, out_stride, nullptr, stream, 0);
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = set_error(NWQ_ECUDA, "timing failed");
      if (rc) break;
      if (bms < 0 || ms / reps < bms) {
        bms = ms / reps;
        bt = th;
        bf = f;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->threads = bt;
  b->fusion = bf;
  if (best_threads) *best_threads = bt;
  if (best_fusion) *best_fusion = bf;
  if (best_ms) *best_ms = bms;
  return rc;
}

extern "C" int nwq_batch_destroy(nwq_batch* b) {
  if (!b) return NWQ_OK;
  if (b->cap_stream) cudaStreamSynchronize(b->cap_stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->dev) cudaFreeAsync(b->dev, b->stream);  // after the runs queued on the creation stream
  delete b;
  return NWQ_OK;
}

// ------------------------------------------------------------------ quantum trajectories
// Noise descriptor of every gate (the device noise model of
// nwq_dm_apply_circuit_noisy), or an error.
static int traj_noise(const nwq_gate* g, size_t ng, int n, const nwq_noise_model* nm, std::vector<TNoise>& out,
                      int* draws) {
  out.assign(ng, TNoise{});
  *draws = 0;
  if (!nm) return NWQ_OK;
  if (nm->n < n || !nm->T1_us || !nm->T2_us) return set_error(NWQ_EINVAL, "noise model does not cover the qubits");
  for (size_t i = 0; i < ng; i++) {
    TNoise& T = out[i];
    const bool two = g[i].kind >= NWQ_GATE_CX;
    T.k = two ? 2 : 1;
    if ((nm->flags & NWQ_NOISE_RZ_VIRTUAL) && g[i].kind == NWQ_GATE_RZ) continue;
    const int np = 1 << (2 * T.k);
    double p = two ? nm->p2 : nm->p1;
    if (nm->flags & NWQ_NOISE_DEPOL_PAULI_FORM) p = p * np / (np - 1.0);
    if (p < 0 || p > np / (np - 1.0)) return set_error(NWQ_EINVAL, "depolarising parameter out of range");
    T.pdep = p;
    if (p > 0) *draws += 1;
    const double tns = two ? nm->t2q_ns : nm->t1q_ns;
    if (tns > 0) {
      T.relax = 1;
      for (int w = 0; w < T.k; w++) {
        const int q = g[i].q[w];
        const double T1 = nm->T1_us[q], T2 = nm->T2_us[q];
        if (!(T1 > 0) || !(T2 > 0)) return set_error(NWQ_EINVAL, "T1 and T2 must be positive");
        const double gamma = 1.0 - std::exp(-tns / (T1 * 1e3)), eta = std::exp(-tns / (T2 * 1e3));
        double oml = eta * eta / (1.0 - gamma);
        if (oml > 1.0 + 1e-15) return set_error(NWQ_EINVAL, "trajectories need T2 <= 2 T1 (amplitude plus phase damping)");
        if (oml > 1.0) oml = 1.0;
        T.gamma[w] = gamma;
        T.lambda[w] = 1.0 - oml;
      }
      *draws += 2 * T.k;
    }
  }
  return NWQ_OK;
}

extern "C" int nwq_traj_draws(const nwq_gate* gates, size_t ng, int n, const nwq_noise_model* noise, size_t* draws) {
  if (!draws || (ng && !gates)) return set_error(NWQ_EINVAL, "NULL argument");
  std::vector<TNoise> tn;
  int d = 0;
  int rc = traj_noise(gates, ng, n, noise, tn, &d);
  if (rc) return rc;
  *draws = (size_t)d;
  return NWQ_OK;
}

extern "C" int nwq_traj_run(int n, int dtype, const nwq_gate* gates, size_t ng, const nwq_noise_model* noise,
                            const nwq_pauli_term* terms, size_t nt, const double* coeffs, int ne,
                            const double* uniforms, int ntraj, double* out, void* stream) {
  NvtxRange range("nwq trajectories");
  if ((ng && !gates) || (nt && !terms) || ne < 1 || !coeffs || ntraj < 1 || !out) return set_error(NWQ_EINVAL, "bad trajectory arguments");
  if (dtype != NWQ_F32 && dtype != NWQ_F64) return set_error(NWQ_EINVAL, "unsupported dtype");
  if (n < 1 || n > (dtype == NWQ_F64 ? 13 : 14)) return set_error(NWQ_EINVAL, "trajectory qubit count outside [1, 13] (F64) / [1, 14] (F32)");
  std::vector<BGate> bg(ng);
  std::string err;
  for (size_t i = 0; i < ng; i++) {
    if (gates[i].reserved || gates[i].reserved2) return set_error(NWQ_EINVAL, "reserved gate field not 0");
    if (!lower_batch_gate(gates[i], n, 0, bg[i], err)) return set_error(NWQ_EINVAL, err.c_str());
  }
  std::vector<TNoise> tn;
  int draws = 0;
  int rc = traj_noise(gates, ng, n, noise, tn, &draws);
  if (rc) return rc;
  if (draws > 0 && !uniforms) return set_error(NWQ_EINVAL, "uniforms is NULL");
  const uint64_t qmask = (1ull << n) - 1;
  std::vector<BTerm> bt;
  for (size_t i = 0; i < nt; i++) {
    if ((terms[i].x_mask & ~qmask) || (terms[i].z_mask & ~qmask)) return set_error(NWQ_EINVAL, "Pauli mask out of range");
    bt.push_back(BTerm{(uint32_t)terms[i].x_mask, (uint32_t)terms[i].z_mask,
                       __builtin_popcountll(terms[i].x_mask & terms[i].z_mask) & 3, 0});
  }
  const bool f64 = dtype == NWQ_F64;
  if (traj_smem_bytes(f64, n, (int)ng, (int)nt) > (size_t)kBatchMaxSmem)
    return set_error(NWQ_EUNSUPPORTED, "trajectory state plus gate tables exceed shared memory");
  int dev = 0, sms = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(NWQ_ECUDA, cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t og = 0, on = al(og + bg.size() * sizeof(BGate)), ot = al(on + tn.size() * sizeof(TNoise));
  const size_t oc = al(ot + bt.size() * sizeof(BTerm)), ocnt = al(oc + (size_t)ne * nt * sizeof(double));
  void* d = nullptr;
  if (cudaMallocAsync(&d, ocnt + 256, s) != cudaSuccess) return set_error(NWQ_ENOMEM, "trajectory table allocation failed");
  char* dc = (char*)d;
  const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
  if (!bg.empty()) e = cudaMemcpyAsync(dc + og, bg.data(), bg.size() * sizeof(BGate), h2d, s);
  if (e == cudaSuccess && !tn.empty()) e = cudaMemcpyAsync(dc + on, tn.data(), tn.size() * sizeof(TNoise), h2d, s);
  if (e == cudaSuccess && !bt.empty()) e = cudaMemcpyAsync(dc + ot, bt.data(), bt.size() * sizeof(BTerm), h2d, s);
  if (e == cudaSuccess && nt) e = cudaMemcpyAsync(dc + oc, coeffs, (size_t)ne * nt * sizeof(double), h2d, s);
  if (e == cudaSuccess) {
    TrajArgs a{};
    a.gates = (const BGate*)(dc + og);
    a.noise = (const TNoise*)(dc + on);
    a.terms = (const BTerm*)(dc + ot);
    a.coeffs = (const double*)(dc + oc);
    a.u = uniforms;
    a.out = out;
    a.counter = (int*)(dc + ocnt);
    a.n = n;
    a.ng = (int)ng;
    a.nt = (int)nt;
    a.ne = ne;
    a.draws = draws;
    a.ntraj = ntraj;
    a.threads = 256;
    // FP64 trajectories in double words unless NWQ_DW=0 (read on every call)
    const char* env_dw = std::getenv("NWQ_DW");
    a.dw = f64 && !(env_dw && env_dw[0] == '0');
    e = launch_traj(f64, a, sms, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host tables go out of scope
  cudaFreeAsync(d, s);
  return e == cudaSuccess ? NWQ_OK : set_error(NWQ_ECUDA, cudaGetErrorString(e));
}

extern "C" int nwq_batch_energy(int n, int dtype, const nwq_gate* gates, size_t ng, const double* params, int nsets,
                                int nparams, const nwq_pauli_term* terms, size_t nt, const double* coeffs, int ne,
                                double* out, void* stream) {
  nwq_batch_template t{};
  t.n = n;
  t.gates = gates;
  t.ngates = ng;
  t.terms = terms;
  t.nterms = nt;
  t.coeffs = coeffs;
  t.ne = ne;
  nwq_batch* b = nullptr;
  int rc = nwq_batch_create(dtype, &t, 1, nparams, stream, &b);
  if (rc) return rc;
  rc = nwq_batch_run(b, params, nullptr, nsets, out, ne, nullptr, stream, 0);
  if (!rc) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) rc = set_error(NWQ_ECUDA, cudaGetErrorString(e));
  }
  nwq_batch_destroy(b);
  return rc;
}
