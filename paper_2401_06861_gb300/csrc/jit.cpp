// Run-time specialised phase kernels (NVRTC).
//
// The register-phase kernel interprets each sweep's operator list: for every
// group of 16 amplitudes it reads operator records, branches on their codes
// and derives register offsets from the phase's bit positions.  On large
// complex64 states that interpretation, not the arithmetic and not HBM, bounds
// the sweeps.  This file writes, for each distinct sweep structure, CUDA
// source in which the structure is fixed (tile geometry, register offsets,
// the operator sequence with its masks, forms, permutations and diagonal index
// bits), compiles it once with NVRTC for sm_103a and caches the kernel by its
// source text, so sweeps that differ only in angles share one kernel.
// Coefficients of dense, KRON and register-indexed diagonal operators travel
// in the kernel's parameter bank (read directly as FMA operands); diagonal
// tables indexed by bits outside the registers are staged in shared memory.
// Every operator uses the interpreted kernel's arithmetic in the same order.
#include "jit.hpp"

#include <dlfcn.h>
#include <nvrtc.h>

#include <array>
#include <atomic>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <thread>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <vector>

namespace nwq {

namespace {

constexpr int kJitThreads = 256;
constexpr size_t kParamLimit = 28 * 1024;  // packed coefficients per launch (kernel parameter bank)
constexpr int kDefaultMinBits = 18;        // smaller states: interpreted kernel (no compile latency)

// ------------------------------------------------------------------ NVRTC (loaded on first use)
struct Nvrtc {
  bool ok = false;
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*) = nullptr;
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*) = nullptr;
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*) = nullptr;
  nvrtcResult (*cubin)(nvrtcProgram, char*) = nullptr;
  nvrtcResult (*log_size)(nvrtcProgram, size_t*) = nullptr;
  nvrtcResult (*log)(nvrtcProgram, char*) = nullptr;
  nvrtcResult (*destroy)(nvrtcProgram*) = nullptr;
};

Nvrtc& nvrtc() {
  static Nvrtc N;
  static std::once_flag once;
  std::call_once(once, [] {
    void* h = dlopen("libnvrtc.so.13", RTLD_NOW | RTLD_LOCAL);
    if (!h) h = dlopen("libnvrtc.so", RTLD_NOW | RTLD_LOCAL);
    if (!h) return;
    N.create = (decltype(N.create))dlsym(h, "nvrtcCreateProgram");
    N.compile = (decltype(N.compile))dlsym(h, "nvrtcCompileProgram");
    N.cubin_size = (decltype(N.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
    N.cubin = (decltype(N.cubin))dlsym(h, "nvrtcGetCUBIN");
    N.log_size = (decltype(N.log_size))dlsym(h, "nvrtcGetProgramLogSize");
    N.log = (decltype(N.log))dlsym(h, "nvrtcGetProgramLog");
    N.destroy = (decltype(N.destroy))dlsym(h, "nvrtcDestroyProgram");
    N.ok = N.create && N.compile && N.cubin_size && N.cubin && N.log_size && N.log && N.destroy;
  });
  return N;
}

bool jit_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("NWQ_JIT");
    return !(e && e[0] == '0');
  }();
  return on;
}
bool jit_sync_all() {  // compile one-shot plans' kernels before running them too
  static const bool on = [] {
    const char* e = std::getenv("NWQ_JIT_SYNC");
    return e && e[0] == '1';
  }();
  return on;
}
// __launch_bounds__ minimum resident blocks per SM: NWQ_JIT_MINB, else 3 for
// double-word complex kernels (measured: n = 33 complex128 plan run 4.16 ->
// 3.99 s) and FP32 density-matrix kernels (n = 13: 7.05 -> 6.92 ms per step),
// 2 for the others (double-word DM 28.1 ms per step at 2, 30.2 at 3)
int jit_min_blocks(bool dw_complex, bool fp32_real) {
  static const int env = [] {
    const char* e = std::getenv("NWQ_JIT_MINB");
    const int v = e ? std::atoi(e) : 0;
    return v < 0 ? 0 : (v > 4 ? 4 : v);
  }();
  return env ? env : ((dw_complex || fp32_real) ? 3 : 2);
}
int jit_min_bits() {
  static const int b = [] {
    const char* e = std::getenv("NWQ_JIT_MIN_BITS");
    return e ? std::atoi(e) : kDefaultMinBits;
  }();
  return b;
}

// Register bits of real (density-matrix) phases, 4..6 (NWQ_JIT_REAL_RB for
// FP32 plans, NWQ_JIT_REAL_RB_DW for double-word ones).  FP32 plans take 6:
// two noisy two-qubit operators sharing a qubit fit one phase, which halves
// the shared-memory passes of these shared-memory-bound kernels (n = 13 noisy
// TFIM: 9.18 -> 7.06 ms per step); their kernels run 128 threads per CTA (one
// register group of 64 coefficients per thread).  Double-word plans, bound by
// their arithmetic, keep 4.
int real_register_bits(bool fp32) {
  auto env = [](const char* name, int dflt) {
    const char* e = std::getenv(name);
    const int v = e ? std::atoi(e) : dflt;
    return v < 4 ? 4 : (v > 6 ? 6 : v);
  };
  static const int f32 = env("NWQ_JIT_REAL_RB", 6), f64 = env("NWQ_JIT_REAL_RB_DW", 4);
  return fp32 ? f32 : f64;
}

// ------------------------------------------------------------------ compiled kernels
// One packed parameter range: cnt > 0: coefficients [pc0 + rel, + cnt) of the
// complex table; cnt == 0: the coefficient of entry ent0 + rel of a real plan.
struct RecipeItem {
  uint32_t rel, cnt;
};

// A specialised kernel, cached by the structure of the sweeps it serves.  The
// first sweep of a structure writes its description (source, the packing
// recipe of its parameters, shared memory); later sweeps only pack their own
// coefficients by the recipe.
struct JitKernel {
  std::mutex mu;
  std::atomic<bool> done{false}, ok{false}, queued{false}, described{false};
  cudaLibrary_t lib = nullptr;
  cudaKernel_t k = nullptr;
  std::atomic<int> attr_dev{-1};
  std::string src;
  std::vector<RecipeItem> recipe;
  size_t smem = 0;
  int threads = kJitThreads;
  bool usable = false;  // the generator accepted the structure
};

std::mutex g_cache_mu;
std::map<std::string, std::shared_ptr<JitKernel>> g_cache;
std::atomic<int> g_compiled{0}, g_failed{0};

// Source -> sm_103a cubin (host only; needs no device).
bool compile_cubin(const std::string& src, std::vector<char>& bin, std::string* log) {
  Nvrtc& N = nvrtc();
  if (!N.ok) {
    if (log) *log = "libnvrtc not found";
    return false;
  }
  nvrtcProgram prog;
  if (N.create(&prog, src.c_str(), "nwq_jit_sweep.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) return false;
  // NWQ_JIT_PTXAS=1: the assembler's resource report of every kernel on stderr
  static const bool ptxas_v = [] {
    const char* e = std::getenv("NWQ_JIT_PTXAS");
    return e && e[0] == '1';
  }();
  const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-default-device", "--ptxas-options=-v"};
  bool ok = N.compile(prog, ptxas_v ? 4 : 3, opts) == NVRTC_SUCCESS;
  if (ok && ptxas_v) {
    size_t ls = 0;
    if (N.log_size(prog, &ls) == NVRTC_SUCCESS && ls > 1) {
      std::string l(ls, '\0');
      N.log(prog, &l[0]);
      std::fprintf(stderr, "%s\n", l.c_str());
    }
  }
  if (!ok && log) {
    size_t ls = 0;
    if (N.log_size(prog, &ls) == NVRTC_SUCCESS && ls > 1) {
      log->resize(ls);
      N.log(prog, &(*log)[0]);
    }
  }
  if (ok) {
    size_t sz = 0;
    ok = N.cubin_size(prog, &sz) == NVRTC_SUCCESS && sz > 0;
    if (ok) {
      bin.resize(sz);
      ok = N.cubin(prog, bin.data()) == NVRTC_SUCCESS;
    }
  }
  N.destroy(&prog);
  return ok;
}

bool compile(const std::string& src, JitKernel& jk) {
  std::vector<char> bin;
  if (!compile_cubin(src, bin, nullptr)) return false;
  if (cudaLibraryLoadData(&jk.lib, bin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cudaLibraryGetKernel(&jk.k, jk.lib, "nwq_jit_sweep") != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

void build_kernel(JitKernel& jk) {
  std::lock_guard<std::mutex> lk(jk.mu);
  if (jk.done) return;
  jk.ok = compile(jk.src, jk);
  jk.done = true;
  (jk.ok ? g_compiled : g_failed) += 1;
}

// One background thread compiles kernels queued by one-shot plans; it is
// stopped and joined when the library unloads.
struct AsyncCompiler {
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<JitKernel>> q;
  bool stop = false;
  std::thread th;
  AsyncCompiler() : th([this] { run(); }) {}
  ~AsyncCompiler() { shutdown(); }
  void push(std::shared_ptr<JitKernel> jk) {
    {
      std::lock_guard<std::mutex> lk(mu);
      if (stop) return;  // after shutdown: the kernel stays interpreted
      q.push_back(std::move(jk));
    }
    cv.notify_one();
  }
  void shutdown() {  // drop queued jobs, finish the one in progress, join
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
      q.clear();
    }
    cv.notify_all();
    if (th.joinable()) th.join();
  }
  void run() {
    for (;;) {
      std::shared_ptr<JitKernel> job;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [this] { return stop || !q.empty(); });
        if (stop) return;
        job = std::move(q.front());
        q.pop_front();
      }
      build_kernel(*job);
    }
  }
};
AsyncCompiler& async_compiler() {
  // NVRTC is loaded and has compiled once on this thread (its lazily built
  // state and helper libraries exist) before the compiler thread does, so at
  // exit the compiler is stopped and joined before NVRTC's own teardown runs:
  // exit handlers run in reverse order of registration.
  static AsyncCompiler* ac = [] {
    std::vector<char> bin;
    compile_cubin("extern \"C\" __global__ void nwq_jit_warm() {}\n", bin, nullptr);
    static AsyncCompiler a;
    return &a;
  }();
  return *ac;
}
std::atomic<bool> g_async_started{false};

// Cache entry of a structure key (created empty on first request).
std::shared_ptr<JitKernel> entry_for(const std::string& key) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto& slot = g_cache[key];
  if (!slot) slot = std::make_shared<JitKernel>();
  return slot;
}

// Compile a described entry.  Synchronous: before returning.  Asynchronous:
// queued for the background compiler on first request; until it is ready the
// caller runs the interpreted kernel.
void request_compile(const std::shared_ptr<JitKernel>& jk, bool async) {
  if (jk->done) return;
  if (!async) {
    build_kernel(*jk);
  } else if (!jk->queued.exchange(true)) {
    g_async_started = true;
    async_compiler().push(jk);
  }
}

// ------------------------------------------------------------------ source generation
int popc(unsigned v) { return __builtin_popcount(v); }
int dep4(int v, int mask) {  // deposit v's low bits on mask's set bits
  int out = 0, bit = 0;
  for (int p = 0; p < 4; p++)
    if ((mask >> p) & 1) {
      if ((v >> bit) & 1) out |= 1 << p;
      bit++;
    }
  return out;
}
int pext4(int v, int mask) {  // gather v's bits at mask positions
  int out = 0, bit = 0;
  for (int p = 0; p < 4; p++)
    if ((mask >> p) & 1) {
      if ((v >> p) & 1) out |= 1 << bit;
      bit++;
    }
  return out;
}
// Padded tile layout for es-byte elements: 16 bytes of pad after every 128
// bytes (additive over disjoint index bits; 16-byte vectors stay aligned).
uint32_t swz(int es, uint32_t l) {
  return es == 16 ? l + (l >> 3) : (es == 8 ? l + ((l >> 4) << 1) : l + ((l >> 5) << 2));
}
std::string swz_expr(int es, const std::string& v) {
  return es == 16 ? "(" + v + " + (" + v + " >> 3))"
                  : (es == 8 ? "(" + v + " + ((" + v + " >> 4) << 1))" : "(" + v + " + ((" + v + " >> 5) << 2))");
}
size_t padded_elems(int T) { return ((size_t)1 << T) + ((size_t)1 << T) / 8; }

// Double words (NWQ_PLAN_DW): an FP64 value v as floats h + l, h = v rounded
// to float, l = the rest rounded to float (about 48 significant bits).
void append_dw(std::vector<unsigned char>& out, double v) {
  const float w[2] = {(float)v, (float)(v - (double)(float)v)};
  const unsigned char* b = reinterpret_cast<const unsigned char*>(w);
  out.insert(out.end(), b, b + 8);
}
// Append nbytes of FP64 coefficients, as double words when dw.
void append_coefs(std::vector<unsigned char>& out, const unsigned char* src, size_t nbytes, bool dw) {
  if (!dw) {
    out.insert(out.end(), src, src + nbytes);
    return;
  }
  for (size_t i = 0; i + 8 <= nbytes; i += 8) {
    double v;
    std::memcpy(&v, src + i, 8);
    append_dw(out, v);
  }
}

// Device arithmetic of double words, written into double-word kernels.  The
// product takes the exact error of the high parts' product from an FMA and
// adds the cross terms (Dekker's product with an FMA); the sum of the product
// and c adds the high parts with Knuth's TwoSum (exact) and the low parts in
// float (Joldes, Muller, Popescu 2017, double-word building blocks).  Results
// are not renormalised (no final Fast2Sum): the pair (rounded sum, collected
// error) already represents the value to a few 2^-48 of |a b| + |c|, the next
// operation treats it the same way, and the conversion back to FP64 adds the
// two parts exactly.  The _rn intrinsics keep the compiler from contracting or
// reordering these steps.
constexpr double kDwFmaInstr = 12, kDwMulInstr = 4;  // FP32 instructions of fma() and operator* below
const char* kDwPrelude = R"DW(struct __align__(8) dw {
  float h, l;
  dw() = default;
  __device__ explicit dw(int z) : h((float)z), l(0.f) {}
  __device__ dw(float a, float b) : h(a), l(b) {}
};
__device__ __forceinline__ dw d2w(double x) {
  const float h = __double2float_rn(x);
  return dw(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ dw operator-(dw a) { return dw(-a.h, -a.l); }
__device__ __forceinline__ dw operator*(dw a, dw b) {
  const float ph = __fmul_rn(a.h, b.h);
  float pl = __fmaf_rn(a.h, b.h, -ph);
  pl = __fmaf_rn(a.h, b.l, pl);
  pl = __fmaf_rn(a.l, b.h, pl);
  return dw(ph, pl);
}
__device__ __forceinline__ dw fma(dw a, dw b, dw c) {
  const float ph = __fmul_rn(a.h, b.h);
  float pl = __fmaf_rn(a.h, b.h, -ph);
  pl = __fmaf_rn(a.h, b.l, pl);
  pl = __fmaf_rn(a.l, b.h, pl);
  const float s = __fadd_rn(ph, c.h);
  const float v = __fsub_rn(s, ph);
  const float e = __fadd_rn(__fsub_rn(ph, __fsub_rn(s, v)), __fsub_rn(c.h, v));
  return dw(s, __fadd_rn(e, __fadd_rn(pl, c.l)));
}
)DW";

struct Gen {
  const Plan& p;
  const SweepDesc& sd;
  bool c128;
  size_t cs;                        // bytes per coefficient
  std::vector<unsigned char> param; // packed coefficients
  std::vector<RecipeItem> recipe;   // where they came from (relative to the sweep)
  struct Tab {
    uint32_t src, cnt, dst;  // sweep-relative source index, count, shared-memory index
  };
  std::vector<Tab> tabs;
  uint32_t ntab = 0;
  std::ostringstream o;
  bool ok = true;

  // complex plans: complex64 / complex128 elements; real (density-matrix)
  // plans: FP64 elements.  8-byte elements share the complex64 tile layout.
  bool real;
  Gen(const Plan& p_, const SweepDesc& sd_, bool dw_)
      : p(p_),
        sd(sd_),
        c128(p_.is_complex && p_.dtype == NWQ_F64),
        cs(p_.is_complex ? (c128 ? 16 : 8) : (p_.dtype == NWQ_F64 ? 8 : 4)),
        real(!p_.is_complex),
        es((int)cs),
        dw(dw_ && p_.dtype == NWQ_F64) {}
  int es;   // bytes per state element (= per coefficient)
  bool dw;  // FP64 values as double words (two floats), FP32-pipe arithmetic
  int rrb = 4;          // register bits of real phases
  int th = kJitThreads;  // threads per CTA

  uint32_t pack_real(size_t entry, double v) {  // one real coefficient (entry index of the plan)
    uint32_t at = (uint32_t)(param.size() / cs);
    if (es == 8 && dw) {
      append_dw(param, v);
    } else if (es == 8) {
      const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
      param.insert(param.end(), b, b + 8);
    } else {
      const float f = (float)v;  // exact: the entry holds a float
      const unsigned char* b = reinterpret_cast<const unsigned char*>(&f);
      param.insert(param.end(), b, b + 4);
    }
    recipe.push_back({(uint32_t)(entry - sd.ent0), 0});
    return at;
  }

  // Real operator (DevOp rows + entries) on the register bits u[0..3]: every
  // output row is its unit entry (+-input or 0) followed by one FMA per
  // remaining entry, in the row kernel's order; identity rows cost nothing.
  void op_real(const DevOp& d, const uint8_t* u) {
    auto regbit = [&](int pos) {
      for (int q = 0; q < rrb; q++)
        if (u[q] == pos) return q;
      return -1;
    };
    auto reg = [&](uint32_t off) {  // register index of a tile-local offset over the operator bits
      uint32_t x = 0;
      for (int q = 0; q < rrb; q++)
        if ((off >> u[q]) & 1u) x |= 1u << q;
      return x;
    };
    const int NRR = 1 << rrb;
    if (d.k < 1 || d.k > 4) {
      ok = false;
      return;
    }
    uint32_t rmask = 0;
    for (int t = 0; t < d.k; t++) {
      const int q = regbit(d.lb[t]);
      if (q < 0) {
        ok = false;
        return;
      }
      rmask |= 1u << q;
    }
    const int D = 1 << d.k;
    const size_t esz = p.ent_bytes;
    for (int ob = 0; ob < NRR; ob++) {
      if (ob & rmask) continue;
      o << "    {";
      for (int s = 0; s < NRR; s++)
        if ((s & ~(int)rmask) == 0) o << " const R t" << (ob | s) << " = " << r(ob | s) << ";";
      o << "\n";
      for (int i = 0; i < D; i++) {
        const RowMeta& rm = d.row[i];
        if (rm.kind == ROW_ID) continue;
        std::string ex = rm.base == 0 ? std::string("R(0)")
                                      : (rm.base == 1 ? "t" : "-t") + std::to_string(ob | reg(rm.boff));
        if (rm.kind == ROW_GEN) {
          for (int e = 0; e < rm.cnt[0]; e++) {
            const size_t at = ((size_t)d.ent + rm.beg + e) * esz;
            if (at + esz > p.ents.size()) {
              ok = false;
              return;
            }
            double c;
            uint32_t off;
            if (es == 8) {
              std::memcpy(&c, &p.ents[at], 8);
            } else {
              float f;
              std::memcpy(&f, &p.ents[at], 4);
              c = f;
            }
            std::memcpy(&off, &p.ents[at + es], 4);
            ex = "fma(" + K(pack_real((size_t)d.ent + rm.beg + e, c)) + ", t" + std::to_string(ob | reg(off)) + ", " +
                 ex + ")";
          }
        }
        o << "      " << r(ob | reg(rm.out)) << " = " << ex << ";\n";
      }
      o << "    }\n";
    }
  }

  // Register phases of a real sweep: consecutive operators while their bits
  // fit rrb register bits (padded with the lowest unused tile bits).
  bool real_phases(std::vector<std::pair<std::array<uint8_t, 6>, std::vector<int>>>& out) {
    uint32_t U = 0;
    std::vector<int> cur;
    auto flush = [&]() {
      if (cur.empty()) return;
      for (int b = 0; b < sd.T && __builtin_popcount(U) < rrb; b++) U |= 1u << b;
      std::array<uint8_t, 6> u{};
      int q = 0;
      for (int b = 0; b < sd.T; b++)
        if ((U >> b) & 1u) u[q++] = (uint8_t)b;
      out.emplace_back(u, cur);
      cur.clear();
      U = 0;
    };
    for (int o2 = 0; o2 < sd.nops; o2++) {
      const DevOp& d = p.ops[sd.op0 + o2];
      if (d.k < 1 || d.k > 4) return false;
      uint32_t bits = 0;
      for (int t = 0; t < d.k; t++) bits |= 1u << d.lb[t];
      if (__builtin_popcount(U | bits) > rrb) flush();
      U |= bits;
      cur.push_back(o2);
    }
    flush();
    return true;
  }

  // Pack cnt coefficients starting at absolute index a; returns the packed index.
  uint32_t pack(uint32_t a, uint32_t cnt) {
    if ((size_t)(a + cnt) * cs > p.pcoef.size()) {
      ok = false;
      return 0;
    }
    uint32_t at = (uint32_t)(param.size() / cs);
    append_coefs(param, &p.pcoef[(size_t)a * cs], (size_t)cnt * cs, dw);
    recipe.push_back({a - sd.pc0, cnt});
    return at;
  }
  uint32_t table(uint32_t a, uint32_t cnt) {
    if ((size_t)(a + cnt) * cs > p.pcoef.size() || a < sd.pc0) {
      ok = false;
      return 0;
    }
    tabs.push_back({a - sd.pc0, cnt, ntab});
    ntab += cnt;
    return ntab - cnt;
  }

  std::string K(uint32_t i) { return "K.c[" + std::to_string(i) + "]"; }
  std::string r(int i) { return "r" + std::to_string(i); }

  // Dense operator on register mask M (form f), coefficients at packed index pb.
  void dense(int NR, int M, int f, uint32_t pb) {
    const int D = 1 << popc(M);
    for (int ob = 0; ob < NR; ob++) {
      if (ob & M) continue;
      o << "    {";
      for (int j = 0; j < D; j++) o << " const C i" << j << " = " << r(ob | dep4(j, M)) << ";";
      o << "\n";
      if (f == PD_XROT) {
        o << "      " << r(ob) << " = C{fma(" << K(pb) << ".x, i0.x, -" << K(pb + 1) << ".y * i1.y), fma(" << K(pb)
          << ".x, i0.y, " << K(pb + 1) << ".y * i1.x)};\n";
        o << "      " << r(ob | M) << " = C{fma(" << K(pb + 3) << ".x, i1.x, -" << K(pb + 2) << ".y * i0.y), fma("
          << K(pb + 3) << ".x, i1.y, " << K(pb + 2) << ".y * i0.x)};\n";
      } else if (f == PD_XROTU) {  // unit diagonal: 4 FMA per pair
        o << "      " << r(ob) << " = C{fma(-" << K(pb + 1) << ".y, i1.y, i0.x), fma(" << K(pb + 1)
          << ".y, i1.x, i0.y)};\n";
        o << "      " << r(ob | M) << " = C{fma(-" << K(pb + 2) << ".y, i0.y, i1.x), fma(" << K(pb + 2)
          << ".y, i0.x, i1.y)};\n";
      } else {
        for (int i = 0; i < D; i++) {
          o << "      { C a{R(0), R(0)};";
          for (int j = 0; j < D; j++) {
            const std::string c = K(pb + i * D + j);
            if (f == PD_REAL)
              o << " a.x = fma(" << c << ".x, i" << j << ".x, a.x); a.y = fma(" << c << ".x, i" << j << ".y, a.y);";
            else
              o << " a.x = fma(" << c << ".x, i" << j << ".x, fma(-" << c << ".y, i" << j << ".y, a.x)); a.y = fma("
                << c << ".x, i" << j << ".y, fma(" << c << ".y, i" << j << ".x, a.y));";
          }
          o << " " << r(ob | dep4(i, M)) << " = a; }\n";
        }
      }
      o << "    }\n";
    }
  }

  void op(int NR, const PhaseOp& po) {
    const int code = po.code;
    if (code < 16) {  // diagonal, register part SU
      const int SU = code, ks = popc(SU);
      if (SU >= NR || po.dnu > 8) {
        ok = false;
        return;
      }
      if (po.dnu == 0) {
        const uint32_t pb = pack(po.coef, 1u << ks);
        for (int i = 0; i < NR; i++)
          o << "    { const C f = " << K(pb + pext4(i, SU)) << "; const C v = " << r(i) << "; " << r(i)
            << " = C{fma(f.x, v.x, -f.y * v.y), fma(f.x, v.y, f.y * v.x)}; }\n";
      } else {
        const uint32_t tb = table(po.coef, 1u << (ks + po.dnu));
        o << "    { unsigned ig = 0u";
        for (int t = 0; t < po.dnu; t++) o << " | (((gb >> " << (int)po.dpos[t] << ") & 1u) << " << t << ")";
        o << ";\n      const C* dg = dtab + " << tb << " + (ig << " << ks << ");\n";
        for (int i = 0; i < NR; i++)
          o << "      { const C f = dg[" << pext4(i, SU) << "]; const C v = " << r(i) << "; " << r(i)
            << " = C{fma(f.x, v.x, -f.y * v.y), fma(f.x, v.y, f.y * v.x)}; }\n";
        o << "    }\n";
      }
      return;
    }
    if (code == PCODE_KRON) {
      for (int P = 0; P < 4; P++) {
        if (!((po.mask >> P) & 1)) continue;
        if ((1 << P) >= NR) {
          ok = false;
          return;
        }
        const uint32_t pb = pack(po.coef + 4 * P, 4);
        dense(NR, 1 << P, (po.form >> (2 * P)) & 3, pb);
      }
      return;
    }
    const int M = code & 15, cls = code >> 4;
    if (M == 0 || M >= NR || popc(M) > 2 || cls > 4) {
      ok = false;
      return;
    }
    if (cls == 1) {  // signed permutation: register moves and negations only
      const int D = 1 << popc(M);
      for (int ob = 0; ob < NR; ob++) {
        if (ob & M) continue;
        o << "    {";
        for (int j = 0; j < D; j++) o << " const C i" << j << " = " << r(ob | dep4(j, M)) << ";";
        for (int i = 0; i < D; i++) {
          const int src = po.perm[i] & 15;
          if (src >= D) {
            ok = false;
            return;
          }
          if (po.perm[i] & 0x80) o << " " << r(ob | dep4(i, M)) << " = C{-i" << src << ".x, -i" << src << ".y};";
          else o << " " << r(ob | dep4(i, M)) << " = i" << src << ";";
        }
        o << " }\n";
      }
      return;
    }
    const int form = cls == 2 ? PD_GEN : (cls == 3 ? PD_REAL : PD_XROT);
    const int D = 1 << popc(M);
    if (form == PD_XROT && D != 2) {
      ok = false;
      return;
    }
    dense(NR, M, form, pack(po.coef, (uint32_t)(D * D)));
  }

  bool run(std::string& src) {
    rrb = real ? real_register_bits(es == 4) : 4;
    const int T = sd.T, m = sd.m, h = sd.h, RB = real ? rrb : sd.prb, NR = 1 << RB;
    const int lvpe = es == 16 ? 0 : (es == 8 ? 1 : 2);
    if (RB < 1 || RB > (real ? 6 : 4) || T < RB || T > 13 || m < lvpe || m + h != T || p.B - T > 24) return false;
    if (real && p.ent_bytes != (p.dtype == NWQ_F64 ? 16u : 8u)) return false;
    const size_t PE = padded_elems(T);
    const uint32_t NG = 1u << (T - RB);
    // wider real phases: one register group per thread in CTAs of 128
    th = (real && rrb > 4 && NG < (uint32_t)kJitThreads) ? 128 : kJitThreads;
    std::vector<std::pair<std::array<uint8_t, 6>, std::vector<int>>> rph;
    if (real && !real_phases(rph)) return false;
    const uint32_t nphase = real ? (uint32_t)rph.size() : sd.nph;
    std::ostringstream body;
    o.swap(body);
    for (uint32_t ph = 0; ph < nphase && ok; ph++) {
      PhaseDesc P{};
      uint8_t ub[6] = {0, 0, 0, 0, 0, 0};  // tile bit of register bit b
      if (real) {
        for (int q = 0; q < RB; q++) ub[q] = rph[ph].first[q];
      } else {
        P = p.phases[sd.ph0 + ph];
        for (int q = 0; q < 4; q++) ub[q] = P.u[q];
      }
      o << "    // phase " << ph << "\n";
      o << "    for (unsigned g = threadIdx.x; g < " << NG << "u; g += " << th << "u) {\n";
      o << "    unsigned gb = g;\n";
      for (int t = 0; t < RB; t++) {
        const uint32_t lowm = (1u << ub[t]) - 1u;
        o << "    gb = ((gb & " << (~lowm) << "u) << 1) | (gb & " << lowm << "u);\n";
      }
      o << "    C* gt = tile + " << swz_expr(es, "gb") << ";\n";
      uint32_t roff[64];
      for (int i = 0; i < NR; i++) {
        uint32_t l = 0;
        for (int b = 0; b < RB; b++)
          if ((i >> b) & 1) l |= 1u << ub[b];
        roff[i] = swz(es, l);
      }
      // Registers on the tile's lowest bits are consecutive elements: VW of
      // them (16 bytes at most) move as one vector access, 16-byte aligned
      // (gb and the offsets have those bits clear; the row padding keeps
      // runs of VW inside one 128-byte row).
      const int VW = (16 / es >= 4 && RB >= 2 && ub[0] == 0 && ub[1] == 1) ? 4
                     : (16 / es >= 2 && RB >= 1 && ub[0] == 0) ? 2 : 1;
      for (int i = 0; i < NR; i += VW) {
        if (VW == 1) {
          o << "    C " << r(i) << " = gt[" << roff[i] << "];\n";
          continue;
        }
        o << "    C";
        for (int k = 0; k < VW; k++) o << (k ? ", " : " ") << r(i + k);
        o << "; { const Vec" << VW << " v = *reinterpret_cast<const Vec" << VW << "*>(gt + " << roff[i] << ");";
        for (int k = 0; k < VW; k++) o << " " << r(i + k) << " = v.e[" << k << "];";
        o << " }\n";
      }
      const std::string before = o.str();
      if (real) {
        for (int oi : rph[ph].second) op_real(p.ops[sd.op0 + oi], ub);
      } else {
        for (uint32_t q = 0; q < P.nops && ok; q++) op(NR, p.pops[P.op0 + q]);
      }
      {  // arithmetic of one register group (NR elements): every fma( and every " * "
        const std::string code = o.str().substr(before.size());
        size_t nf = 0, nm = 0;
        for (size_t at = code.find("fma("); at != std::string::npos; at = code.find("fma(", at + 4)) nf++;
        for (size_t at = code.find(" * "); at != std::string::npos; at = code.find(" * ", at + 3)) nm++;
        fma_per_elem += (double)nf / NR;
        mul_per_elem += (double)nm / NR;
      }
      for (int i = 0; i < NR; i += VW) {
        if (VW == 1) {
          o << "    gt[" << roff[i] << "] = " << r(i) << ";\n";
          continue;
        }
        o << "    { Vec" << VW << " v;";
        for (int k = 0; k < VW; k++) o << " v.e[" << k << "] = " << r(i + k) << ";";
        o << " *reinterpret_cast<Vec" << VW << "*>(gt + " << roff[i] << ") = v; }\n";
      }
      o << "    }\n    __syncthreads();\n";
    }
    if (!ok) return false;
    if (param.size() > kParamLimit) return false;
    o.swap(body);
    const size_t npk = param.empty() ? 1 : param.size() / cs;
    const size_t hoff_byte = ((2 * PE + ntab) * cs + 15) & ~(size_t)15;
    const size_t btab_byte = hoff_byte + ((size_t)8 << h);  // 4 x 2^pb tile-base pieces
    const int F = p.B - T, pb = F <= 4 ? 1 : (F + 3) / 4;     // tile-index bits per piece
    const uint32_t nb = 1u << pb;
    smem = btab_byte + 4 * (size_t)nb * 8;
    if (smem > (size_t)kMaxDynSmem) return false;
    if (dw) {
      o << kDwPrelude << "typedef dw R;\n";
      if (real) o << "typedef dw C;\n";
      else o << "struct __align__(16) C { dw x, y; };\n";
      o << "typedef " << (real ? "double" : "double2") << " CT;\n";  // FP64 diagonal tables in global memory
      o << "__device__ __forceinline__ C from_table(CT v) { return " << (real ? "d2w(v)" : "C{d2w(v.x), d2w(v.y)}")
        << "; }\n";
    } else {
      const char* RT = (c128 || (real && es == 8)) ? "double" : "float";
      const char* CT = real ? RT : (c128 ? "double2" : "float2");
      o << "typedef " << RT << " R;\ntypedef " << CT << " C;\ntypedef C CT;\n"
        << "__device__ __forceinline__ C from_table(CT v) { return v; }\n";
    }
    o << "struct Coef { C c[" << npk << "]; };\n"
      << "struct __align__(2 * sizeof(C)) Vec2 { C e[2]; };\n"
      << "struct __align__(4 * sizeof(C) <= 16 ? 4 * sizeof(C) : 16) Vec4 { C e[4]; };\n"
      << "__device__ __forceinline__ unsigned long long dep(unsigned long long v, unsigned long long mask) {\n"
      << "  unsigned long long out = 0;\n"
      << "  while (v && mask) { unsigned long long lb = mask & (~mask + 1ull); if (v & 1ull) out |= lb; v >>= 1; mask ^= lb; }\n"
      << "  return out;\n}\n"
      << "__device__ __forceinline__ void cpa16(void* s, const void* g) {\n"
      << "  unsigned a = (unsigned)__cvta_generic_to_shared(s);\n"
      << "  asm volatile(\"cp.async.cg.shared.global [%0], [%1], 16;\\n\" :: \"r\"(a), \"l\"(g) : \"memory\");\n}\n"
      << "extern \"C\" __global__ void __launch_bounds__(" << th << ", " << jit_min_blocks(dw && !real, real && es == 4)
      << ") nwq_jit_sweep(C* __restrict__ state, "
      << "unsigned long long ntiles, unsigned long long hmask, unsigned long long fmask, const CT* __restrict__ pcs, "
      << "const Coef K) {\n"
      << "  extern __shared__ __align__(16) unsigned char sm[];\n"
      << "  C* tile = (C*)sm;\n  C* ntile = tile + " << PE << ";\n  C* dtab = tile + " << 2 * PE << ";\n"
      << "  unsigned long long* hoff = (unsigned long long*)(sm + " << hoff_byte << ");\n"
      << "  unsigned long long* btab = (unsigned long long*)(sm + " << btab_byte << ");\n"
      << "  for (unsigned j = threadIdx.x; j < " << (1u << h) << "u; j += " << th << "u) hoff[j] = dep(j, hmask);\n"
      << "  // tile base = OR of 4 pieces, each depositing " << pb << " bits of the tile index on fmask\n"
      << "  for (unsigned j = threadIdx.x; j < " << 4 * nb << "u; j += " << th
      << "u) btab[j] = dep((unsigned long long)(j & " << nb - 1 << "u) << (" << pb << "u * (j >> " << pb
      << ")), fmask);\n";
    for (const Tab& t : tabs)
      o << "  for (unsigned j = threadIdx.x; j < " << t.cnt << "u; j += " << th << "u) dtab[" << t.dst
        << " + j] = from_table(pcs[" << t.src << " + j]);\n";
    const int VPE = 16 / es, lvpc = m - lvpe;
    const uint32_t nvec = (1u << T) / VPE;
    const uint32_t NVT = (nvec + th - 1) / th;  // vectors per thread
    const bool ragged = nvec % th != 0;
    // per-thread vector offsets inside a tile (global) and shared-memory slots
    // (swz is additive over the disjoint bits of threadIdx.x * VPE and 256 * i * VPE).
    // The global offsets are read from the shared table where used, once per
    // tile copy, rather than held in 64-bit registers across the tile loop (the
    // registers go to the phases); the copy guard covers threads past the last vector.
    o << "  __syncthreads();\n"
      << "  const unsigned s0 = " << swz_expr(es, "(threadIdx.x * " + std::to_string(VPE) + "u)") << ";\n";
    for (uint32_t i = 0; i < NVT; i++) {
      const std::string v = "(threadIdx.x + " + std::to_string(i * th) + "u)";
      o << "#define o" << i << " (hoff[" << v << " >> " << lvpc << "] + (unsigned long long)(" << v << " & "
        << ((1u << lvpc) - 1u) << "u) * " << VPE << ")\n";
    }
    auto sidx = [&](uint32_t i) { return std::to_string(swz(es, i * th * VPE)); };
    auto guard = [&](uint32_t i) -> std::string {
      return (ragged && i == NVT - 1) ? "if (threadIdx.x + " + std::to_string(i * th) + "u < " +
                                            std::to_string(nvec) + "u) "
                                      : "";
    };
    auto base_of = [&](const char* t) {
      std::string s = "(";
      for (int q = 0; q < 4; q++) {
        if (q) s += " | ";
        s += "btab[" + std::to_string(q * nb) + "u + ((" + t + " >> " + std::to_string(q * pb) + ") & " +
             std::to_string(nb - 1) + "u)]";
      }
      return s + ")";
    };
    o << "  if (blockIdx.x < ntiles) {\n"
      << "    const unsigned long long tb = blockIdx.x;\n"
      << "    const unsigned long long b = " << base_of("tb") << ";\n";
    for (uint32_t i = 0; i < NVT; i++)
      o << "    " << guard(i) << "cpa16(tile + s0 + " << sidx(i) << ", state + b + o" << i << ");\n";
    o << "    asm volatile(\"cp.async.commit_group;\\n\" ::: \"memory\");\n  }\n"
      << "  for (unsigned long long tileid = blockIdx.x; tileid < ntiles; tileid += gridDim.x) {\n"
      << "    const unsigned long long base = " << base_of("tileid") << ";\n"
      << "    const unsigned long long next = tileid + gridDim.x;\n"
      << "    if (next < ntiles) {\n"
      << "      const unsigned long long nb = " << base_of("next") << ";\n";
    for (uint32_t i = 0; i < NVT; i++)
      o << "      " << guard(i) << "cpa16(ntile + s0 + " << sidx(i) << ", state + nb + o" << i << ");\n";
    o << "      asm volatile(\"cp.async.commit_group;\\n\" ::: \"memory\");\n"
      << "      asm volatile(\"cp.async.wait_group 1;\\n\" ::: \"memory\");\n"
      << "    } else {\n"
      << "      asm volatile(\"cp.async.wait_group 0;\\n\" ::: \"memory\");\n"
      << "    }\n"
      << "    __syncthreads();\n"
      << body.str();
    for (uint32_t i = 0; i < NVT; i++)
      o << "    " << guard(i) << "*reinterpret_cast<uint4*>(state + base + o" << i
        << ") = *reinterpret_cast<const uint4*>(tile + s0 + " << sidx(i) << ");\n";
    o << "    __syncthreads();\n"
      << "    C* t = tile; tile = ntile; ntile = t;\n"
      << "  }\n"
      << "  asm volatile(\"cp.async.wait_group 0;\\n\" ::: \"memory\");\n"
      << "}\n";
    src = o.str();
    return true;
  }
  size_t smem = 0;
  // arithmetic per state element of this sweep, counted on the emitted source:
  // multiply-adds and multiplies of R values (one FP64 instruction each; a
  // double-word multiply-add is 12 FP32 instructions, a multiply 4)
  double fma_per_elem = 0.0, mul_per_elem = 0.0;
};

// Structure key of a sweep: everything the generator reads except coefficient
// values (tile geometry, register bits, operator codes, masks, forms, index
// bits and permutations, coefficient positions relative to the sweep; for
// real plans the operator rows and entry offsets).  Sweeps with equal keys
// get identical kernel source.
std::string struct_key(const Plan& p, const SweepDesc& sd, bool dw) {
  std::string key;
  auto put = [&](const void* d, size_t n) { key.append(reinterpret_cast<const char*>(d), n); };
  const int32_t hdr[9] = {p.is_complex ? 1 : 0, p.dtype, p.B - sd.T, sd.T, sd.m, sd.h,
                          p.is_complex ? sd.prb : real_register_bits(p.dtype == NWQ_F32 && !dw),
                          jit_min_blocks(dw && p.is_complex && p.dtype == NWQ_F64,
                                         !p.is_complex && p.dtype == NWQ_F32),
                          dw ? 1 : 0};
  put(hdr, sizeof(hdr));
  if (p.is_complex) {
    for (uint32_t ph = 0; ph < sd.nph; ph++) {
      const PhaseDesc& P = p.phases[sd.ph0 + ph];
      put(P.u, sizeof(P.u));
      put(&P.nops, sizeof(P.nops));
      for (uint32_t q = 0; q < P.nops; q++) {
        const PhaseOp& o = p.pops[P.op0 + q];
        const uint8_t f[6] = {o.cls, o.k, o.mask, o.form, o.code, o.dnu};
        put(f, sizeof(f));
        put(o.dpos, sizeof(o.dpos));
        put(o.perm, sizeof(o.perm));
        const uint32_t rel = o.coef - sd.pc0;
        put(&rel, sizeof(rel));
      }
    }
  } else {
    for (int oi = 0; oi < sd.nops; oi++) {
      const DevOp& d = p.ops[sd.op0 + oi];
      put(&d.k, 1);
      put(d.lb, sizeof(d.lb));
      for (int i = 0; i < (1 << d.k) && i < 16; i++) {
        const RowMeta& rm = d.row[i];
        put(&rm, sizeof(RowMeta));
        if (rm.kind != ROW_GEN) continue;
        for (int e = 0; e < rm.cnt[0]; e++) {
          const size_t at = ((size_t)d.ent + rm.beg + e) * p.ent_bytes + (p.dtype == NWQ_F64 ? 8 : 4);
          if (at + 4 <= p.ents.size()) key.append(reinterpret_cast<const char*>(&p.ents[at]), 4);  // entry offset
        }
      }
    }
  }
  return key;
}

// Write the entry's description from this sweep (once per structure).
bool describe(JitKernel& jk, const Plan& p, const SweepDesc& sd, bool dw) {
  if (jk.described) return jk.usable;
  std::lock_guard<std::mutex> lk(jk.mu);  // never held by a compile here: compiles need a description
  if (!jk.described) {
    Gen g(p, sd, dw);
    std::string src;
    jk.usable = g.run(src);
    if (jk.usable) {
      jk.src = std::move(src);
      jk.recipe = std::move(g.recipe);
      jk.smem = g.smem;
      jk.threads = g.th;
    }
    jk.described = true;
  }
  return jk.usable;
}

// This sweep's parameter bytes by the structure's recipe (empty on a range error).
std::vector<unsigned char> pack_params(const Plan& p, const SweepDesc& sd, const std::vector<RecipeItem>& recipe,
                                       bool dw) {
  const size_t cs = p.is_complex ? (p.dtype == NWQ_F64 ? 16 : 8) : (p.dtype == NWQ_F64 ? 8 : 4);
  dw = dw && p.dtype == NWQ_F64;
  std::vector<unsigned char> out;
  for (const RecipeItem& it : recipe) {
    if (it.cnt) {
      const size_t a = (size_t)sd.pc0 + it.rel;
      if ((a + it.cnt) * cs > p.pcoef.size()) return {};
      append_coefs(out, &p.pcoef[a * cs], it.cnt * cs, dw);
    } else {
      const size_t at = ((size_t)sd.ent0 + it.rel) * p.ent_bytes;
      if (at + cs > p.ents.size()) return {};
      append_coefs(out, &p.ents[at], cs, dw);
    }
  }
  if (out.empty()) out.resize(cs, 0);
  return out;
}

// Per-plan state: one entry per sweep, built on the plan's first launch.
struct JitSweep {
  std::shared_ptr<JitKernel> k;  // null: run the interpreted kernel
  std::vector<unsigned char> param;
  size_t smem = 0;
  int per_sm = 0;
};
struct JitPlan {  // [0]: kernels in the plan's own precision, [1]: double-word kernels
  std::mutex mu;
  bool built[2] = {false, false};
  std::vector<JitSweep> sw[2];
};

}  // namespace

bool jit_source(const Plan& p, size_t sweep, std::string& src, size_t* param_bytes, size_t* smem_bytes) {
  src.clear();
  if (sweep >= p.sweeps.size() || p.sweeps[sweep].nops == 0 || (p.is_complex && p.sweeps[sweep].nph == 0))
    return false;
  Gen g(p, p.sweeps[sweep], p.dw);
  if (!g.run(src)) {
    src.clear();
    return false;
  }
  if (param_bytes) *param_bytes = g.param.size();
  if (smem_bytes) *smem_bytes = g.smem;
  return true;
}

int jit_build_check(const Plan& p, int* eligible, int* built, std::string* log) {
  *eligible = *built = 0;
  std::map<std::string, bool> seen;  // one compile per distinct structure, as at run time
  for (size_t i = 0; i < p.sweeps.size(); i++) {
    std::string src;
    if (!jit_source(p, i, src, nullptr, nullptr)) continue;
    (*eligible)++;
    auto it = seen.find(src);
    if (it == seen.end()) {
      std::vector<char> bin;
      it = seen.emplace(src, compile_cubin(src, bin, log)).first;
    }
    if (!it->second) return 0;
    (*built)++;
  }
  return 0;
}

int jit_min_state_bits() { return jit_enabled() ? jit_min_bits() : 64; }

int jit_plan_arith(const Plan& p, bool dw, double* fma_per_elem, double* mul_per_elem, double* instr_per_elem) {
  *fma_per_elem = *mul_per_elem = 0.0;
  int eligible = 0;
  for (size_t i = 0; i < p.sweeps.size(); i++) {
    const SweepDesc& sd = p.sweeps[i];
    if (sd.nops == 0 || (p.is_complex && sd.nph == 0)) continue;
    Gen g(p, sd, dw);
    std::string src;
    if (!g.run(src)) continue;
    *fma_per_elem += g.fma_per_elem;
    *mul_per_elem += g.mul_per_elem;
    eligible++;
  }
  // instructions of the arithmetic pipe: one each (FP64 or FP32 kernels), or
  // the FP32 instructions of the double-word operations of kDwPrelude
  *instr_per_elem = dw && p.dtype == NWQ_F64 ? kDwFmaInstr * *fma_per_elem + kDwMulInstr * *mul_per_elem
                                             : *fma_per_elem + *mul_per_elem;
  return eligible;
}

void jit_shutdown() {
  if (g_async_started) async_compiler().shutdown();
}

int jit_prefetch(const Plan& p) {
  if (!jit_enabled()) return 0;
  int queued = 0;
  for (size_t i = 0; i < p.sweeps.size(); i++) {
    const SweepDesc& sd = p.sweeps[i];
    if (sd.nops == 0 || (p.is_complex && sd.nph == 0)) continue;
    std::shared_ptr<JitKernel> k = entry_for(struct_key(p, sd, p.dw));
    if (!describe(*k, p, sd, p.dw)) continue;
    request_compile(k, true);
    if (!k->done) queued++;
  }
  return queued;
}

void jit_stats(int* compiled, int* failed) {
  if (compiled) *compiled = g_compiled.load();
  if (failed) *failed = g_failed.load();
}

// The plan's kernels of one mode (0: its own precision, 1: double words),
// described and requested on first use; null when specialised kernels are off.
static JitPlan* jit_plan_mode(Plan& p, int mode) {
  if (!jit_enabled() || p.interpreted || p.B < jit_min_bits()) return nullptr;
  if (!p.jit) p.jit = std::make_shared<JitPlan>();
  JitPlan& jp = *std::static_pointer_cast<JitPlan>(p.jit);
  std::lock_guard<std::mutex> lk(jp.mu);
  if (!jp.built[mode]) {
    jp.sw[mode].resize(p.sweeps.size());
    for (size_t i = 0; i < p.sweeps.size(); i++) {
      const SweepDesc& sd = p.sweeps[i];
      if (sd.nops == 0 || (p.is_complex && sd.nph == 0)) continue;
      std::shared_ptr<JitKernel> k = entry_for(struct_key(p, sd, mode == 1));
      if (!describe(*k, p, sd, mode == 1)) continue;
      // one-shot plans never wait for a compile: their sweeps run interpreted
      // until the kernel of that structure is ready
      request_compile(k, p.stream_ordered && !jit_sync_all());
      if (k->done && !k->ok) continue;
      std::vector<unsigned char> param = pack_params(p, sd, k->recipe, mode == 1);
      if (param.empty()) continue;
      JitSweep& js = jp.sw[mode][i];
      js.k = k;
      js.param = std::move(param);
      js.smem = k->smem;
    }
    jp.built[mode] = true;
  }
  return &jp;
}

bool jit_dw_ready(Plan& p) {
  if (!p.dw) return false;
  JitPlan* jp = jit_plan_mode(p, 1);
  if (!jp) return false;
  bool any = false;
  for (size_t i = 0; i < p.sweeps.size(); i++) {
    if (p.sweeps[i].nops == 0) continue;
    const JitSweep& js = jp->sw[1][i];
    if (!js.k || !js.k->done || !js.k->ok) return false;
    any = true;
  }
  return any;
}

bool jit_launch_sweep(Plan& p, size_t sweep, const PhaseTables& pt, void* state, int sm_count, cudaStream_t s,
                      cudaError_t* err, bool dw) {
  if (sweep >= p.sweeps.size()) return false;
  JitPlan* jpp = jit_plan_mode(p, dw ? 1 : 0);
  if (!jpp) return false;
  JitSweep& js = jpp->sw[dw ? 1 : 0][sweep];
  if (!js.k || !js.k->done || !js.k->ok) return false;
  const void* fn = (const void*)js.k->k;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaError_t e = cudaSuccess;
  if (js.k->attr_dev.load() != dev) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e != cudaSuccess) {
      *err = e;
      return true;
    }
    js.k->attr_dev = dev;
  }
  if (js.per_sm == 0) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, js.k->threads, js.smem);
    if (e != cudaSuccess) {
      *err = e;
      return true;
    }
    js.per_sm = per_sm < 1 ? 1 : per_sm;
    if (const char* v = std::getenv("NWQ_JIT_VERBOSE"); v && v[0] == '1') {  // resources of each sweep's kernel
      cudaFuncAttributes fa{};
      cudaFuncGetAttributes(&fa, fn);
      std::fprintf(stderr, "jit sweep %zu: T %d, %d registers, %d local bytes, smem %zu, %d CTAs per SM\n", sweep,
                   p.sweeps[sweep].T, fa.numRegs, (int)fa.localSizeBytes, js.smem, js.per_sm);
    }
  }
  const SweepDesc& sd = p.sweeps[sweep];
  unsigned long long ntiles = 1ull << (p.B - sd.T);
  unsigned long long grid = (unsigned long long)sm_count * js.per_sm;
  if (grid > ntiles) grid = ntiles;
  unsigned long long hmask = sd.hmask, fmask = sd.fmask;
  const void* pcs = p.is_complex && pt.pc ? (const char*)pt.pc + (size_t)sd.pc0 * (p.dtype == NWQ_F64 ? 16 : 8)
                                          : nullptr;
  void* args[] = {&state, &ntiles, &hmask, &fmask, (void*)&pcs, js.param.data()};
  e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(js.k->threads), args, js.smem, s);
  g_launches += 1;
  *err = e;
  return true;
}

}  // namespace nwq
