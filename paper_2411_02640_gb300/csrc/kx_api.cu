// C ABI of the kx library: mechanism handles, NVRTC compilation of the
// emitted kernels for sm_103a with an on-disk cubin cache, and launches.
//
// The runtime is the CUDA runtime API linked statically, so the shared
// library loads on machines without a GPU (for builds and CPU tests) and
// talks to whatever driver is present when a kernel is first launched.
// Kernels are loaded as context-independent libraries (cudaLibraryLoadData)
// and launched with cudaLaunchKernel on the caller's stream.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "kx_internal.h"

#define KX_VERSION "kx-1.0"

namespace {

thread_local std::string g_last_error;

kx_status fail(kx_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

kx_status cuda_fail(cudaError_t e, const char* what) {
  return fail(KX_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct Kernel {
  std::string name;            // e.g. "wdot_fp64"
  std::string entry;           // extern "C" symbol in the emitted source
  kx::KernelKind kind;
  kx::EmitOptions eopt;
  kx::OpCounts ops;
  std::string source;
  std::vector<char> cubin;
  cudaLibrary_t lib = nullptr;
  cudaKernel_t fn = nullptr;
  double compile_seconds = 0;
  int registers = -1, local_bytes = -1;
  int max_blocks = 0;          // resident blocks for a persistent grid (per device 0 at load)
  int blocks_per_sm = 0;       // resident blocks per SM
  int smem = 0;                // dynamic shared memory per block, bytes
  int states_per_block = 0;    // states one block serves per pass of its grid-stride loop (0: one per thread)
  double lane_use = 1.0;       // warp-cooperative kernels: lane use of their class rounds
  int device = -1;
  std::mutex mu;
  bool ready = false;
  kx_status status = KX_OK;
  std::string error;
};

}  // namespace

// The call's own streams and events of kx_evaluate_host, kept for reuse: a
// call takes one set (of the current device) from the handle's free list and
// puts it back on return, with its work possibly still in flight; the next
// call on the same set queues behind it on the same streams.
struct HostPipe {
  int device = -1;
  cudaStream_t qc = nullptr, qd = nullptr;   // copy-out stream, odd chunks' kernels
  cudaEvent_t ev[8] = {};
};

struct kx_mech {
  kx::Mechanism m;
  kx_options opt{};
  std::string cache_dir;
  std::vector<std::unique_ptr<Kernel>> kernels;
  std::mutex pipe_mu;
  std::vector<std::unique_ptr<HostPipe>> pipes;   // every set this handle made
  std::vector<HostPipe*> free_pipes;
};

namespace {

uint64_t fnv1a(const std::string& s, uint64_t h = 1469598103934665603ULL) {
  for (unsigned char ch : s) { h ^= ch; h *= 1099511628211ULL; }
  return h;
}

std::string default_cache_dir() {
  if (const char* e = std::getenv("KX_CACHE_DIR")) return e;
  const char* home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/kx";
}

void mkdirs(const std::string& path) {
  std::string cur;
  std::stringstream ss(path);
  std::string part;
  if (!path.empty() && path[0] == '/') cur = "/";
  while (std::getline(ss, part, '/')) {
    if (part.empty()) continue;
    cur += part + "/";
    mkdir(cur.c_str(), 0755);
  }
}

bool read_file(const std::string& p, std::vector<char>& out) {
  std::ifstream f(p, std::ios::binary);
  if (!f) return false;
  out.assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
  return !out.empty();
}

void write_file_atomic(const std::string& p, const std::vector<char>& data) {
  std::string tmp = p + "." + std::to_string(getpid()) + "." +
                    std::to_string(std::hash<std::thread::id>()(std::this_thread::get_id())) + ".tmp";
  {
    std::ofstream f(tmp, std::ios::binary);
    if (!f) return;
    f.write(data.data(), (std::streamsize)data.size());
  }
  std::rename(tmp.c_str(), p.c_str());
}

// "ptxas info    : Used 255 registers, ...", "N bytes stack frame, M bytes spill stores": the
// registers and the per-thread local memory (stack frame: local arrays and spills) of the kernel
void parse_ptxas_info(const std::string& log, int& regs, int& local) {
  size_t p = log.rfind("Used ");
  if (p != std::string::npos) regs = std::atoi(log.c_str() + p + 5);
  size_t q = log.find("bytes stack frame");
  if (q != std::string::npos) {
    size_t s = q;
    while (s > 0 && log[s - 1] == ' ') --s;
    while (s > 0 && log[s - 1] >= '0' && log[s - 1] <= '9') --s;
    local = std::atoi(log.c_str() + s);
  }
}

// Emit + compile (or fetch from the cache) one kernel.  Host only.
kx_status compile_kernel(kx_mech* h, Kernel& k) {
  auto t0 = std::chrono::steady_clock::now();
  k.source = kx::emit_kernel(h->m, k.kind, k.eopt, k.entry, &k.ops);
  if (k.source.empty()) return fail(KX_ERR_UNSUPPORTED, "kernel " + k.name + " is not available");
  std::vector<std::string> opts = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "--ptxas-options=-v"};
  if (h->opt.libmath) opts.push_back("-DKX_LIBMATH");

  std::string key = std::string(KX_VERSION) + "\n";
  for (auto& o : opts) key += o + "\n";
  int ver_major = 0, ver_minor = 0;
  nvrtcVersion(&ver_major, &ver_minor);
  key += std::to_string(ver_major) + "." + std::to_string(ver_minor) + "\n" + k.source;
  char hex[32];
  std::snprintf(hex, sizeof hex, "%016llx", (unsigned long long)fnv1a(key));
  const std::string base = h->cache_dir + "/" + k.name + "-" + hex;
  std::vector<char> info;
  if (read_file(base + ".cubin", k.cubin)) {
    if (read_file(base + ".log", info)) {
      std::string log(info.begin(), info.end());
      parse_ptxas_info(log, k.registers, k.local_bytes);
    }
  } else {
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, k.source.c_str(), (k.name + ".cu").c_str(), 0, nullptr, nullptr) != NVRTC_SUCCESS)
      return fail(KX_ERR_COMPILE, "nvrtcCreateProgram failed");
    std::vector<const char*> copts;
    for (auto& o : opts) copts.push_back(o.c_str());
    nvrtcResult rc = nvrtcCompileProgram(prog, (int)copts.size(), copts.data());
    size_t log_size = 0;
    nvrtcGetProgramLogSize(prog, &log_size);
    std::string log(log_size, '\0');
    if (log_size) nvrtcGetProgramLog(prog, &log[0]);
    if (rc != NVRTC_SUCCESS) {
      nvrtcDestroyProgram(&prog);
      if (h->opt.verbose) std::fprintf(stderr, "kx: compile of %s failed:\n%s\n", k.name.c_str(), log.c_str());
      // keep the failing source for inspection
      write_file_atomic(base + ".failed.cu", std::vector<char>(k.source.begin(), k.source.end()));
      return fail(KX_ERR_COMPILE, "NVRTC failed on " + k.name + ": " + log.substr(0, 2000));
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    k.cubin.resize(n);
    nvrtcGetCUBIN(prog, k.cubin.data());
    nvrtcDestroyProgram(&prog);
    parse_ptxas_info(log, k.registers, k.local_bytes);
    mkdirs(h->cache_dir);
    if (std::getenv("KX_DUMP_SOURCE"))
      write_file_atomic(base + ".cu", std::vector<char>(k.source.begin(), k.source.end()));
    write_file_atomic(base + ".cubin", k.cubin);
    write_file_atomic(base + ".log", std::vector<char>(log.begin(), log.end()));
  }
  k.compile_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (h->opt.verbose)
    std::fprintf(stderr, "kx: %s: %.1f s, %d registers, %d bytes of local memory per thread, %zu source bytes\n", k.name.c_str(),
                 k.compile_seconds, k.registers, k.local_bytes, k.source.size());
  return KX_OK;
}

kx_status load_kernel(Kernel& k) {
  cudaError_t e = cudaLibraryLoadData(&k.lib, k.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLibraryLoadData");
  e = cudaLibraryGetKernel(&k.fn, k.lib, k.entry.c_str());
  if (e != cudaSuccess) return cuda_fail(e, "cudaLibraryGetKernel");
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  if (k.smem > 0) {
    e = cudaKernelSetAttributeForDevice(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaKernelSetAttributeForDevice");
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k.fn, k.eopt.block, k.smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  k.max_blocks = sms * (per_sm > 0 ? per_sm : 1);
  k.blocks_per_sm = per_sm > 0 ? per_sm : 1;
  k.device = dev;
  return KX_OK;
}

kx_status ensure_ready(kx_mech* h, Kernel& k) {
  std::lock_guard<std::mutex> lock(k.mu);
  if (k.ready) return KX_OK;
  if (k.status != KX_OK) return fail(k.status, k.error);
  kx_status s = KX_OK;
  if (k.cubin.empty()) s = compile_kernel(h, k);
  if (s == KX_OK && !h->opt.compile_only) s = load_kernel(k);
  if (s != KX_OK) {
    k.status = s;
    k.error = g_last_error;
    return s;
  }
  k.ready = !h->opt.compile_only;
  return KX_OK;
}

Kernel* find_kernel(kx_mech* h, const std::string& name) {
  for (auto& k : h->kernels)
    if (k->name == name) return k.get();
  return nullptr;
}

kx_status launch(kx_mech* h, const char* name, void** args, int64_t n, void* stream) {
  Kernel* k = find_kernel(h, name);
  if (!k) return fail(KX_ERR_UNSUPPORTED, std::string("no kernel ") + name);
  if (h->opt.compile_only) return fail(KX_ERR_UNSUPPORTED, "handle was loaded with compile_only");
  kx_status s = ensure_ready(h, *k);
  if (s != KX_OK) return s;
  const int spb = k->states_per_block > 0 ? k->states_per_block : k->eopt.block;
  const int64_t want = (n + spb - 1) / spb;
  // warp-cooperative kernels: one resident wave, each warp looping over groups of states (their
  // per-warp shared-memory slices); one-state-per-thread kernels: one state per thread, the block
  // scheduler balancing blocks of unequal cost (hot states against cold ones, whose reactions mostly
  // take the rate kernels' float32 path).  Measured on 53/325 against a grid of four resident waves
  // striding over the batch: production rates 5.68 -> 5.40 ms per 2^20 states and 35.1 -> 23.0 ms
  // per 2^22 (the strided grid's blocks accumulated the imbalance over 13 states per thread);
  // thermo and transport 0-10 % faster.
  const int64_t cap = k->states_per_block > 0 ? (int64_t)k->max_blocks : (int64_t)INT_MAX;
  const int grid = (int)std::min<int64_t>(want, cap);
  cudaError_t e =
      cudaLaunchKernel((const void*)k->fn, dim3(grid), dim3(k->eopt.block), args, k->smem, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchKernel");
  return KX_OK;
}

// Scratch of kx_production_rates_noalloc: a file-scope device array whose
// device address is looked up once per device.  In host code the symbol
// names a host-side shadow, not device memory, so only the looked-up
// address is ever handed to a kernel.
static __device__ __align__(256) unsigned char kx_noalloc_scratch[KX_NOALLOC_SCRATCH_BYTES];

struct NoAllocDevice {
  std::once_flag once;
  void* scratch = nullptr;
  cudaError_t err = cudaSuccess;
};
constexpr int kMaxDevices = 64;
NoAllocDevice g_noalloc[kMaxDevices];

// Must run with device `dev` current.
kx_status noalloc_device(int dev, NoAllocDevice** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(KX_ERR_UNSUPPORTED, "device index out of range");
  NoAllocDevice& d = g_noalloc[dev];
  std::call_once(d.once, [&] { d.err = cudaGetSymbolAddress(&d.scratch, kx_noalloc_scratch); });
  if (d.err != cudaSuccess) return cuda_fail(d.err, "no-alloc scratch address (cudaGetSymbolAddress)");
  *out = &d;
  return KX_OK;
}

kx_status check_state(kx_mech* h, const double* T, const double* p, const double* Y, int64_t ld, int64_t n) {
  if (!h) return fail(KX_ERR_ARG, "null handle");
  if (n < 0) return fail(KX_ERR_ARG, "negative point count");
  if (n > 0 && (!T || !p || !Y)) return fail(KX_ERR_ARG, "null state pointer");
  if (ld < n) return fail(KX_ERR_ARG, "leading dimension smaller than the point count");
  return KX_OK;
}

}  // namespace

extern "C" {

const char* kx_status_string(kx_status s) {
  switch (s) {
    case KX_OK: return "ok";
    case KX_ERR_IO: return "mechanism file cannot be read";
    case KX_ERR_PARSE: return "malformed mechanism file";
    case KX_ERR_UNBALANCED: return "reaction does not conserve atoms";
    case KX_ERR_ARG: return "invalid argument";
    case KX_ERR_OOM: return "out of memory";
    case KX_ERR_COMPILE: return "kernel compilation failed";
    case KX_ERR_CUDA: return "CUDA error";
    case KX_ERR_TIMEOUT: return "timed out";
    case KX_ERR_NONFINITE_INPUT: return "non-finite input";
    case KX_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* kx_last_error(void) { return g_last_error.c_str(); }

kx_status kx_load_mechanism(const char* path, const kx_options* opt, kx_handle* out) {
  if (!path || !out) return fail(KX_ERR_ARG, "null argument");
  *out = nullptr;
  std::unique_ptr<kx_mech> h(new (std::nothrow) kx_mech());
  if (!h) return fail(KX_ERR_OOM, "host allocation failed");
  if (opt) h->opt = *opt;
  if (h->opt.block == 0) h->opt.block = 128;
  if (h->opt.block < 32 || h->opt.block > 1024 || h->opt.block % 32) return fail(KX_ERR_ARG, "block must be a multiple of 32 in [32, 1024]");
  if (h->opt.diff_mode < 0 || h->opt.diff_mode > 2) return fail(KX_ERR_ARG, "diff_mode must be 0, 1 or 2");
  if (h->opt.kc_mode < 0 || h->opt.kc_mode > 1) return fail(KX_ERR_ARG, "kc_mode must be 0 or 1");
  if (h->opt.tr_mode < 0 || h->opt.tr_mode > 1) return fail(KX_ERR_ARG, "tr_mode must be 0 or 1");
  if (h->opt.rates_mode < 0 || h->opt.rates_mode > 2) return fail(KX_ERR_ARG, "rates_mode must be 0, 1 or 2");
  if (h->opt.rates_arith < 0 || h->opt.rates_arith > 2) return fail(KX_ERR_ARG, "rates_arith must be 0, 1 or 2");
  if (h->opt.tr_layout < 0 || h->opt.tr_layout > 3) return fail(KX_ERR_ARG, "tr_layout must be 0, 1, 2 or 3");
  if (h->opt.maxrreg < 0 || h->opt.maxrreg > 255) return fail(KX_ERR_ARG, "maxrreg must be in [0, 255]");
  if (h->opt.rates_layout < 0 || h->opt.rates_layout > 2) return fail(KX_ERR_ARG, "rates_layout must be 0, 1 or 2");
  if (h->opt.vjp_form < 0 || h->opt.vjp_form > 1) return fail(KX_ERR_ARG, "vjp_form must be 0 or 1");
  if (h->opt.vjp_layout < 0 || h->opt.vjp_layout > 2) return fail(KX_ERR_ARG, "vjp_layout must be 0, 1 or 2");
  if (h->opt.rates_negligible < 0 || h->opt.rates_negligible > 1) return fail(KX_ERR_ARG, "rates_negligible must be 0 or 1");
  if (h->opt.rates_group < 0 || h->opt.rates_group > 32 || (h->opt.rates_group & (h->opt.rates_group - 1)))
    return fail(KX_ERR_ARG, "rates_group must be 0 or a power of two up to 32");
  h->cache_dir = h->opt.cache_dir ? h->opt.cache_dir : default_cache_dir();
  h->opt.cache_dir = nullptr;
  std::string err;
  kx_status s = kx::parse_mechanism(path, h->m, err);
  if (s != KX_OK) return fail(s, err);

  struct Spec { const char* name; kx::KernelKind kind; bool mixed; int part; };
  const Spec specs[] = {
      {"wdot_fp64", kx::KernelKind::Wdot, false, 0},      {"wdot_mixed", kx::KernelKind::Wdot, true, 0},
      {"rop_fp64", kx::KernelKind::Rop, false, 0},        {"rop_mixed", kx::KernelKind::Rop, true, 0},
      {"thermo", kx::KernelKind::Thermo, false, 0},       {"visc_fp64", kx::KernelKind::Transport, false, 1},
      {"diff_fp64", kx::KernelKind::Transport, false, 2}, {"visc_mixed", kx::KernelKind::Transport, true, 1},
      {"diff_mixed", kx::KernelKind::Transport, true, 2}, {"vjp", kx::KernelKind::Vjp, false, 0},
      {"wdot_fp64_noalloc", kx::KernelKind::Wdot, false, 0}, {"wdot_fp64_wc", kx::KernelKind::Wdot, false, 0},
      {"vjp_wc", kx::KernelKind::Vjp, false, 0},
  };
  for (const Spec& sp : specs) {
    std::unique_ptr<Kernel> k(new Kernel());
    k->name = sp.name;
    k->entry = std::string("kx_") + sp.name;
    k->kind = sp.kind;
    k->eopt.mixed = sp.mixed;
    k->eopt.block = h->opt.block;
    k->eopt.diff_mode = h->opt.diff_mode == 2 ? 2 : 1;
    k->eopt.kc_mode = h->opt.kc_mode;
    k->eopt.tr_mode = h->opt.tr_mode;
    k->eopt.part = sp.part;
    k->eopt.maxrreg = h->opt.maxrreg;
    k->eopt.rates_mode = h->opt.rates_mode;
    k->eopt.rates_arith = h->opt.rates_arith;
    k->eopt.scratch = std::strcmp(sp.name, "wdot_fp64_noalloc") == 0;
    const bool wc_spec = std::strcmp(sp.name, "wdot_fp64_wc") == 0;
    k->eopt.rates_layout = wc_spec ? 2 : h->opt.rates_layout;
    if (wc_spec) k->eopt.rates_arith = 0;
    k->eopt.rates_group = h->opt.rates_group;
    k->eopt.vjp_form = h->opt.vjp_form;
    k->eopt.vjp_layout = h->opt.vjp_layout;
    k->eopt.rates_negligible = h->opt.rates_negligible;
    const bool vjp_wc_spec = std::strcmp(sp.name, "vjp_wc") == 0;
    if (vjp_wc_spec) {
      // the warp-cooperative adjoint beside the default one, for small batches
      if (h->opt.vjp_layout != 0 || h->opt.rates_arith == 1) continue;
      k->eopt.vjp_layout = 2;
      kx::EmitOptions one = k->eopt;
      one.rates_group = 1;
      k->lane_use = kx::wdot_wc_shape(h->m, one).lane_use;
    }
    if (kx::vjp_is_wc(h->m, sp.kind, k->eopt)) {
      k->smem = kx::vjp_wc_smem(h->m, k->eopt);
      k->states_per_block = k->eopt.block / 32;
      if (k->smem > 200 * 1024) {
        if (vjp_wc_spec) continue;   // too large for small batches too: the default adjoint serves them
        return fail(KX_ERR_UNSUPPORTED, "warp-cooperative adjoint: one block's shared memory exceeds 200 KB (vjp_layout 1)");
      }
    }
    if (kx::wdot_is_wc(h->m, sp.kind, k->eopt)) {
      const kx::WcShape w = kx::wdot_wc_shape(h->m, k->eopt);
      if (w.smem_per_block > 200 * 1024)
        return fail(KX_ERR_UNSUPPORTED, "warp-cooperative rate kernel: one block's shared memory exceeds 200 KB "
                                        "(choose a smaller rates_group or rates_layout 1)");
      k->smem = w.smem_per_block;
      k->states_per_block = w.states_per_block;
      k->lane_use = w.lane_use;
    }
    if (sp.kind == kx::KernelKind::Transport) {
      // species vectors staged in shared memory: as many threads as fit in ~216 KB, a multiple of 32
      k->eopt.tr_layout = h->opt.tr_layout == 0 ? 3 : h->opt.tr_layout;
      const int per = kx::transport_smem_per_thread(h->m, sp.mixed, sp.part, k->eopt.tr_layout);
      int b = per == 0 ? h->opt.block : std::min(std::max(h->opt.block, 256), std::min(1024, (216 * 1024 / per) / 32 * 32));
      if (b >= 128) b = b / 128 * 128;   // whole warps on every SM sub-partition
      if (b < 32) return fail(KX_ERR_UNSUPPORTED, "mechanism too large for the transport kernel");
      k->eopt.block = b;
      k->smem = per * b;
    }
    h->kernels.push_back(std::move(k));
  }
  if (!h->opt.lazy) {
    // compile the kernels of the production-rate, thermo and transport calls
    // in parallel (NVRTC programs are independent) and load them; the
    // rates-of-progress and adjoint kernels compile on first use
    std::vector<Kernel*> eager;
    for (auto& k : h->kernels)
      if (k->kind != kx::KernelKind::Rop && k->kind != kx::KernelKind::Vjp) eager.push_back(k.get());
    std::vector<std::thread> th;
    std::vector<kx_status> st(eager.size(), KX_OK);
    std::vector<std::string> msg(eager.size());
    for (size_t i = 0; i < eager.size(); ++i)
      th.emplace_back([&, i] {
        st[i] = compile_kernel(h.get(), *eager[i]);
        if (st[i] != KX_OK) msg[i] = g_last_error;
      });
    for (auto& t : th) t.join();
    for (size_t i = 0; i < st.size(); ++i)
      if (st[i] != KX_OK) return fail(st[i], msg[i]);
    if (!h->opt.compile_only) {
      for (Kernel* k : eager) {
        s = ensure_ready(h.get(), *k);
        if (s != KX_OK) return s;
      }
      // the no-alloc call's scratch address, looked up here with this device current
      int dev = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
      NoAllocDevice* nd = nullptr;
      s = noalloc_device(dev, &nd);
      if (s != KX_OK) return s;
    }
  }
  *out = h.release();
  return KX_OK;
}

kx_status kx_free_mechanism(kx_handle h) {
  if (!h) return fail(KX_ERR_ARG, "null handle");
  for (auto& hp : h->pipes) {
    for (cudaEvent_t e : hp->ev) if (e) cudaEventDestroy(e);
    if (hp->qc) cudaStreamDestroy(hp->qc);
    if (hp->qd) cudaStreamDestroy(hp->qd);
  }
  for (auto& k : h->kernels)
    if (k->lib) cudaLibraryUnload(k->lib);
  delete h;
  return KX_OK;
}

kx_status kx_mechanism_info(kx_handle h, int* n_species, int* n_reactions, double* W) {
  if (!h) return fail(KX_ERR_ARG, "null handle");
  if (n_species) *n_species = h->m.ns;
  if (n_reactions) *n_reactions = h->m.nr();
  if (W) std::memcpy(W, h->m.W.data(), sizeof(double) * h->m.ns);
  return KX_OK;
}

}  // extern "C"

namespace {

// The production-rate kernel for a batch of n states.  Small float64-accurate batches go to the
// warp-cooperative kernel, whose warps share each state: the thread-per-state kernel would leave
// SMs idle and take one state's whole latency.  The crossover, measured on GB300, sits near 48k
// states times the lane use of the warp-cooperative class rounds (53/325: ~44k, 160/900: ~46k, 9/21
// with its few reactions per class: ~11k), and never above the thread-per-state kernel's resident
// capacity.
kx_status wdot_kernel_for(kx_mech* h, int64_t n, kx_precision precision, const char** name) {
  *name = precision == KX_FP64 ? "wdot_fp64" : "wdot_mixed";
  if (precision != KX_FP64 || h->opt.rates_layout != 0 || h->opt.rates_arith == 1) return KX_OK;
  Kernel* tps = find_kernel(h, "wdot_fp64");
  Kernel* wc = find_kernel(h, "wdot_fp64_wc");
  kx_status s = ensure_ready(h, *tps);
  if (s == KX_OK) s = ensure_ready(h, *wc);
  if (s != KX_OK) return s;
  const int64_t cap = (int64_t)tps->max_blocks * tps->eopt.block;
  if (n < std::min<int64_t>(cap, (int64_t)(49152.0 * wc->lane_use))) *name = "wdot_fp64_wc";
  return KX_OK;
}

// The adjoint kernel for a batch of n states.  Small batches go to the warp-cooperative adjoint (one
// state per warp) by default.  Its throughput grows with its resident warps per SM and, twice, with
// the lane use u of its class rounds (reaction rounds and, for small mechanisms, the species
// phases); the crossover measured on GB300 fits 8192 x resident warps per SM x u^2 states (9/21:
// ~8k measured, 6.3k by the rule; 53/325: 65k-131k, 84k; 160/900: ~32k, 29k), and is kept below
// the thread-per-state kernel's resident capacity.
kx_status vjp_kernel_for(kx_mech* h, int64_t n, const char** name) {
  *name = "vjp";
  Kernel* wc = find_kernel(h, "vjp_wc");
  if (!wc) return KX_OK;
  Kernel* tps = find_kernel(h, "vjp");
  kx_status s = ensure_ready(h, *tps);
  if (s == KX_OK) s = ensure_ready(h, *wc);
  if (s != KX_OK) return s;
  const int64_t cap = (int64_t)tps->max_blocks * tps->eopt.block;
  const double warps = (double)wc->blocks_per_sm * (wc->eopt.block / 32);
  if (n < std::min<int64_t>(cap, (int64_t)(8192.0 * warps * wc->lane_use * wc->lane_use))) *name = "vjp_wc";
  return KX_OK;
}

// Production rates of n states with the kernel `name`.
kx_status production_rates_with(kx_mech* h, const char* name, const double* T, const double* p, const double* Y,
                                int64_t ld, double* wdot, int64_t n, void* stream) {
  if (n == 0) return KX_OK;
  long long ldl = ld, nl = n;
  void* args[] = {&T, &p, &Y, &ldl, &wdot, &nl};
  return launch(h, name, args, n, stream);
}

}  // namespace

extern "C" {

kx_status kx_production_rates(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld,
                              double* wdot, int64_t n, kx_precision precision, void* stream) {
  kx_status s = check_state(h, T, p, Y, ld, n);
  if (s != KX_OK) return s;
  if (n > 0 && !wdot) return fail(KX_ERR_ARG, "null output");
  if (precision != KX_FP64 && precision != KX_MIXED) return fail(KX_ERR_ARG, "bad precision");
  if (n == 0) return KX_OK;
  const char* name = nullptr;
  if ((s = wdot_kernel_for(h, n, precision, &name)) != KX_OK) return s;
  return production_rates_with(h, name, T, p, Y, ld, wdot, n, stream);
}

kx_status kx_production_rates_noalloc(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld,
                                      double* wdot, int64_t n, void* stream) {
  kx_status s = check_state(h, T, p, Y, ld, n);
  if (s != KX_OK) return s;
  if (n > 0 && !wdot) return fail(KX_ERR_ARG, "null output");
  if (n == 0) return KX_OK;
  if (h->opt.compile_only) return fail(KX_ERR_UNSUPPORTED, "handle was loaded with compile_only");
  Kernel* k = find_kernel(h, "wdot_fp64_noalloc");
  s = ensure_ready(h, *k);
  if (s != KX_OK) return s;
  int dev = 0;
  cudaError_t ge = cudaGetDevice(&dev);
  if (ge != cudaSuccess) return cuda_fail(ge, "cudaGetDevice");
  NoAllocDevice* nd = nullptr;
  s = noalloc_device(dev, &nd);
  if (s != KX_OK) return s;
  const int B = k->eopt.block;
  const int64_t fit = (int64_t)(KX_NOALLOC_SCRATCH_BYTES / (size_t)kx::rates_scratch_per_thread(h->m)) / B;
  if (fit < 1) return fail(KX_ERR_UNSUPPORTED, "one block of the rate kernel does not fit the no-alloc scratch");
  const int64_t want = (n + B - 1) / B;
  const int grid = (int)std::min<int64_t>(std::min<int64_t>(want, (int64_t)k->max_blocks), fit);
  long long ldl = ld, nl = n, nthr = (long long)grid * B;
  unsigned char* scr = (unsigned char*)nd->scratch;
  void* args[] = {&T, &p, &Y, &ldl, &wdot, &scr, &nthr, &nl};
  // no ordering between calls: two calls that overlap on the GPU share the array and race
  cudaError_t e = cudaLaunchKernel((const void*)k->fn, dim3(grid), dim3(B), args, k->smem, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchKernel");
  return KX_OK;
}

kx_status kx_last_point_status(kx_handle h, void* stream, int64_t* first_bad_point) {
  if (!h || !first_bad_point) return fail(KX_ERR_ARG, "null argument");
  *first_bad_point = -1;
  if (h->opt.compile_only) return fail(KX_ERR_UNSUPPORTED, "handle was loaded with compile_only");
  // every loaded kernel keeps its own word; read each and set it back to "none" behind the work queued on stream
  std::vector<void*> addr;
  for (auto& k : h->kernels) {
    {
      std::lock_guard<std::mutex> lock(k->mu);
      if (!k->ready) continue;
    }
    void* d = nullptr;
    size_t bytes = 0;
    cudaError_t e = cudaLibraryGetGlobal(&d, &bytes, k->lib, "kx_bad_first");
    if (e != cudaSuccess) return cuda_fail(e, "cudaLibraryGetGlobal");
    if (bytes != sizeof(unsigned long long)) return fail(KX_ERR_CUDA, "unexpected size of the point status word");
    addr.push_back(d);
  }
  std::vector<unsigned long long> word(addr.size(), ~0ull);
  for (size_t j = 0; j < addr.size(); ++j) {
    cudaError_t e = cudaMemcpyAsync(&word[j], addr[j], sizeof(unsigned long long), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(addr[j], 0xff, sizeof(unsigned long long), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "point status word");
  }
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  unsigned long long first = ~0ull;
  for (unsigned long long w : word) first = std::min(first, w);
  if (first == ~0ull) return KX_OK;
  *first_bad_point = (int64_t)first;
  return fail(KX_ERR_NONFINITE_INPUT, "point " + std::to_string(first) +
                                          " is outside the domain (T or p not positive and finite, or sum Y/W not positive and finite)");
}

kx_status kx_rates_of_progress(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld, double* q,
                               int64_t n, kx_precision precision, void* stream) {
  kx_status s = check_state(h, T, p, Y, ld, n);
  if (s != KX_OK) return s;
  if (n > 0 && !q) return fail(KX_ERR_ARG, "null output");
  if (precision != KX_FP64 && precision != KX_MIXED) return fail(KX_ERR_ARG, "bad precision");
  if (n == 0) return KX_OK;
  long long ldl = ld, nl = n;
  void* args[] = {&T, &p, &Y, &ldl, &q, &nl};
  return launch(h, precision == KX_FP64 ? "rop_fp64" : "rop_mixed", args, n, stream);
}

kx_status kx_thermo(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld, double* cp,
                    double* hmass, int64_t n, void* stream) {
  kx_status s = check_state(h, T, p, Y, ld, n);
  if (s != KX_OK) return s;
  if (n > 0 && (!cp || !hmass)) return fail(KX_ERR_ARG, "null output");
  if (n == 0) return KX_OK;
  long long ldl = ld, nl = n;
  void* args[] = {&T, &p, &Y, &ldl, &cp, &hmass, &nl};
  return launch(h, "thermo", args, n, stream);
}

kx_status kx_transport(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld, double* mu,
                       double* lambda, double* Dk, int64_t n, kx_precision precision, void* stream) {
  kx_status s = kx_viscosity_conductivity(h, T, p, Y, ld, mu, lambda, n, precision, stream);
  if (s != KX_OK) return s;
  return kx_diffusion(h, T, p, Y, ld, Dk, n, precision, stream);
}

kx_status kx_viscosity_conductivity(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld,
                                    double* mu, double* lambda, int64_t n, kx_precision precision, void* stream) {
  kx_status s = check_state(h, T, p, Y, ld, n);
  if (s != KX_OK) return s;
  if (n > 0 && (!mu || !lambda)) return fail(KX_ERR_ARG, "null output");
  if (precision != KX_FP64 && precision != KX_MIXED) return fail(KX_ERR_ARG, "bad precision");
  if (n == 0) return KX_OK;
  long long ldl = ld, nl = n;
  double* none = nullptr;
  void* args[] = {&T, &p, &Y, &ldl, &mu, &lambda, &none, &nl};
  return launch(h, precision == KX_FP64 ? "visc_fp64" : "visc_mixed", args, n, stream);
}

kx_status kx_diffusion(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld, double* Dk,
                       int64_t n, kx_precision precision, void* stream) {
  kx_status s = check_state(h, T, p, Y, ld, n);
  if (s != KX_OK) return s;
  if (n > 0 && !Dk) return fail(KX_ERR_ARG, "null output");
  if (precision != KX_FP64 && precision != KX_MIXED) return fail(KX_ERR_ARG, "bad precision");
  if (n == 0) return KX_OK;
  long long ldl = ld, nl = n;
  double* none = nullptr;
  void* args[] = {&T, &p, &Y, &ldl, &none, &none, &Dk, &nl};
  return launch(h, precision == KX_FP64 ? "diff_fp64" : "diff_mixed", args, n, stream);
}

kx_status kx_production_rates_vjp(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld,
                                  const double* v, double* gT, double* gY, int64_t n, void* stream) {
  kx_status s = check_state(h, T, p, Y, ld, n);
  if (s != KX_OK) return s;
  if (n > 0 && (!v || !gT || !gY)) return fail(KX_ERR_ARG, "null argument");
  if (n == 0) return KX_OK;
  const char* name = nullptr;
  if ((s = vjp_kernel_for(h, n, &name)) != KX_OK) return s;
  long long ldl = ld, nl = n;
  void* args[] = {&T, &p, &Y, &ldl, &v, &gT, &gY, &nl};
  return launch(h, name, args, n, stream);
}

kx_status kx_kernel_info(kx_handle h, const char* kernel, int* registers, int* local_bytes, double* compile_seconds,
                         double* fp64_ops, double* fp32_ops, double* exps) {
  if (!h || !kernel) return fail(KX_ERR_ARG, "null argument");
  Kernel* k = find_kernel(h, kernel);
  if (!k) return fail(KX_ERR_ARG, std::string("no kernel ") + kernel);
  if (k->cubin.empty()) {
    std::lock_guard<std::mutex> lock(k->mu);
    if (k->cubin.empty()) {
      kx_status s = compile_kernel(h, *k);
      if (s != KX_OK) return s;
    }
  }
  if (registers) *registers = k->registers;
  if (local_bytes) *local_bytes = k->local_bytes;
  if (compile_seconds) *compile_seconds = k->compile_seconds;
  const kx::OpCounts& c = k->ops;
  if (fp64_ops) *fp64_ops = c.fp64;
  if (fp32_ops) *fp32_ops = c.fp32;
  if (exps) *exps = c.exp64 + c.exp32;
  return KX_OK;
}

kx_status kx_kernel_op_counts(kx_handle h, const char* kernel, double* counts) {
  if (!counts) return fail(KX_ERR_ARG, "null counts");
  if (!h || !kernel) return fail(KX_ERR_ARG, "null argument");
  Kernel* k = find_kernel(h, kernel);
  if (!k) return fail(KX_ERR_ARG, std::string("no kernel ") + kernel);
  {
    // the counts come from the emitter alone: emit the source if it is not there yet (no compile)
    std::lock_guard<std::mutex> lock(k->mu);
    if (k->source.empty()) {
      k->source = kx::emit_kernel(h->m, k->kind, k->eopt, k->entry, &k->ops);
      if (k->source.empty()) return fail(KX_ERR_UNSUPPORTED, "kernel " + k->name + " is not available");
    }
  }
  const kx::OpCounts& c = k->ops;
  const double v[8] = {c.fp64, c.fp32, c.exp64, c.log64, c.div64, c.exp32, c.log32, c.div32};
  std::memcpy(counts, v, sizeof v);
  return KX_OK;
}

int64_t kx_evaluate_host_bytes_per_state(kx_handle h, int outputs) {
  if (!h) return 0;
  const int64_t ns = h->m.ns;
  int64_t v = 2 + ns;                                   // T, p, Y
  if (outputs & KX_OUT_WDOT) v += ns;
  if (outputs & KX_OUT_THERMO) v += 2;
  if (outputs & KX_OUT_TRANSPORT) v += 2 + ns;
  return 8 * v;
}

kx_status kx_evaluate_host(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld, double* wdot,
                           double* cp, double* hmass, double* mu, double* lambda, double* Dk, int64_t ldo, int64_t n,
                           kx_precision precision, int outputs, void* workspace, size_t workspace_bytes,
                           int64_t max_chunk, void* stream_a, void* stream_b) {
  kx_status s = check_state(h, T, p, Y, ld, n);
  if (s != KX_OK) return s;
  if (outputs <= 0 || outputs > 7) return fail(KX_ERR_ARG, "no outputs selected");
  if (precision != KX_FP64 && precision != KX_MIXED) return fail(KX_ERR_ARG, "bad precision");
  if (((outputs & KX_OUT_WDOT) && !wdot) || ((outputs & KX_OUT_THERMO) && (!cp || !hmass)) ||
      ((outputs & KX_OUT_TRANSPORT) && (!mu || !lambda || !Dk)))
    return fail(KX_ERR_ARG, "null output");
  if (ldo < n) return fail(KX_ERR_ARG, "output leading dimension smaller than the point count");
  if (n == 0) return KX_OK;
  const int64_t ns = h->m.ns, per = kx_evaluate_host_bytes_per_state(h, outputs);
  // chunk: two slots in the workspace, a multiple of 256 states (32-byte aligned rows)
  int64_t c = (int64_t)(workspace_bytes / (2 * (size_t)per)) / 256 * 256;
  if (max_chunk > 0) c = std::min(c, std::max<int64_t>(256, max_chunk / 256 * 256));
  if (c < 256) return fail(KX_ERR_ARG, "workspace smaller than two chunks of 256 states");
  // ... and, where it holds one, a whole number of waves of the launched kernels (states that fill
  // every SM's resident blocks once): a partial last wave in every chunk would idle SMs per chunk
  // every chunk takes the production-rate kernel that one call over all n states would take, so
  // that the results do not depend on the chunking
  const char* wdot_name = nullptr;
  if ((s = wdot_kernel_for(h, n, precision, &wdot_name)) != KX_OK) return s;
  {
    const bool fp = precision == KX_FP64;
    std::vector<const char*> used;
    if (outputs & KX_OUT_WDOT) used.push_back(wdot_name);
    if (outputs & KX_OUT_THERMO) used.push_back("thermo");
    if (outputs & KX_OUT_TRANSPORT) { used.push_back(fp ? "visc_fp64" : "visc_mixed"); used.push_back(fp ? "diff_fp64" : "diff_mixed"); }
    int64_t wave = 0;
    for (const char* name : used) {
      Kernel* k = find_kernel(h, name);
      if (!k) return fail(KX_ERR_UNSUPPORTED, std::string("no kernel ") + name);
      if ((s = ensure_ready(h, *k)) != KX_OK) return s;
      wave = std::max<int64_t>(wave, (int64_t)k->max_blocks * (k->states_per_block > 0 ? k->states_per_block : k->eopt.block));
    }
    if (wave > 0 && c >= wave) c = c / wave * wave;
  }
  c = std::min(c, (n + 255) / 256 * 256);
  // the kernels of even chunks on stream_a and of odd chunks on a second compute stream of this call
  // (so that one chunk's last blocks overlap the next chunk's first: no SM idles at a kernel's
  // tail), the inputs copied in on stream_b one chunk ahead, the outputs copied out on a copy-out
  // stream of this call (so that the two copy directions run at once); per-slot events order them,
  // and on return stream_a and stream_b wait for everything the call's own streams hold
  cudaStream_t qa0 = (cudaStream_t)stream_a, qb = (cudaStream_t)stream_b;
  HostPipe* hp = nullptr;
  {
    int dev = 0;
    cudaError_t ge = cudaGetDevice(&dev);
    if (ge != cudaSuccess) return cuda_fail(ge, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(h->pipe_mu);
    for (size_t j = 0; j < h->free_pipes.size(); ++j)
      if (h->free_pipes[j]->device == dev) {
        hp = h->free_pipes[j];
        h->free_pipes.erase(h->free_pipes.begin() + (long)j);
        break;
      }
    if (!hp) {
      std::unique_ptr<HostPipe> np(new HostPipe());
      np->device = dev;
      cudaError_t e = cudaSuccess;
      for (int j = 0; j < 8 && e == cudaSuccess; ++j) e = cudaEventCreateWithFlags(&np->ev[j], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&np->qc, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&np->qd, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        for (cudaEvent_t x : np->ev) if (x) cudaEventDestroy(x);
        if (np->qc) cudaStreamDestroy(np->qc);
        if (np->qd) cudaStreamDestroy(np->qd);
        return cuda_fail(e, "evaluate_host streams and events");
      }
      hp = np.get();
      h->pipes.push_back(std::move(np));
    }
  }
  cudaStream_t qc = hp->qc, qd = hp->qd;
  cudaEvent_t* ev = hp->ev;
  // on return (also on an error): stream_b waits for the copy-out stream and stream_a for the odd
  // chunks' kernel stream, and the set goes back to the free list
  struct Guard {
    kx_mech* h;
    HostPipe* hp;
    cudaStream_t qa, qb;
    ~Guard() {
      if (cudaEventRecord(hp->ev[6], hp->qc) == cudaSuccess) cudaStreamWaitEvent(qb, hp->ev[6], 0);
      if (cudaEventRecord(hp->ev[7], hp->qd) == cudaSuccess) cudaStreamWaitEvent(qa, hp->ev[7], 0);
      std::lock_guard<std::mutex> lock(h->pipe_mu);
      h->free_pipes.push_back(hp);
    }
  } guard{h, hp, qa0, qb};
  {
    // the call's streams start after whatever the caller queued on stream_a and stream_b
    cudaError_t e = cudaEventRecord(ev[6], qb);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(qc, ev[6], 0);
    if (e == cudaSuccess && (e = cudaEventRecord(ev[7], qa0)) == cudaSuccess) e = cudaStreamWaitEvent(qd, ev[7], 0);
    if (e != cudaSuccess) return cuda_fail(e, "event ordering");
  }
  cudaEvent_t* in_done = ev;          // inputs of the slot copied in
  cudaEvent_t* comp_done = ev + 2;    // kernels of the slot finished
  cudaEvent_t* out_done = ev + 4;     // outputs of the slot copied out
  // chunk bounds: a first and a last chunk of about a quarter slot (the copy-in and the copy-out
  // that nothing hides are short; their kernels share the GPU with the neighbouring chunk's, which
  // run on the other stream), full slots between them.  Every bound is a multiple of 256 states, so
  // that each warp of a chunk holds the same states as in one call over all n: the float-pair rate
  // kernel's float32 path is chosen per warp
  std::vector<int64_t> at{0};
  {
    int64_t pos = 0;
    const bool ends = n > 2 * c && c >= 1024;
    const int64_t q = c / 4 / 256 * 256;
    if (ends) at.push_back(pos = q);
    while (pos < n) {
      int64_t next = std::min(n, pos + c);
      if (ends && next == n && (n - q) / 256 * 256 > pos) next = (n - q) / 256 * 256;
      at.push_back(pos = next);
    }
  }
  const int64_t nchunks = (int64_t)at.size() - 1;
  auto slot = [&](int64_t i, double** dT, double** dp, double** dY, double** dw, double** dcp, double** dh, double** dmu,
                  double** dl, double** dD) {
    double* b = (double*)((char*)workspace + (size_t)(i % 2) * (size_t)c * (size_t)per);
    *dT = b; *dp = b + c; *dY = b + 2 * c;
    double* nx = *dY + ns * c;
    *dw = *dcp = *dh = *dmu = *dl = *dD = nullptr;
    if (outputs & KX_OUT_WDOT) { *dw = nx; nx += ns * c; }
    if (outputs & KX_OUT_THERMO) { *dcp = nx; *dh = nx + c; nx += 2 * c; }
    if (outputs & KX_OUT_TRANSPORT) { *dmu = nx; *dl = nx + c; *dD = nx + 2 * c; }
  };
  auto copy_in = [&](int64_t i) -> kx_status {
    double *dT, *dp, *dY, *dw, *dcp, *dh, *dmu, *dl, *dD;
    slot(i, &dT, &dp, &dY, &dw, &dcp, &dh, &dmu, &dl, &dD);
    const int64_t c0 = at[i], m = at[i + 1] - at[i];
    // the slot's inputs are free once the kernels of chunk i - 2 finished
    cudaError_t e = i >= 2 ? cudaStreamWaitEvent(qb, comp_done[i % 2], 0) : cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(dT, T + c0, m * 8, cudaMemcpyHostToDevice, qb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, p + c0, m * 8, cudaMemcpyHostToDevice, qb);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    kx_status s2 = kx_copy_rows_async(dY, c, Y + c0, ld, ns, m, qb);
    if (s2 != KX_OK) return s2;
    e = cudaEventRecord(in_done[i % 2], qb);
    return e == cudaSuccess ? KX_OK : cuda_fail(e, "cudaEventRecord");
  };
  if ((s = copy_in(0)) != KX_OK) return s;
  for (int64_t i = 0; i < nchunks; ++i) {
    // the next chunk's inputs, into the other slot
    if (i + 1 < nchunks && (s = copy_in(i + 1)) != KX_OK) return s;
    double *dT, *dp, *dY, *dw, *dcp, *dh, *dmu, *dl, *dD;
    slot(i, &dT, &dp, &dY, &dw, &dcp, &dh, &dmu, &dl, &dD);
    const int64_t c0 = at[i], m = at[i + 1] - at[i];
    cudaStream_t qa = i % 2 ? qd : qa0;
    cudaError_t e = cudaStreamWaitEvent(qa, in_done[i % 2], 0);
    if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(qa, out_done[i % 2], 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    if ((outputs & KX_OUT_WDOT) && (s = production_rates_with(h, wdot_name, dT, dp, dY, c, dw, m, qa)) != KX_OK) return s;
    if ((outputs & KX_OUT_THERMO) && (s = kx_thermo(h, dT, dp, dY, c, dcp, dh, m, qa)) != KX_OK) return s;
    if ((outputs & KX_OUT_TRANSPORT) && (s = kx_transport(h, dT, dp, dY, c, dmu, dl, dD, m, precision, qa)) != KX_OK) return s;
    e = cudaEventRecord(comp_done[i % 2], qa);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(qc, comp_done[i % 2], 0);
    if (e != cudaSuccess) return cuda_fail(e, "event ordering");
    if ((outputs & KX_OUT_WDOT) && (s = kx_copy_rows_async(wdot + c0, ldo, dw, c, ns, m, qc)) != KX_OK) return s;
    if (outputs & KX_OUT_THERMO) {
      e = cudaMemcpyAsync(cp + c0, dcp, m * 8, cudaMemcpyDeviceToHost, qc);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hmass + c0, dh, m * 8, cudaMemcpyDeviceToHost, qc);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    }
    if (outputs & KX_OUT_TRANSPORT) {
      e = cudaMemcpyAsync(mu + c0, dmu, m * 8, cudaMemcpyDeviceToHost, qc);
      if (e == cudaSuccess) e = cudaMemcpyAsync(lambda + c0, dl, m * 8, cudaMemcpyDeviceToHost, qc);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
      if ((s = kx_copy_rows_async(Dk + c0, ldo, dD, c, ns, m, qc)) != KX_OK) return s;
    }
    e = cudaEventRecord(out_done[i % 2], qc);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  }
  return KX_OK;
}

kx_status kx_copy_rows_async(void* dst, int64_t dst_ld, const void* src, int64_t src_ld, int64_t rows, int64_t n,
                             void* stream) {
  if (rows < 0 || n < 0 || dst_ld < n || src_ld < n) return fail(KX_ERR_ARG, "bad row copy shape");
  if (rows == 0 || n == 0) return KX_OK;
  if (!dst || !src) return fail(KX_ERR_ARG, "null pointer");
  cudaError_t e = cudaMemcpy2DAsync(dst, (size_t)dst_ld * sizeof(double), src, (size_t)src_ld * sizeof(double),
                                    (size_t)n * sizeof(double), (size_t)rows, cudaMemcpyDefault, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync");
  return KX_OK;
}

kx_status kx_kernel_source_hash(kx_handle h, const char* kernel, uint64_t* hash) {
  if (!h || !kernel || !hash) return fail(KX_ERR_ARG, "null argument");
  kx_status s = kx_kernel_info(h, kernel, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
  if (s != KX_OK) return s;
  *hash = fnv1a(find_kernel(h, kernel)->source);
  return KX_OK;
}

kx_status kx_kernel_source(kx_handle h, const char* kernel, char* buf, size_t cap, size_t* len) {
  if (!h || !kernel || !len) return fail(KX_ERR_ARG, "null argument");
  kx_status s = kx_kernel_info(h, kernel, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
  if (s != KX_OK) return s;
  const std::string& src = find_kernel(h, kernel)->source;
  *len = src.size();
  if (buf && cap > 0) {
    const size_t m = std::min(cap - 1, src.size());
    std::memcpy(buf, src.data(), m);
    buf[m] = '\0';
  }
  return KX_OK;
}

}  // extern "C"
