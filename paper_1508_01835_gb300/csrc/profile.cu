// profile.cu -- optional timing of the library's own launches.
//
// When enabled, every profiled launch is bracketed by two CUDA events on the
// stream it is launched on, tagged with the kernel name and the algorithmic
// flops and bytes of that launch.  Collection synchronises once and sums the
// event intervals per kernel name.
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <set>

#include "system.cuh"

namespace ifmm {

static std::atomic<unsigned long long> g_launches{0};
static thread_local bool t_capturing = false;
static thread_local unsigned long long t_captured = 0;

void count_launch() {
  if (t_capturing) t_captured++;
  else g_launches.fetch_add(1, std::memory_order_relaxed);
}
unsigned long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

namespace prof {

struct Pending {
  const char* name;
  cudaEvent_t a, b;
  double flops, bytes;
};
struct Stat {
  long long launches = 0;
  double seconds = 0.0, flops = 0.0, bytes = 0.0;
};

static std::mutex mu;
static bool on = false;
static std::vector<Pending> pending;
static std::vector<cudaEvent_t> pool;
static std::map<std::string, Stat> stats;
static unsigned long long launches_at_start = 0;

static cudaEvent_t get_event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  return e;
}

bool enabled() { return on; }

Capture*& capture() {
  thread_local Capture* c = nullptr;
  return c;
}

void* begin(const char* name, double flops, double bytes, cudaStream_t s) {
  if (!on) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  Pending p{name, get_event(), get_event(), flops, bytes};
  CK(cudaEventRecord(p.a, s));
  pending.push_back(p);
  return reinterpret_cast<void*>(pending.size());
}

void end(void* token, cudaStream_t s) {
  if (!on || !token) return;
  std::lock_guard<std::mutex> g(mu);
  const size_t i = reinterpret_cast<size_t>(token) - 1;
  CK(cudaEventRecord(pending[i].b, s));
}

static void drain() {
  CK(cudaDeviceSynchronize());
  for (Pending& p : pending) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, p.a, p.b));
    Stat& st = stats[p.name];
    st.launches++;
    st.seconds += ms * 1e-3;
    st.flops += p.flops;
    st.bytes += p.bytes;
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
}

void start() {
  std::lock_guard<std::mutex> g(mu);
  if (on) drain();
  stats.clear();
  svd_jacobi_flops_take();
  launches_at_start = launches_total();
  on = true;
}

int stop(ifmm_kernel_stat* out, int capacity) {
  std::lock_guard<std::mutex> g(mu);
  drain();
  on = false;
  {
    auto it = stats.find("k_svd_left");
    const double jf = (double)svd_jacobi_flops_take();
    if (it != stats.end()) it->second.flops += jf;
  }
  Stat& all = stats["(all launches)"];
  all.launches = (long long)(launches_total() - launches_at_start);
  int n = 0;
  for (auto& kv : stats) {
    if (out && n < capacity) {
      ifmm_kernel_stat& o = out[n];
      std::memset(&o, 0, sizeof(o));
      std::strncpy(o.name, kv.first.c_str(), sizeof(o.name) - 1);
      o.launches = kv.second.launches;
      o.seconds = kv.second.seconds;
      o.flops = kv.second.flops;
      o.bytes = kv.second.bytes;
    }
    n++;
  }
  return n;
}

}  // namespace prof

void set_max_dynamic_smem(const void* fn, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(mu);
  if (done.count({fn, dev})) return;
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert({fn, dev});
}

bool graphs_enabled() {
  static const bool v = [] {
    const char* e = std::getenv("IFMM_GRAPHS");
    return !(e && e[0] == '0');
  }();
  return v;
}

void GraphCache::reset() {
  if (exec) cudaGraphExecDestroy(exec);
  exec = nullptr;
  key = -1;
}

GraphCache::~GraphCache() {
  reset();
  if (cs) cudaStreamDestroy(cs);
}

void run_graph(GraphCache& g, long long key, const char* name, cudaStream_t s,
               const std::function<void(cudaStream_t)>& body) {
  // while the launch profile records, run the body eagerly so that every
  // kernel gets its own event pair (a graph replay would be one interval)
  if (!graphs_enabled() || prof::enabled()) {
    body(s);
    return;
  }
  if (!g.exec || g.key != key) {
    g.reset();
    if (!g.cs) CK(cudaStreamCreateWithFlags(&g.cs, cudaStreamNonBlocking));
    prof::Capture cap;
    CK(cudaStreamBeginCapture(g.cs, cudaStreamCaptureModeThreadLocal));
    prof::capture() = &cap;
    t_capturing = true;
    t_captured = 0;
    cudaGraph_t gr = nullptr;
    try {
      body(g.cs);
    } catch (...) {
      prof::capture() = nullptr;
      t_capturing = false;
      cudaStreamEndCapture(g.cs, &gr);
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
      throw;
    }
    prof::capture() = nullptr;
    t_capturing = false;
    CK(cudaStreamEndCapture(g.cs, &gr));
    g.kernels = t_captured;
    const cudaError_t e = cudaGraphInstantiate(&g.exec, gr, 0);
    cudaGraphDestroy(gr);
    CK(e);
    g.key = key;
    g.flops = cap.flops;
    g.bytes = cap.bytes;
  }
  Prof p(name, g.flops, g.bytes, s);
  CK(cudaGraphLaunch(g.exec, s));
  g_launches.fetch_add(g.kernels, std::memory_order_relaxed);
}

}  // namespace ifmm

// ---------------------------------------------------------------------------
// Peak arithmetic rates of this GPU, measured: every thread runs NCHAIN
// independent FMA chains of `iters` steps (so the pipe, not the latency,
// bounds the rate), over a grid of 8 CTAs of 256 threads per SM; rate =
// 2 x FMAs / CUDA-event time of the launch (after one warm-up launch).
// ---------------------------------------------------------------------------
namespace ifmm {
template <class T>
__global__ void __launch_bounds__(256) k_fma_rate(T* out, int iters, T seed) {
  constexpr int NCHAIN = 8;
  T a[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; c++) a[c] = seed + (T)(threadIdx.x + c);
  const T m = (T)0.999999, d = (T)1e-7;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < NCHAIN; c++) a[c] = a[c] * m + d;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < NCHAIN; c++) s += a[c];
  if (s == (T)-1.2345) out[0] = s;  // never true: keeps the chains live
}

template <class T>
static double fma_rate(int iters) {
  int dev = 0, nsm = 1;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  T* out = nullptr;
  CK(cudaMalloc(&out, sizeof(T)));
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  const int grid = nsm * 8;
  k_fma_rate<T><<<grid, 256>>>(out, iters / 10, (T)1);
  CK_LAUNCH("k_fma_rate");
  CK(cudaEventRecord(a));
  k_fma_rate<T><<<grid, 256>>>(out, iters, (T)1);
  CK_LAUNCH("k_fma_rate");
  CK(cudaEventRecord(b));
  CK(cudaEventSynchronize(b));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  const double fmas = (double)grid * 256 * 8 * (double)iters;
  return 2.0 * fmas / (ms * 1e-3) / 1e12;
}
}  // namespace ifmm

extern "C" ifmm_status ifmm_measure_peaks(ifmm_ctx* ctx, double* fp64_tflops, double* fp32_tflops) {
  if (!ctx || !fp64_tflops || !fp32_tflops) return IFMM_ERR_INVALID_ARG;
  try {
    CK(cudaSetDevice(ctx->device));
    *fp64_tflops = ifmm::fma_rate<double>(1 << 14);
    *fp32_tflops = ifmm::fma_rate<float>(1 << 17);
    return IFMM_OK;
  } catch (const ifmm::Error& e) {
    ctx->last_error = e.what();
    return e.st;
  } catch (const std::exception& e) {
    ctx->last_error = e.what();
    return IFMM_ERR_CUDA;
  }
}

extern "C" ifmm_status ifmm_launch_count(unsigned long long* launches) {
  if (!launches) return IFMM_ERR_INVALID_ARG;
  *launches = ifmm::launches_total();
  return IFMM_OK;
}
