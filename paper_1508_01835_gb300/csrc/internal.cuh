// internal.cuh -- shared types of the IFMM CUDA library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ifmm.h"

namespace ifmm {

struct Error : std::runtime_error {
  ifmm_status st;
  Error(ifmm_status s, const std::string& m) : std::runtime_error(m), st(s) {}
};

inline void cuda_check(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    throw Error(IFMM_ERR_OOM, std::string(what) + ": out of device memory");
  }
  if (e != cudaSuccess) throw Error(IFMM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(x) ::ifmm::cuda_check((x), #x)
// every launch site of the library is followed by CK_LAUNCH, which also counts
// it: into the process-wide total, or into the capturing thread's count while a
// graph is being recorded (the graph adds its count at every replay)
void count_launch();
unsigned long long launches_total();
#define CK_LAUNCH(name) \
  (::ifmm::count_launch(), ::ifmm::cuda_check(cudaGetLastError(), name))

inline void require(bool ok, const std::string& m) {
  if (!ok) throw Error(IFMM_ERR_INVALID_ARG, m);
}

// ---------------------------------------------------------------------------
// Optional host-side bounds validation (IFMM_VALIDATE=1): every device range
// handed out by an Arena, and every caller buffer, is registered; before a
// launch the task builders check each descriptor's extent against them and
// throw instead of launching an out-of-range access.
// ---------------------------------------------------------------------------
struct Ranges {
  static bool on() {
    static const bool v = [] {
      const char* e = std::getenv("IFMM_VALIDATE");
      return e && e[0] == '1';
    }();
    return v;
  }
  static std::map<uintptr_t, size_t>& map() {
    static std::map<uintptr_t, size_t> m;
    return m;
  }
  static std::mutex& mu() {
    static std::mutex m;
    return m;
  }
  static void add(const void* p, size_t n) {
    if (!on() || !p) return;
    std::lock_guard<std::mutex> g(mu());
    map()[(uintptr_t)p] = n;
  }
  static void remove(const void* p) {
    if (!on() || !p) return;
    std::lock_guard<std::mutex> g(mu());
    map().erase((uintptr_t)p);
  }
  // registers [p, p + n) unless an existing range already holds it; true if added
  static bool add_if_uncovered(const void* p, size_t n) {
    if (!on() || !p || n == 0) return false;
    std::lock_guard<std::mutex> g(mu());
    auto& m = map();
    auto it = m.upper_bound((uintptr_t)p);
    if (it != m.begin()) {
      --it;
      if ((uintptr_t)p >= it->first && (uintptr_t)p + n <= it->first + it->second) return false;
    }
    if (m.count((uintptr_t)p)) return false;
    m[(uintptr_t)p] = n;
    return true;
  }
  static void check(const void* p, size_t bytes, const char* what) {
    if (!on() || bytes == 0) return;
    std::lock_guard<std::mutex> g(mu());
    auto& m = map();
    auto it = m.upper_bound((uintptr_t)p);
    bool ok = false;
    if (it != m.begin()) {
      --it;
      ok = (uintptr_t)p >= it->first && (uintptr_t)p + bytes <= it->first + it->second;
    }
    if (!ok) throw Error(IFMM_ERR_CUDA, std::string("bounds check failed: ") + what);
  }
};
// bytes spanned by a column-major rows x cols matrix with leading dimension ld
inline size_t mat_bytes(long long rows, long long cols, long long ld, size_t elem = 8) {
  if (rows <= 0 || cols <= 0) return 0;
  if (cols > 1 && ld < rows)
    throw Error(IFMM_ERR_CUDA, "bounds check failed: leading dimension < rows");
  return (size_t)((cols - 1) * ld + rows) * elem;
}
// a caller's buffer registered for the duration of one call (left alone when a
// registered allocation already holds it)
struct ScopedRange {
  const void* p;
  bool added;
  ScopedRange(const void* q, size_t n) : p(q), added(Ranges::add_if_uncovered(q, n)) {}
  ~ScopedRange() {
    if (added) Ranges::remove(p);
  }
};

// ---------------------------------------------------------------------------
// Launch profiler (profile.cu): Prof p("k_gemm", flops, bytes, stream) before
// a launch, destroyed after it, records an event pair when profiling is on.
// ---------------------------------------------------------------------------
namespace prof {
bool enabled();
void* begin(const char* name, double flops, double bytes, cudaStream_t s);
void end(void* token, cudaStream_t s);
void start();
int stop(ifmm_kernel_stat* out, int capacity);
// While a launch sequence is captured into a graph, profiled launches add
// their flops and bytes here instead of recording events.
struct Capture { double flops = 0.0, bytes = 0.0; };
Capture*& capture();
}  // namespace prof
struct Prof {
  void* tok = nullptr;
  cudaStream_t s;
  Prof(const char* name, double flops, double bytes, cudaStream_t st) : s(st) {
    if (prof::Capture* c = prof::capture()) {
      c->flops += flops;
      c->bytes += bytes;
      return;
    }
    if (prof::enabled()) tok = prof::begin(name, flops, bytes, st);
  }
  ~Prof() { if (tok) prof::end(tok, s); }
};

// A fixed launch sequence replayed as one CUDA graph.  The sequence is
// captured on a private stream the first time (and again when `key` changes)
// and launched on the caller's stream; a profiled replay is one entry named
// `name` carrying the summed flops and bytes of the captured launches, and
// each replay adds the captured kernel count to the launch counter.
// IFMM_GRAPHS=0 runs the sequence directly instead.
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  long long key = -1;
  unsigned long long kernels = 0;
  double flops = 0.0, bytes = 0.0;
  GraphCache() = default;
  GraphCache(const GraphCache&) = delete;
  GraphCache& operator=(const GraphCache&) = delete;
  void reset();
  ~GraphCache();
};
bool graphs_enabled();
void run_graph(GraphCache& g, long long key, const char* name, cudaStream_t s,
               const std::function<void(cudaStream_t)>& body);
// One graph per key (the right-hand-side count of a plan built for more
// columns), so alternating block widths replay instead of re-capturing.
struct GraphSet {
  std::map<long long, std::unique_ptr<GraphCache>> g;
  GraphCache& at(long long key) {
    std::unique_ptr<GraphCache>& p = g[key];
    if (!p) p.reset(new GraphCache());
    return *p;
  }
  void reset() { g.clear(); }
};

// ---------------------------------------------------------------------------
// Device memory: a chunked bump allocator.  Blocks are 256-byte aligned.
// reset() rewinds without freeing, so per-colour scratch reuses its chunks.
// ---------------------------------------------------------------------------
struct Arena {
  size_t chunk_bytes = size_t(256) << 20;
  std::vector<std::pair<char*, size_t>> chunks;
  size_t cur = 0;       // index of the chunk being filled
  size_t off = 0;       // bytes used in it
  size_t held = 0;      // bytes of device memory held
  size_t high = 0;      // bytes handed out since the last reset
  Arena() = default;
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  ~Arena() { release(); }
  char* alloc_bytes(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    while (cur < chunks.size()) {
      if (off + bytes <= chunks[cur].second) {
        char* p = chunks[cur].first + off;
        off += bytes;
        high += bytes;
        return p;
      }
      cur++;
      off = 0;
    }
    size_t sz = bytes > chunk_bytes ? bytes : chunk_bytes;
    char* p = nullptr;
    CK(cudaMalloc(&p, sz));
    Ranges::add(p, sz);
    chunks.push_back({p, sz});
    held += sz;
    cur = chunks.size() - 1;
    off = bytes;
    high += bytes;
    return p;
  }
  template <class T>
  T* alloc(size_t n) { return reinterpret_cast<T*>(alloc_bytes(n * sizeof(T))); }
  void reset() { cur = 0; off = 0; high = 0; }
  void release() {
    for (auto& c : chunks) {
      Ranges::remove(c.first);
      cudaFree(c.first);
    }
    chunks.clear();
    cur = off = held = high = 0;
  }
};

// cudaFuncSetAttribute(fn, MaxDynamicSharedMemorySize, bytes) once per device
// (thread-safe).
void set_max_dynamic_smem(const void* fn, int bytes);

// A device copy of a host vector of POD tasks.
template <class T>
T* upload(Arena& ar, const std::vector<T>& v, cudaStream_t s) {
  if (v.empty()) return nullptr;
  T* d = ar.alloc<T>(v.size());
  CK(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return d;
}

// ---------------------------------------------------------------------------
// Batched dense kernels (kernels_linalg.cu).  All matrices are FP64
// column-major; element (r, c) of a matrix with leading dimension ld is
// p[r + c * ld].
// ---------------------------------------------------------------------------

// dst(r, c) = beta * dst(r, c) + alpha * S(r, c) * (cscale ? cscale[c] : 1)
// S = src(r, c), src(c, r) (trans), the identity (kind 1) or zero (kind 2).
// beta == 0 never reads dst.
struct CopyTask {
  const double* src;
  double* dst;
  const double* cscale;
  int lds, ldd, rows, cols;
  int trans, kind;
  double alpha, beta;
};
void launch_copy(const CopyTask* d_tasks, int ntasks, cudaStream_t s);
void validate(const CopyTask& t);

// C = alpha op(A) op(B) + beta C; beta == 0 never reads C.
struct GemmTask {
  const double* A;
  const double* B;
  double* C;
  int lda, ldb, ldc;
  int M, N, K;
  int transA, transB;
  double alpha, beta;
};
struct GemmTile {
  int task, m0, n0;
};
void validate(const GemmTask& t);
// Host helper: append the 64x64 output tiles of task `t`.
void gemm_tiles(const GemmTask& t, int task_index, std::vector<GemmTile>& tiles);
void launch_gemm(const GemmTask* d_tasks, const GemmTile* d_tiles, int ntiles, cudaStream_t s,
                 double flops = 0.0);
// Convenience: run a host list of GEMM tasks (uploads into `ar`).
void run_gemms(Arena& ar, const std::vector<GemmTask>& tasks, cudaStream_t s);

// Tensor-core form of run_gemms for the Schur products (kernels_tc.cu):
// operands packed once (TF32, TF32 head + tail for the three-term compensated
// product, or BF16; prec = IFMM_P_TF32 / IFMM_P_FP32 / IFMM_P_BF16), 128 x 128
// output tiles of a persistent pipelined kernel, FP32 accumulation in tensor
// memory, FP64 epilogue.  *d_err is set to 1 if a bounded wait ran out.
void run_gemms_tc(Arena& ar, const std::vector<GemmTask>& tasks, int prec, int* d_err,
                  cudaStream_t s);

// Edge redirection of Algorithm 3 (kernels_edges.cu), one CTA per
// recompressed box.  Per level (device arrays, uploaded once): interaction
// lists and, for list entry k of box j with q = far[k], the blocks K(j, q)
// (y_out[k], ld rcap[j]) and K(q, j) (y_in[k], ld rcap[q]).
struct EdgeLevel {
  const int* far_ptr;
  const int* far;
  double* const* y_out;
  double* const* y_in;
  const int* rcap;
};
// Per colour: ranks before / after recompression of every box of the level,
// r_j (rm, r_new x r_old, ld r_new) and t_j (tm, same shape) of the
// recompressed boxes (null for the others), and the recompressed boxes.
struct EdgeColour {
  const int* r_old;
  const int* r_new;
  const double* const* rm;
  const double* const* tm;
  const int* boxes;
  int rmax;  // largest rank (old or new) of any box touched, <= 64
};
void launch_edge_redirect(const EdgeLevel& L, const EdgeColour& E, int nboxes, cudaStream_t s,
                          double flops);

// Batched LU with partial pivoting (right-looking, panel width LU_NB).
struct LuTask {
  double* A;
  int lda, n;
  int* piv;      // n entries, 0-based global row swapped with row k at step k
  int* info;     // 0, or 1 + first column whose pivot failed the test
  double* amax;  // scratch: max |A| before factorisation
};
constexpr int LU_NB = 64;
void run_getrf(Arena& ar, const std::vector<LuTask>& tasks, cudaStream_t s);

// X = A^-1 B in place of B, with A = P L U from run_getrf.
struct RsTask {
  const double* LU;
  int lda, n;
  const int* piv;
  double* B;
  int ldb, ncols;
};
void run_getrs(Arena& ar, const std::vector<RsTask>& tasks, cudaStream_t s);

// Pre-uploaded form of run_getrs: every launch's task arrays live in the
// arena given to plan_getrs, so exec_getrs can be replayed without host work.
struct GemmLaunch {
  const GemmTask* tasks = nullptr;
  const GemmTile* tiles = nullptr;
  int ntiles = 0;
  double flops = 0.0;
};
GemmLaunch plan_gemms(Arena& ar, const std::vector<GemmTask>& tasks, cudaStream_t s);
struct GetrsPlan {
  const RsTask* d = nullptr;
  int nt = 0, nmax = 0, gy = 1;
  std::vector<GemmLaunch> fwd, bwd;  // per panel, forward / backward order
  // Few right-hand sides (<= GETRS_SMALL_COLS): solved panel by panel, every
  // panel one launch over all tasks, with the inverses of the diagonal blocks
  // formed once when the plan is made.
  bool panel = false;
  const struct RsPanel* pd = nullptr;
  int nblk_max = 0;
};
constexpr int GETRS_SMALL_COLS = 8;
constexpr int GETRS_PANEL = 64;   // panel width of the panel solve
constexpr int GETRS_PROWS = 128;  // rows of the update per CTA
struct RsPanel {
  const double* LU;
  int lda, n;
  const int* perm;  // row interchanges as a gather index: (P b)[i] = b[perm[i]]
  double* B;
  int ldb, ncols;
  double *w1, *w2;  // n x ncols each (ld n): gathered input / forward result
  double* dinv;     // 2 nblk blocks of 64 x 64 (ld 64): inverses of the diagonal
                    // blocks of L (unit lower), then of U
  int nblk;
};
GetrsPlan plan_getrs(Arena& ar, const std::vector<RsTask>& tasks, cudaStream_t s);
void exec_getrs(const GetrsPlan& p, cudaStream_t s);

// Left singular vectors and values of M (a x w, a <= w after zero padding is
// implied): W (a x a, ld a) and sigma (a), sorted by decreasing sigma.
// work: a*a + 16a doubles of scratch for a > SVD_SMEM_A (null: taken from the
// arena given to run_svd_left); unused otherwise.
struct SvdTask {
  const double* M;
  int ldm, a, w;
  double* W;
  double* sigma;
  double* work;
};
void run_svd_left(Arena& ar, const std::vector<SvdTask>& tasks, cudaStream_t s);
// FP64 flops of the one-sided Jacobi sweeps of every k_svd_left CTA since the
// last call (device counter, read and reset; synchronises the device).  The
// launch profiler adds them to k_svd_left's counted flops (the streaming LQ
// part, 2 a^2 w per task, is counted at launch).
unsigned long long svd_jacobi_flops_take();

// Randomised left SVD (Sec. 2.4) for blocks taller than rsvd_rows: top k left singular
// vectors W (a x k, ld a) and values sigma (k); every task of a call has the same k.
struct RsvdTask {
  const double* M;
  int ldm, a, w, k;
  unsigned long long seed;
  double* W;
  double* sigma;
};
void run_rsvd_left(Arena& ar, const std::vector<RsvdTask>& tasks, cudaStream_t s);
constexpr int SVD_SMEM_A = 160;       // largest block the shared-memory SVD takes
constexpr int SVD_SMEM_BUDGET = 29000;  // doubles of dynamic shared memory per SVD CTA
constexpr int RSVD_ROWS_DEFAULT = 160;  // truncated blocks taller than this use run_rsvd_left
constexpr int RSVD_OVERSAMPLE = 16;  // oversampling p of the randomised SVD (Sec. 2.4)
unsigned long long rsvd_seed(int level, int box, int side);
// inv[c] = 1 / s[c] where s[c] > 1e-10 s[0], else 0
struct InvSigma {
  const double* s;
  double* inv;
  int k;
};
void run_inv_sigma(Arena& ar, const std::vector<InvSigma>& v, cudaStream_t s);

// r_out[j] = min(max(#(sigU > tau), #(sigV > tau)), full, cap) (tau <= 0: full)
struct RankTask {
  const double* sigU;
  const double* sigV;
  int full;  // number of singular values available (= a)
  int cap;
  int* out;
  int* capped;  // incremented when the cap binds
};
void launch_rank(const RankTask* d, int n, double tau, cudaStream_t s);

// ---------------------------------------------------------------------------
// Block-row sparse products (kernels_ops.cu): for each output row-block
// y = beta y + sum_e alpha_e op(A_e) x_e, nrhs columns.  A == nullptr means
// the identity.  Column c of x / y sits at x + c * ldx / y + c * ldy.
// ---------------------------------------------------------------------------
struct SpRow {
  double* y;
  long long ldy;
  int m;
  int e0, ne;
  double beta;
};
struct SpEnt {
  const double* A;
  const double* x;
  long long ldx;
  int lda, k, transA;
  double alpha;
};
void validate_spmm(const std::vector<SpRow>& rows, const std::vector<SpEnt>& ents, int nrhs);

// Work split of one launch.  A job sums one contiguous range of a row's
// concatenated columns (entries in order, each contributing k columns) over
// segments; a row whose work exceeds the per-job target is split over several
// jobs that write partial sums, and a second pass adds them in job order, so
// results do not depend on scheduling.
struct SpJob {
  int row, s0, ns;
  int r0, mt;      // rows r0 .. r0 + mt - 1 of the row (one tile of 8, 16 or 32 rows)
  long long part;  // offset of this job's partial sums (mt rows); < 0: the job writes y
};
struct SpSeg { int ent, k0, k1; };
struct SpRed {
  int row, nj, r0, mt;
  long long base;  // partial sums of job j of the tile at base + j * mt
};
struct SpmmPlan {
  const SpRow* rows = nullptr;
  const SpEnt* ents = nullptr;
  const SpJob* jobs = nullptr;
  const SpSeg* segs = nullptr;
  const SpRed* reds = nullptr;
  int njobs = 0, nreds = 0;
  int ncls[3] = {0, 0, 0};  // jobs per row class (m <= 8, <= 16, > 16), in that order
  double* part = nullptr;   // partial sums: part[job.part + r + c * part_ld]
  long long part_ld = 0;
  int cap = 0;              // right-hand sides per pass
  double flops = 0.0;   // per right-hand side
  double bytes = 0.0;   // matrix entries, read once per pass of <= 32 right-hand sides
  double vbytes = 0.0;  // x and y per right-hand side
};
// Plans rows/ents (uploaded to `ar`, with room for `cap` right-hand sides).
SpmmPlan plan_spmm(Arena& ar, const std::vector<SpRow>& rows, const std::vector<SpEnt>& ents,
                   int cap, cudaStream_t s);
void launch_spmm(const SpmmPlan& p, int nrhs, cudaStream_t s);

// FP32 block-row products (the reduced-precision substitution sweeps):
// y = beta y + sum_e alpha_e A_e x_e, A non-transposed (or nullptr: identity).
struct SpRowF {
  float* y;
  long long ldy;
  int m;
  int e0, ne;
  float beta;
};
struct SpEntF {
  const float* A;
  const float* x;
  long long ldx;
  int lda, k;
  float alpha;
};
struct SpmmPlanF {
  const SpRowF* rows = nullptr;
  const SpEntF* ents = nullptr;
  const SpJob* jobs = nullptr;
  const SpSeg* segs = nullptr;
  const SpRed* reds = nullptr;
  int njobs = 0, nreds = 0;
  int ncls[3] = {0, 0, 0};  // jobs per row class (m <= 8, <= 16, > 16), in that order
  float* part = nullptr;
  long long part_ld = 0;
  int cap = 0;
  double flops = 0.0;   // per right-hand side
  double bytes = 0.0;   // matrix entries, read once per pass of <= 32 right-hand sides
  double vbytes = 0.0;  // x and y per right-hand side
};
SpmmPlanF plan_spmm_f32(Arena& ar, const std::vector<SpRowF>& rows,
                        const std::vector<SpEntF>& ents, int cap, cudaStream_t s);
void launch_spmm_f32(const SpmmPlanF& p, int nrhs, cudaStream_t s);
void launch_gather_rows_f32(const long long* perm, long long N, const double* in, long long ldi,
                            float* out, long long ldo, int ncols, cudaStream_t s);
void launch_scatter_rows_f32(const long long* perm, long long N, const float* in, long long ldi,
                             double* out, long long ldo, int ncols, cudaStream_t s);
struct NarrowTask {
  const double* src;
  float* dst;
  long long n;
};
void launch_narrow(Arena& ar, const std::vector<NarrowTask>& v, cudaStream_t s);

// Block rows whose blocks are all nd x nd (M2M, M2L, L2L; kernels_m2l.cu):
// tables stored as nd columns of ndp = uniform_ndp(nd) entries (zero padded),
// coefficient vectors with ndp entries per box; y, A, x 16-byte aligned.
template <class T>
struct UniRow {
  T* y;
  long long ldy;
  int e0, ne;
};
template <class T>
struct UniEnt {
  const T* A;
  const T* x;
  long long ldx;
};
template <class T>
struct UniPlan {
  const UniRow<T>* rows = nullptr;
  const UniEnt<T>* ents = nullptr;
  int nrows = 0, nd = 0, ndp = 0;
  double flops = 0.0, bytes = 0.0;  // flops per right-hand side; bytes per pass
};
int uniform_ndp(int nd);
bool uniform_supported(int nd);
template <class T>
UniPlan<T> plan_uniform(Arena& ar, const std::vector<UniRow<T>>& rows,
                        const std::vector<UniEnt<T>>& ents, int nd, int cap, cudaStream_t s);
template <class T>
void launch_uniform(const UniPlan<T>& p, int nrhs, cudaStream_t s);
// count FP64 tables nd x nd (column-major; transposed if asked) to the padded
// layout above, in T
template <class T>
void launch_pad_tables(const double* src, T* dst, int count, int nd, bool transpose,
                       cudaStream_t s);

// dst (cols x rows, ld cols) = FP32 transpose of src (rows x cols, ld rows)
struct NarrowTTask {
  const double* src;
  float* dst;
  int rows, cols;
};
void launch_narrow_t(Arena& ar, const std::vector<NarrowTTask>& v, cudaStream_t s);
// out64[t, c] = in[perm[t], c] and out32[t, c] = (float) in[perm[t], c]
void launch_gather_rows_2(const long long* perm, long long N, const double* in, long long ldi,
                          double* out64, float* out32, long long ldo, int ncols, cudaStream_t s);
// out[perm[t], c] = in64[t, c] + (double) in32[t, c]
void launch_scatter_rows_add(const long long* perm, long long N, const double* in64,
                             const float* in32, long long ldi, double* out, long long ldo,
                             int ncols, cudaStream_t s);

}  // namespace ifmm
