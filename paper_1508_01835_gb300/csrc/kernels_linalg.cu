// kernels_linalg.cu -- batched FP64 dense kernels of the IFMM factorisation.
//
// The elimination of a box (Sec. 2.2, Algorithm 2) is a block Gaussian
// elimination: LU of the pivot block E(P,P) with partial pivoting, the solve
// G = E(P,P)^-1 E(P,C), the Schur product E(R,P) G, and truncated SVDs of the
// fill-in and of the weighted bases (Eqs. P2P_kj, U_j_recomp, V_j_recomp).
// Each kernel here runs one such operation for every box of a colour in one
// launch (boxes of a colour are independent).
#include <cfloat>

#include "internal.cuh"

#include <chrono>
#include <cstdio>
#include <cstdlib>

namespace ifmm {

// ---------------------------------------------------------------------------
// block copy / axpby / identity
// ---------------------------------------------------------------------------
__global__ void k_copy(const CopyTask* __restrict__ tasks) {
  const CopyTask t = tasks[blockIdx.x];
  const long long total = (long long)t.rows * t.cols;
  const long long per = (total + gridDim.y - 1) / gridDim.y;
  const long long e0 = per * blockIdx.y;
  const long long e1 = min(total, e0 + per);
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int r = (int)(e % t.rows);
    const int c = (int)(e / t.rows);
    double s;
    if (t.kind == 1) s = (r == c) ? 1.0 : 0.0;
    else if (t.kind == 2) s = 0.0;
    else s = t.trans ? t.src[c + (long long)r * t.lds] : t.src[r + (long long)c * t.lds];
    if (t.cscale) s *= t.cscale[c];
    double* d = t.dst + r + (long long)c * t.ldd;
    *d = (t.beta == 0.0) ? t.alpha * s : t.beta * (*d) + t.alpha * s;
  }
}

void validate(const CopyTask& t) {
  if (!Ranges::on() || t.rows <= 0 || t.cols <= 0) return;
  Ranges::check(t.dst, mat_bytes(t.rows, t.cols, t.ldd), "copy dst");
  if (t.kind == 0)
    Ranges::check(t.src, t.trans ? mat_bytes(t.cols, t.rows, t.lds) : mat_bytes(t.rows, t.cols, t.lds),
                  "copy src");
  if (t.cscale) Ranges::check(t.cscale, sizeof(double) * t.cols, "copy scale");
}

void validate(const GemmTask& t) {
  if (!Ranges::on() || t.M <= 0 || t.N <= 0) return;
  Ranges::check(t.C, mat_bytes(t.M, t.N, t.ldc), "gemm C");
  if (t.K <= 0) return;
  Ranges::check(t.A, t.transA ? mat_bytes(t.K, t.M, t.lda) : mat_bytes(t.M, t.K, t.lda), "gemm A");
  Ranges::check(t.B, t.transB ? mat_bytes(t.N, t.K, t.ldb) : mat_bytes(t.K, t.N, t.ldb), "gemm B");
}

void launch_copy(const CopyTask* d_tasks, int ntasks, cudaStream_t s) {
  if (ntasks <= 0) return;
  dim3 grid(ntasks, 16);
  k_copy<<<grid, 256, 0, s>>>(d_tasks);
  CK_LAUNCH("k_copy");
}

// ---------------------------------------------------------------------------
// tiled FP64 GEMM over a list of output tiles (64 x 64, 256 threads, 4x4 each)
// ---------------------------------------------------------------------------
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) k_gemm(const GemmTask* __restrict__ tasks,
                                              const GemmTile* __restrict__ tiles) {
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask t = tasks[tl.task];
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < t.K; k0 += GK) {
    for (int idx = threadIdx.x; idx < GT * GK; idx += 256) {
      int m, k;
      if (t.transA) { k = idx % GK; m = idx / GK; }
      else { m = idx % GT; k = idx / GT; }
      const int gm = tl.m0 + m, gk = k0 + k;
      double v = 0.0;
      if (gm < t.M && gk < t.K)
        v = t.transA ? t.A[gk + (long long)gm * t.lda] : t.A[gm + (long long)gk * t.lda];
      As[k][m] = v;
    }
    for (int idx = threadIdx.x; idx < GT * GK; idx += 256) {
      int n, k;
      if (t.transB) { n = idx % GT; k = idx / GT; }
      else { k = idx % GK; n = idx / GK; }
      const int gn = tl.n0 + n, gk = k0 + k;
      double v = 0.0;
      if (gn < t.N && gk < t.K)
        v = t.transB ? t.B[gn + (long long)gk * t.ldb] : t.B[gk + (long long)gn * t.ldb];
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GK; k++) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int gm = tl.m0 + ty + 16 * i;
    if (gm >= t.M) continue;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int gn = tl.n0 + tx + 16 * j;
      if (gn >= t.N) continue;
      double* c = t.C + gm + (long long)gn * t.ldc;
      *c = (t.beta == 0.0) ? t.alpha * acc[i][j] : t.beta * (*c) + t.alpha * acc[i][j];
    }
  }
}

// Small tiles for small products (M, N <= 32): 32 x 32 outputs, 64 threads
// with 4 x 4 each, so a 16 x 16 result does not pay for a 64 x 64 tile.
constexpr int ST = 32;
__global__ void __launch_bounds__(64) k_gemm_small(const GemmTask* __restrict__ tasks,
                                                   const GemmTile* __restrict__ tiles) {
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask t = tasks[tl.task];
  __shared__ double As[GK][ST + 1];
  __shared__ double Bs[GK][ST + 1];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < t.K; k0 += GK) {
    for (int idx = threadIdx.x; idx < ST * GK; idx += 64) {
      int m, k;
      if (t.transA) { k = idx % GK; m = idx / GK; }
      else { m = idx % ST; k = idx / ST; }
      const int gm = tl.m0 + m, gk = k0 + k;
      double v = 0.0;
      if (gm < t.M && gk < t.K)
        v = t.transA ? t.A[gk + (long long)gm * t.lda] : t.A[gm + (long long)gk * t.lda];
      As[k][m] = v;
    }
    for (int idx = threadIdx.x; idx < ST * GK; idx += 64) {
      int n, k;
      if (t.transB) { n = idx % ST; k = idx / ST; }
      else { k = idx % GK; n = idx / GK; }
      const int gn = tl.n0 + n, gk = k0 + k;
      double v = 0.0;
      if (gn < t.N && gk < t.K)
        v = t.transB ? t.B[gn + (long long)gk * t.ldb] : t.B[gk + (long long)gn * t.ldb];
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GK; k++) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[k][ty + 8 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[k][tx + 8 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int gm = tl.m0 + ty + 8 * i;
    if (gm >= t.M) continue;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int gn = tl.n0 + tx + 8 * j;
      if (gn >= t.N) continue;
      double* c = t.C + gm + (long long)gn * t.ldc;
      *c = (t.beta == 0.0) ? t.alpha * acc[i][j] : t.beta * (*c) + t.alpha * acc[i][j];
    }
  }
}

static inline bool small_task(const GemmTask& t) { return t.M <= ST && t.N <= ST; }

void gemm_tiles(const GemmTask& t, int ti, std::vector<GemmTile>& tiles) {
  if (t.M <= 0 || t.N <= 0) return;
  for (int n0 = 0; n0 < t.N; n0 += GT)
    for (int m0 = 0; m0 < t.M; m0 += GT) tiles.push_back({ti, m0, n0});
}

void launch_gemm(const GemmTask* d_tasks, const GemmTile* d_tiles, int ntiles, cudaStream_t s,
                 double flops) {
  if (ntiles <= 0) return;
  Prof p("k_gemm_fp64", flops, 0.0, s);
  k_gemm<<<ntiles, 256, 0, s>>>(d_tasks, d_tiles);
  CK_LAUNCH("k_gemm");
}

static void launch_gemm_small(const GemmTask* d_tasks, const GemmTile* d_tiles, int ntiles,
                              cudaStream_t s, double flops) {
  if (ntiles <= 0) return;
  Prof p("k_gemm_fp64_small", flops, 0.0, s);
  k_gemm_small<<<ntiles, 64, 0, s>>>(d_tasks, d_tiles);
  CK_LAUNCH("k_gemm_small");
}

void run_gemms(Arena& ar, const std::vector<GemmTask>& tasks, cudaStream_t s) {
  if (tasks.empty()) return;
  std::vector<GemmTask> kept, kept_s;
  std::vector<GemmTile> tiles, tiles_s;
  double flops = 0.0, flops_s = 0.0;
  for (const GemmTask& t : tasks) {
    if (t.M <= 0 || t.N <= 0) continue;
    validate(t);
    if (t.K > 0 && small_task(t)) {
      flops_s += 2.0 * t.M * (double)t.N * t.K;
      tiles_s.push_back({(int)kept_s.size(), 0, 0});
      kept_s.push_back(t);
      continue;
    }
    if (t.K > 0) flops += 2.0 * t.M * (double)t.N * t.K;
    if (t.K <= 0) {
      // C = beta C: express as a copy task with zero source
      CopyTask c{nullptr, t.C, nullptr, 1, t.ldc, t.M, t.N, 0, 2, 0.0, t.beta};
      CopyTask* d = upload(ar, std::vector<CopyTask>{c}, s);
      launch_copy(d, 1, s);
      continue;
    }
    gemm_tiles(t, (int)kept.size(), tiles);
    kept.push_back(t);
  }
  if (!tiles_s.empty())
    launch_gemm_small(upload(ar, kept_s, s), upload(ar, tiles_s, s), (int)tiles_s.size(), s,
                      flops_s);
  if (tiles.empty()) return;
  const GemmTask* dt = upload(ar, kept, s);
  const GemmTile* dl = upload(ar, tiles, s);
  launch_gemm(dt, dl, (int)tiles.size(), s, flops);
}

// ---------------------------------------------------------------------------
// block reductions
// ---------------------------------------------------------------------------
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum; `red` holds >= 33 doubles; all threads get the result
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double s = (lane < nw) ? red[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// ---------------------------------------------------------------------------
// LU with partial pivoting: panel factorisation, row swaps, triangular solve
// ---------------------------------------------------------------------------
__global__ void k_amax(const LuTask* __restrict__ tasks) {
  const LuTask t = tasks[blockIdx.x];
  __shared__ double red[64];
  double m = 0.0;
  const long long total = (long long)t.n * t.n;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int r = (int)(e % t.n), c = (int)(e / t.n);
    m = fmax(m, fabs(t.A[r + (long long)c * t.lda]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) mm = fmax(mm, red[w]);
    *t.amax = mm;
    *t.info = 0;
  }
}

// Unblocked LU of the panel rows [k0, n) x columns [k0, k0+jb) (getf2).
// Pivot rule: the first row of largest magnitude.
__global__ void __launch_bounds__(256) k_getf2_panel(const LuTask* __restrict__ tasks, int k0) {
  const LuTask t = tasks[blockIdx.x];
  if (t.n <= k0) return;
  const int jb = min(LU_NB, t.n - k0);
  __shared__ double sval[32];
  __shared__ int sidx[32];
  __shared__ int piv_s;
  double* A = t.A;
  const long long lda = t.lda;
  const double tol = 1e-14 * (*t.amax);
  for (int j = k0; j < k0 + jb; j++) {
    // pivot search
    double best = -1.0;
    int bi = t.n;
    for (int i = j + threadIdx.x; i < t.n; i += blockDim.x) {
      const double v = fabs(A[i + j * lda]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { sval[threadIdx.x >> 5] = best; sidx[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = -1.0;
      int ii = t.n;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++)
        if (sval[w] > b || (sval[w] == b && sidx[w] < ii)) { b = sval[w]; ii = sidx[w]; }
      if (ii >= t.n) ii = j;
      piv_s = ii;
      t.piv[j] = ii;
      if (!(b > tol) && *t.info == 0) *t.info = j + 1;
    }
    __syncthreads();
    const int p = piv_s;
    if (p != j) {
      for (int c = k0 + threadIdx.x; c < k0 + jb; c += blockDim.x) {
        const double tmp = A[j + c * lda];
        A[j + c * lda] = A[p + c * lda];
        A[p + c * lda] = tmp;
      }
    }
    __syncthreads();
    double d = A[j + j * lda];
    if (d == 0.0) d = 1e-300;  // keep the arithmetic finite; info already records it
    const double inv = 1.0 / d;
    for (int i = j + 1 + threadIdx.x; i < t.n; i += blockDim.x) A[i + j * lda] *= inv;
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < t.n; i += blockDim.x) {
      const double l = A[i + j * lda];
      for (int c = j + 1; c < k0 + jb; c++) A[i + c * lda] -= l * A[j + c * lda];
    }
    __syncthreads();
  }
}

// apply the panel's swaps to columns outside [k0, k0+jb)
__global__ void k_laswp_lu(const LuTask* __restrict__ tasks, int k0) {
  const LuTask t = tasks[blockIdx.x];
  if (t.n <= k0) return;
  const int jb = min(LU_NB, t.n - k0);
  for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < t.n; c += gridDim.y * blockDim.x) {
    if (c >= k0 && c < k0 + jb) continue;
    for (int j = k0; j < k0 + jb; j++) {
      const int p = t.piv[j];
      if (p != j) {
        const double tmp = t.A[j + (long long)c * t.lda];
        t.A[j + (long long)c * t.lda] = t.A[p + (long long)c * t.lda];
        t.A[p + (long long)c * t.lda] = tmp;
      }
    }
  }
}

// U12 = L11^-1 A12 (unit lower), one thread per column of A12
__global__ void k_trsm_lu(const LuTask* __restrict__ tasks, int k0) {
  const LuTask t = tasks[blockIdx.x];
  if (t.n <= k0 + LU_NB) return;
  const int jb = LU_NB;
  const long long lda = t.lda;
  for (int c = k0 + jb + blockIdx.y * blockDim.x + threadIdx.x; c < t.n;
       c += gridDim.y * blockDim.x) {
    double* b = t.A + k0 + c * lda;
    const double* L = t.A + k0 + k0 * lda;
    for (int i = 1; i < jb; i++) {
      double s = b[i];
      for (int q = 0; q < i; q++) s -= L[i + q * lda] * b[q];
      b[i] = s;
    }
  }
}

void run_getrf(Arena& ar, const std::vector<LuTask>& tasks, cudaStream_t s) {
  if (tasks.empty()) return;
  for (auto& t : tasks) {
    Ranges::check(t.A, mat_bytes(t.n, t.n, t.lda), "getrf A");
    Ranges::check(t.piv, sizeof(int) * t.n, "getrf piv");
    Ranges::check(t.info, sizeof(int), "getrf info");
    Ranges::check(t.amax, sizeof(double), "getrf amax");
  }
  const LuTask* d = upload(ar, tasks, s);
  const int nt = (int)tasks.size();
  int nmax = 0;
  for (auto& t : tasks) nmax = std::max(nmax, t.n);
  k_amax<<<nt, 256, 0, s>>>(d);
  CK_LAUNCH("k_amax");
  for (int k0 = 0; k0 < nmax; k0 += LU_NB) {
    double fl = 0.0;
    for (auto& t : tasks)
      if (t.n > k0) {
        const double m = t.n - k0, jb = std::min(LU_NB, t.n - k0);
        fl += m * jb * jb - jb * jb * jb / 3.0;
      }
    {
      Prof p("k_getf2_panel", fl, 0.0, s);
      k_getf2_panel<<<nt, 256, 0, s>>>(d, k0);
      CK_LAUNCH("k_getf2_panel");
    }
    if (nmax > LU_NB) {
      k_laswp_lu<<<dim3(nt, 8), 128, 0, s>>>(d, k0);
      CK_LAUNCH("k_laswp_lu");
    }
    if (k0 + LU_NB < nmax) {
      k_trsm_lu<<<dim3(nt, 16), 128, 0, s>>>(d, k0);
      CK_LAUNCH("k_trsm_lu");
      std::vector<GemmTask> g;
      for (auto& t : tasks) {
        const int rest = t.n - k0 - LU_NB;
        if (rest <= 0) continue;
        const long long lda = t.lda;
        g.push_back({t.A + (k0 + LU_NB) + k0 * lda, t.A + k0 + (k0 + LU_NB) * lda,
                     t.A + (k0 + LU_NB) + (k0 + LU_NB) * lda, t.lda, t.lda, t.lda, rest, rest,
                     LU_NB, 0, 0, -1.0, 1.0});
      }
      run_gemms(ar, g, s);
    }
  }
}

// ---------------------------------------------------------------------------
// solve with the LU factors: B <- A^-1 B
// ---------------------------------------------------------------------------
__global__ void k_laswp_rhs(const RsTask* __restrict__ tasks) {
  const RsTask t = tasks[blockIdx.x];
  for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < t.ncols; c += gridDim.y * blockDim.x) {
    double* b = t.B + (long long)c * t.ldb;
    for (int j = 0; j < t.n; j++) {
      const int p = t.piv[j];
      if (p != j) { const double tmp = b[j]; b[j] = b[p]; b[p] = tmp; }
    }
  }
}

// diagonal-block solve of rows [k0, k0+jb): lower unit (upper == 0) or upper
__global__ void k_trsm_rhs(const RsTask* __restrict__ tasks, int k0, int upper) {
  const RsTask t = tasks[blockIdx.x];
  if (k0 >= t.n) return;
  const int jb = min(LU_NB, t.n - k0);
  const long long lda = t.lda;
  const double* A = t.LU + k0 + k0 * lda;
  for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < t.ncols; c += gridDim.y * blockDim.x) {
    double* b = t.B + k0 + (long long)c * t.ldb;
    if (!upper) {
      for (int i = 1; i < jb; i++) {
        double s = b[i];
        for (int q = 0; q < i; q++) s -= A[i + q * lda] * b[q];
        b[i] = s;
      }
    } else {
      for (int i = jb - 1; i >= 0; i--) {
        double s = b[i];
        for (int q = i + 1; q < jb; q++) s -= A[i + q * lda] * b[q];
        double d = A[i + i * lda];
        if (d == 0.0) d = 1e-300;
        b[i] = s / d;
      }
    }
  }
}

GemmLaunch plan_gemms(Arena& ar, const std::vector<GemmTask>& tasks, cudaStream_t s) {
  GemmLaunch L;
  std::vector<GemmTask> kept;
  std::vector<GemmTile> tiles;
  for (const GemmTask& t : tasks) {
    if (t.M <= 0 || t.N <= 0 || t.K <= 0) continue;
    validate(t);
    L.flops += 2.0 * t.M * (double)t.N * t.K;
    gemm_tiles(t, (int)kept.size(), tiles);
    kept.push_back(t);
  }
  if (tiles.empty()) return L;
  L.tasks = upload(ar, kept, s);
  L.tiles = upload(ar, tiles, s);
  L.ntiles = (int)tiles.size();
  return L;
}

GetrsPlan plan_getrs(Arena& ar, const std::vector<RsTask>& tasks, cudaStream_t s) {
  GetrsPlan P;
  if (tasks.empty()) return P;
  for (auto& t : tasks) {
    Ranges::check(t.LU, mat_bytes(t.n, t.n, t.lda), "getrs LU");
    Ranges::check(t.piv, sizeof(int) * t.n, "getrs piv");
    Ranges::check(t.B, mat_bytes(t.n, t.ncols, t.ldb), "getrs B");
  }
  P.d = upload(ar, tasks, s);
  P.nt = (int)tasks.size();
  int cmax = 0;
  for (auto& t : tasks) { P.nmax = std::max(P.nmax, t.n); cmax = std::max(cmax, t.ncols); }
  if (P.nmax == 0 || cmax == 0) { P.nt = 0; return P; }
  P.gy = std::min(64, (cmax + 127) / 128);
  for (int k0 = 0; k0 < P.nmax; k0 += LU_NB) {
    std::vector<GemmTask> g;
    if (k0 + LU_NB < P.nmax)
      for (auto& t : tasks) {
        const int rest = t.n - k0 - LU_NB;
        if (rest <= 0 || t.ncols <= 0) continue;
        g.push_back({t.LU + (k0 + LU_NB) + (long long)k0 * t.lda, t.B + k0, t.B + (k0 + LU_NB),
                     t.lda, t.ldb, t.ldb, rest, t.ncols, LU_NB, 0, 0, -1.0, 1.0});
      }
    P.fwd.push_back(plan_gemms(ar, g, s));
  }
  const int last = ((P.nmax - 1) / LU_NB) * LU_NB;
  for (int k0 = last; k0 >= 0; k0 -= LU_NB) {
    std::vector<GemmTask> g;
    if (k0 > 0)
      for (auto& t : tasks) {
        if (k0 >= t.n || t.ncols <= 0) continue;
        const int jb = std::min(LU_NB, t.n - k0);
        g.push_back({t.LU + (long long)k0 * t.lda, t.B + k0, t.B, t.lda, t.ldb, t.ldb, k0, t.ncols,
                     jb, 0, 0, -1.0, 1.0});
      }
    P.bwd.push_back(plan_gemms(ar, g, s));
  }
  return P;
}

void exec_getrs(const GetrsPlan& P, cudaStream_t s) {
  if (P.nt == 0) return;
  k_laswp_rhs<<<dim3(P.nt, P.gy), 128, 0, s>>>(P.d);
  CK_LAUNCH("k_laswp_rhs");
  int step = 0;
  for (int k0 = 0; k0 < P.nmax; k0 += LU_NB, step++) {  // forward: unit lower
    k_trsm_rhs<<<dim3(P.nt, P.gy), 128, 0, s>>>(P.d, k0, 0);
    CK_LAUNCH("k_trsm_rhs");
    const GemmLaunch& g = P.fwd[step];
    launch_gemm(g.tasks, g.tiles, g.ntiles, s, g.flops);
  }
  const int last = ((P.nmax - 1) / LU_NB) * LU_NB;
  step = 0;
  for (int k0 = last; k0 >= 0; k0 -= LU_NB, step++) {  // backward: upper
    k_trsm_rhs<<<dim3(P.nt, P.gy), 128, 0, s>>>(P.d, k0, 1);
    CK_LAUNCH("k_trsm_rhs");
    const GemmLaunch& g = P.bwd[step];
    launch_gemm(g.tasks, g.tiles, g.ntiles, s, g.flops);
  }
}

void run_getrs(Arena& ar, const std::vector<RsTask>& tasks, cudaStream_t s) {
  exec_getrs(plan_getrs(ar, tasks, s), s);
}

// ---------------------------------------------------------------------------
// Left SVD: streaming LQ (M = L Q^T) then one-sided Jacobi on the columns of
// L (L J = W Sigma).  The LQ keeps L (a x a, lower) and a chunk C of CW
// columns of M side by side, [L | C], and annihilates C row by row with
// Householder reflectors; after the last chunk L carries the left singular
// structure of M.  Both phases live in shared memory when a <= SVD_SMEM_A,
// otherwise in the task's global scratch.
// ---------------------------------------------------------------------------
constexpr int SVD_SMEM_A = 144;
constexpr int SVD_CW = 16;

struct SvdView {
  double* L;    // a x a, ld = lda
  double* C;    // a x CW, ld = ldc
  int lda, ldc;
};

// Annihilate chunk columns [0, cw) of C against L (rows 0..a-1).
__device__ void lq_chunk(SvdView v, int a, int cw, double* red, double* vsh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < a; k++) {
    // reflector from (L[k,k], C[k, 0..cw))
    double sq = 0.0;
    for (int c = threadIdx.x; c < cw; c += blockDim.x) {
      const double x = v.C[k + c * v.ldc];
      sq += x * x;
    }
    sq = block_sum(sq, red);
    const double x0 = v.L[k + k * v.lda];
    if (sq == 0.0) continue;                    // nothing to annihilate (block-uniform)
    const double nrm = sqrt(x0 * x0 + sq);
    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
    const double v0 = x0 - alpha;               // v = [v0, C[k, :]], H = I - tau v v^T
    const double tau = -v0 / alpha;             // = (alpha - x0) / alpha
    const double scale = 1.0 / v0;
    // normalised reflector: u = [1, C[k,:]/v0], H = I - tau u u^T
    for (int c = threadIdx.x; c < cw; c += blockDim.x) vsh[c] = v.C[k + c * v.ldc] * scale;
    __syncthreads();
    for (int i = k + 1 + wid; i < a; i += nw) {
      double d = 0.0;
      for (int c = lane; c < cw; c += 32) d += v.C[i + c * v.ldc] * vsh[c];
      d = warp_sum(d) + v.L[i + k * v.lda];
      const double f = tau * d;
      for (int c = lane; c < cw; c += 32) v.C[i + c * v.ldc] -= f * vsh[c];
      if (lane == 0) v.L[i + k * v.lda] -= f;
    }
    __syncthreads();
    if (threadIdx.x == 0) v.L[k + k * v.lda] = alpha;
    for (int c = threadIdx.x; c < cw; c += blockDim.x) v.C[k + c * v.ldc] = 0.0;
    __syncthreads();
  }
}

__device__ void jacobi_columns(double* L, int lda, int a, double* red) {
  // round-robin pairing over n = a rounded up to even; a warp per pair
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = (a + 1) & ~1;
  __shared__ int rotated;
  for (int sweep = 0; sweep < 40; sweep++) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < n - 1; round++) {
      for (int pr = wid; pr < n / 2; pr += nw) {
        // round-robin tournament: seat 0 fixed, seats 1..n-1 rotate by `round`;
        // seat m plays seat n-1-m, so every pair meets once per sweep
        const int ma = pr, mb = n - 1 - pr;
        const int pa = (ma == 0) ? 0 : ((ma - 1 + round) % (n - 1)) + 1;
        const int pb = (mb == 0) ? 0 : ((mb - 1 + round) % (n - 1)) + 1;
        const int p = min(pa, pb), q = max(pa, pb);
        if (q >= a || p == q) continue;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = lane; r < a; r += 32) {
          const double x = L[r + p * lda], y = L[r + q * lda];
          al += x * x; be += y * y; ga += x * y;
        }
        al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
        if (fabs(ga) > 1e-15 * sqrt(al * be) && ga != 0.0) {
          const double zeta = (be - al) / (2.0 * ga);
          const double tt = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
          for (int r = lane; r < a; r += 32) {
            const double x = L[r + p * lda], y = L[r + q * lda];
            L[r + p * lda] = cs * x - sn * y;
            L[r + q * lda] = sn * x + cs * y;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (!rotated) break;
    __syncthreads();
  }
}

// cw: columns streamed per chunk (shared-memory mode); the reflector vector
// lives behind the chunk in dynamic shared memory.
__global__ void __launch_bounds__(1024) k_svd_left(const SvdTask* __restrict__ tasks, int use_smem,
                                                   int cw_max) {
  const SvdTask t = tasks[blockIdx.x];
  const int a = t.a;
  if (a <= 0) return;
  if ((a <= SVD_SMEM_A) != (use_smem != 0)) return;
  extern __shared__ double sm[];
  __shared__ double red[40];
  __shared__ double vsh_g[SVD_CW];
  SvdView v;
  double* vsh;
  int cwm;
  if (use_smem) {
    v.L = sm;
    v.lda = a + 1;                 // odd stride: no bank conflicts on row access
    v.C = sm + (size_t)(a + 1) * a;
    v.ldc = a + 1;
    vsh = v.C + (size_t)(a + 1) * cw_max;
    cwm = cw_max;
  } else {
    v.L = t.work;
    v.lda = a;
    v.C = t.work + (size_t)a * a;
    v.ldc = a;
    vsh = vsh_g;
    cwm = SVD_CW;
  }
  // L starts at zero; every column of M is streamed through the chunk C and
  // annihilated against L (the reflector treats L[k,k] as its first entry).
  for (int e = threadIdx.x; e < a * a; e += blockDim.x) v.L[(e % a) + (e / a) * v.lda] = 0.0;
  __syncthreads();
  for (int c0 = 0; c0 < t.w; c0 += cwm) {
    const int cw = min(cwm, t.w - c0);
    for (int e = threadIdx.x; e < a * cw; e += blockDim.x) {
      const int r = e % a, c = e / a;
      v.C[r + c * v.ldc] = t.M[r + (long long)(c0 + c) * t.ldm];
    }
    __syncthreads();
    lq_chunk(v, a, cw, red, vsh);
  }
  jacobi_columns(v.L, v.lda, a, red);
  // sigma_j = |L_j|; order by decreasing sigma (ties: lower column first).
  // The chunk area (>= a doubles) is free now and holds the column norms.
  double* sg = v.C;
  for (int j = threadIdx.x; j < a; j += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < a; r++) { const double x = v.L[r + j * v.lda]; s += x * x; }
    sg[j] = sqrt(s);
  }
  __syncthreads();
  double smax = 0.0;
  for (int j = 0; j < a; j++) smax = fmax(smax, sg[j]);
  for (int j = threadIdx.x; j < a; j += blockDim.x) {
    int pos = 0;
    for (int k = 0; k < a; k++) pos += (sg[k] > sg[j]) || (sg[k] == sg[j] && k < j);
    t.sigma[pos] = sg[j];
    const double inv = sg[j] > 0.0 ? 1.0 / sg[j] : 0.0;
    for (int r = 0; r < a; r++) t.W[r + (long long)pos * a] = v.L[r + j * v.lda] * inv;
  }
  __syncthreads();
  // complete the basis where sigma is negligible: Gram-Schmidt (twice) against
  // the preceding columns, starting from the column or from unit vectors
  const double small = smax * 1e-13 * a + 1e-300;
  for (int j = 0; j < a; j++) {
    if (t.sigma[j] > small) continue;
    for (int attempt = 0; attempt <= a; attempt++) {
      double* wj = t.W + (long long)j * a;
      if (attempt > 0)
        for (int r = threadIdx.x; r < a; r += blockDim.x) wj[r] = (r == attempt - 1) ? 1.0 : 0.0;
      __syncthreads();
      for (int pass = 0; pass < 2; pass++)
        for (int k = 0; k < j; k++) {
          const double* wk = t.W + (long long)k * a;
          double d = 0.0;
          for (int r = threadIdx.x; r < a; r += blockDim.x) d += wk[r] * wj[r];
          d = block_sum(d, red);
          for (int r = threadIdx.x; r < a; r += blockDim.x) wj[r] -= d * wk[r];
          __syncthreads();
        }
      double nn = 0.0;
      for (int r = threadIdx.x; r < a; r += blockDim.x) nn += wj[r] * wj[r];
      nn = block_sum(nn, red);
      if (nn > 1e-2 || (attempt > 0 && nn > 1e-6)) {
        const double inv = 1.0 / sqrt(nn);
        for (int r = threadIdx.x; r < a; r += blockDim.x) wj[r] *= inv;
        __syncthreads();
        break;
      }
      __syncthreads();
    }
  }
}

// IFMM_TRACE=2: one line per SVD launch on stderr (tasks, shapes, seconds);
// synchronises the stream around each launch.
static bool svd_tracing() {
  static const bool v = [] {
    const char* e = std::getenv("IFMM_TRACE");
    return e && e[0] == '2';
  }();
  return v;
}

void run_svd_left(Arena& ar, const std::vector<SvdTask>& tasks, cudaStream_t s) {
  if (tasks.empty()) return;
  std::chrono::steady_clock::time_point t0;
  if (svd_tracing()) {
    CK(cudaStreamSynchronize(s));
    t0 = std::chrono::steady_clock::now();
  }
  for (auto& t : tasks) {
    if (t.a <= 0) continue;
    Ranges::check(t.M, mat_bytes(t.a, t.w, t.ldm), "svd M");
    Ranges::check(t.W, mat_bytes(t.a, t.a, t.a), "svd W");
    Ranges::check(t.sigma, sizeof(double) * t.a, "svd sigma");
    if (t.a > SVD_SMEM_A)
      Ranges::check(t.work, sizeof(double) * ((size_t)t.a * t.a + (size_t)t.a * SVD_CW), "svd work");
  }
  const SvdTask* d = upload(ar, tasks, s);
  int amax_s = 0;
  bool big = false;
  for (auto& t : tasks) {
    if (t.a <= SVD_SMEM_A) amax_s = std::max(amax_s, t.a);
    else big = true;
  }
  double fl = 0.0;
  for (auto& t : tasks) fl += 2.0 * t.a * (double)t.a * t.w;
  Prof p("k_svd_left", fl, 0.0, s);
  if (amax_s > 0) {
    // widest chunk that fits next to L: (a+1)(a+cw) + cw doubles <= 200 KiB
    const long long budget = (200 * 1024) / 8;
    long long cw = (budget - (long long)(amax_s + 1) * amax_s) / (amax_s + 2);
    int wmax = 0;
    for (auto& t : tasks) if (t.a <= SVD_SMEM_A) wmax = std::max(wmax, t.w);
    cw = std::min<long long>(cw, 2048);
    cw = std::min<long long>(cw, std::max(wmax, 1));
    cw = std::max<long long>(cw, SVD_CW);
    const size_t smem = sizeof(double) * ((size_t)(amax_s + 1) * (amax_s + cw) + cw);
    static bool attr = false;
    if (!attr) {
      CK(cudaFuncSetAttribute(k_svd_left, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              200 * 1024));
      attr = true;
    }
    const int threads = amax_s > 96 ? 512 : 256;
    k_svd_left<<<(int)tasks.size(), threads, smem, s>>>(d, 1, (int)cw);
    CK_LAUNCH("k_svd_left(smem)");
  }
  if (big) {
    k_svd_left<<<(int)tasks.size(), 512, 0, s>>>(d, 0, SVD_CW);
    CK_LAUNCH("k_svd_left(global)");
  }
  if (svd_tracing()) {
    CK(cudaStreamSynchronize(s));
    int amax = 0, wmax = 0;
    double wsum = 0.0;
    for (auto& t : tasks) { amax = std::max(amax, t.a); wmax = std::max(wmax, t.w); wsum += t.w; }
    std::fprintf(stderr, "[svd] tasks %zu, max a %d, max w %d, avg w %.0f, %.4f s\n", tasks.size(),
                 amax, wmax, wsum / tasks.size(),
                 std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
  }
}

// ---------------------------------------------------------------------------
// Randomised left SVD (Sec. 2.4: the fill-in is compressed with the randomised
// SVD of Halko et al.; reading R3b): for a block too tall for the exact
// shared-memory SVD, a test matrix Omega (w x k, uniform in [-1, 1) from a
// counter-based SplitMix64 stream), one power iteration with
// re-orthonormalisation, B = Q^T M and the exact SVD of the k-row matrix B.
// Returns the top k left singular vectors (a x k, ld a) and values.
// ---------------------------------------------------------------------------
__device__ __host__ inline unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// O[e] = 2 u - 1, u = (splitmix64(seed + e) >> 11) 2^-53, e = i + c * rows
__global__ void k_fill_uniform(double* __restrict__ O, long long n, unsigned long long seed) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const unsigned long long x = splitmix64(seed + (unsigned long long)e);
    O[e] = 2.0 * ((double)(x >> 11) * 0x1.0p-53) - 1.0;
  }
}


// inv[c] = 1 / s[c] where s[c] > 1e-10 s[0], else 0: drops numerically null
// directions (above the SVD's basis-completion threshold 1e-13 a s[0], a <= 144)
__global__ void k_inv_sigma(const InvSigma* __restrict__ t, int n) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const InvSigma T = t[i];
  for (int c = threadIdx.x; c < T.k; c += blockDim.x)
    T.inv[c] = (T.s[c] > 1e-10 * T.s[0] && T.s[c] > 0.0) ? 1.0 / T.s[c] : 0.0;
}

void run_inv_sigma(Arena& ar, const std::vector<InvSigma>& v, cudaStream_t s) {
  if (v.empty()) return;
  const InvSigma* d = upload(ar, v, s);
  k_inv_sigma<<<(int)v.size(), 64, 0, s>>>(d, (int)v.size());
  CK_LAUNCH("k_inv_sigma");
}

// Q = orth(X) for X (n x k, ld n): SVD of X^T, Q = X W diag(1/sigma)
static void batched_orth_once(Arena& ar, const std::vector<const double*>& X, std::vector<double*>& Q,
                         const std::vector<int>& n, int k, cudaStream_t s) {
  const int nt = (int)X.size();
  std::vector<CopyTask> tr;
  std::vector<SvdTask> sv;
  std::vector<InvSigma> iv;
  std::vector<double*> XT(nt), W(nt), sg(nt), inv(nt), Ws(nt);
  for (int t = 0; t < nt; t++) {
    XT[t] = ar.alloc<double>((size_t)k * n[t]);
    W[t] = ar.alloc<double>((size_t)k * k);
    Ws[t] = ar.alloc<double>((size_t)k * k);
    sg[t] = ar.alloc<double>(k);
    inv[t] = ar.alloc<double>(k);
    tr.push_back({X[t], XT[t], nullptr, n[t], k, k, n[t], 1, 0, 1.0, 0.0});
    sv.push_back({XT[t], k, k, n[t], W[t], sg[t], nullptr});
    iv.push_back({sg[t], inv[t], k});
  }
  std::vector<CopyTask> keep;
  for (auto& c : tr) { validate(c); keep.push_back(c); }
  launch_copy(upload(ar, keep, s), (int)keep.size(), s);
  run_svd_left(ar, sv, s);
  run_inv_sigma(ar, iv, s);
  keep.clear();
  for (int t = 0; t < nt; t++) {
    CopyTask c{W[t], Ws[t], inv[t], k, k, k, k, 0, 0, 1.0, 0.0};
    validate(c);
    keep.push_back(c);
  }
  launch_copy(upload(ar, keep, s), (int)keep.size(), s);
  std::vector<GemmTask> g;
  for (int t = 0; t < nt; t++) g.push_back({X[t], Ws[t], Q[t], n[t], k, n[t], n[t], k, k, 0, 0, 1.0, 0.0});
  run_gemms(ar, g, s);
}

unsigned long long rsvd_seed(int level, int box, int side) {
  return splitmix64(((unsigned long long)level << 40) ^ ((unsigned long long)box << 2) ^
                    (unsigned long long)side);
}

// Orthonormalise twice: the second pass removes the loss of orthogonality the
// first one suffers in directions with small singular values.
static void batched_orth(Arena& ar, const std::vector<const double*>& X, std::vector<double*>& Q,
                         const std::vector<int>& n, int k, cudaStream_t s) {
  std::vector<double*> Q1(X.size());
  for (size_t t = 0; t < X.size(); t++) Q1[t] = ar.alloc<double>((size_t)n[t] * k);
  batched_orth_once(ar, X, Q1, n, k, s);
  std::vector<const double*> cQ1(Q1.begin(), Q1.end());
  batched_orth_once(ar, cQ1, Q, n, k, s);
}

void run_rsvd_left(Arena& ar, const std::vector<RsvdTask>& tasks, cudaStream_t s) {
  if (tasks.empty()) return;
  const int nt = (int)tasks.size();
  // tasks are grouped by k (all tasks of one call share k)
  const int k = tasks[0].k;
  for (auto& t : tasks)
    if (t.k != k || t.k > SVD_SMEM_A || t.k > t.a)
      throw Error(IFMM_ERR_CUDA, "internal: randomised SVD tasks need a common k <= 144 <= a");
  std::vector<double*> Om(nt), Y(nt), Q(nt), Z(nt), Qz(nt), B(nt), WB(nt);
  std::vector<GemmTask> g;
  for (int t = 0; t < nt; t++) {
    const RsvdTask& T = tasks[t];
    Om[t] = ar.alloc<double>((size_t)T.w * k);
    Y[t] = ar.alloc<double>((size_t)T.a * k);
    Q[t] = ar.alloc<double>((size_t)T.a * k);
    Z[t] = ar.alloc<double>((size_t)T.w * k);
    Qz[t] = ar.alloc<double>((size_t)T.w * k);
    B[t] = ar.alloc<double>((size_t)k * T.w);
    WB[t] = ar.alloc<double>((size_t)k * k);
    const long long n = (long long)T.w * k;
    k_fill_uniform<<<(int)std::min<long long>(1024, (n + 255) / 256), 256, 0, s>>>(Om[t], n, T.seed);
    CK_LAUNCH("k_fill_uniform");
    g.push_back({T.M, Om[t], Y[t], T.ldm, T.w, T.a, T.a, k, T.w, 0, 0, 1.0, 0.0});  // Y = M Om
  }
  run_gemms(ar, g, s);
  std::vector<int> na(nt), nw(nt);
  std::vector<const double*> cY(Y.begin(), Y.end());
  for (int t = 0; t < nt; t++) { na[t] = tasks[t].a; nw[t] = tasks[t].w; }
  batched_orth(ar, cY, Q, na, k, s);
  g.clear();
  for (int t = 0; t < nt; t++)  // Z = M^T Q
    g.push_back({tasks[t].M, Q[t], Z[t], tasks[t].ldm, tasks[t].a, tasks[t].w, tasks[t].w, k,
                 tasks[t].a, 1, 0, 1.0, 0.0});
  run_gemms(ar, g, s);
  std::vector<const double*> cZ(Z.begin(), Z.end());
  batched_orth(ar, cZ, Qz, nw, k, s);
  g.clear();
  for (int t = 0; t < nt; t++)  // Y = M Qz
    g.push_back({tasks[t].M, Qz[t], Y[t], tasks[t].ldm, tasks[t].w, tasks[t].a, tasks[t].a, k,
                 tasks[t].w, 0, 0, 1.0, 0.0});
  run_gemms(ar, g, s);
  batched_orth(ar, cY, Q, na, k, s);
  g.clear();
  for (int t = 0; t < nt; t++)  // B = Q^T M
    g.push_back({Q[t], tasks[t].M, B[t], tasks[t].a, tasks[t].ldm, k, k, tasks[t].w, tasks[t].a,
                 1, 0, 1.0, 0.0});
  run_gemms(ar, g, s);
  std::vector<SvdTask> sv;
  for (int t = 0; t < nt; t++) sv.push_back({B[t], k, k, tasks[t].w, WB[t], tasks[t].sigma, nullptr});
  run_svd_left(ar, sv, s);
  g.clear();
  for (int t = 0; t < nt; t++)  // W = Q W_B
    g.push_back({Q[t], WB[t], tasks[t].W, tasks[t].a, k, tasks[t].a, tasks[t].a, k, k, 0, 0, 1.0, 0.0});
  run_gemms(ar, g, s);
}

// ---------------------------------------------------------------------------
// rank decision (Eq. methods_SVD_rank_spectralnorm, readings R1, R5)
// ---------------------------------------------------------------------------
__global__ void k_rank(const RankTask* __restrict__ tasks, int n, double tau) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RankTask t = tasks[i];
  int r;
  if (tau <= 0.0) {
    r = t.full;
  } else {
    int ru = 0, rv = 0;
    for (int k = 0; k < t.full; k++) ru += t.sigU[k] > tau;
    for (int k = 0; k < t.full; k++) rv += (t.sigV ? t.sigV[k] : 0.0) > tau;
    r = max(ru, rv);
  }
  if (r > t.full) r = t.full;
  if (r > t.cap) { r = t.cap; if (t.capped) atomicAdd(t.capped, 1); }
  *t.out = r;
}

void launch_rank(const RankTask* d, int n, double tau, cudaStream_t s) {
  if (n <= 0) return;
  k_rank<<<(n + 127) / 128, 128, 0, s>>>(d, n, tau);
  CK_LAUNCH("k_rank");
}

}  // namespace ifmm
