// kernels_linalg.cu -- batched FP64 dense kernels of the IFMM factorisation.
//
// The elimination of a box (Sec. 2.2, Algorithm 2) is a block Gaussian
// elimination: LU of the pivot block E(P,P) with partial pivoting, the solve
// G = E(P,P)^-1 E(P,C), the Schur product E(R,P) G, and truncated SVDs of the
// fill-in and of the weighted bases (Eqs. P2P_kj, U_j_recomp, V_j_recomp).
// Each kernel here runs one such operation for every box of a colour in one
// launch (boxes of a colour are independent).
#include <algorithm>
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
  Prof p("k_copy", 0.0, 0.0, s);
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

// Row interchanges of LAPACK getrf (swap j <-> piv[j], j = 0..n-1 in order)
// as a gather index: (P b)[i] = b[perm[i]].  One thread per task.
__global__ void k_piv_to_perm(const RsTask* __restrict__ tasks, int* const* perm, int nt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const RsTask T = tasks[t];
  int* p = perm[t];
  for (int i = 0; i < T.n; i++) p[i] = i;
  for (int j = 0; j < T.n; j++) {
    const int q = T.piv[j];
    if (q != j) { const int tmp = p[j]; p[j] = p[q]; p[q] = tmp; }
  }
}

// Inverse of one jb x jb diagonal block (jb <= 64) of L (unit lower, z = 0)
// or U (upper, z = 1): thread j forms column j of the inverse by
// substitution against e_j; the block is stored zero-padded, ld 64.
__global__ void __launch_bounds__(64) k_getrs_dinv(const RsPanel* __restrict__ tasks) {
  const RsPanel t = tasks[blockIdx.y];
  const int b = blockIdx.x, upper = blockIdx.z;
  if (b >= t.nblk) return;
  const int k0 = b * GETRS_PANEL, jb = min(GETRS_PANEL, t.n - k0);
  const long long lda = t.lda;
  const double* T = t.LU + k0 + k0 * lda;
  __shared__ double X[GETRS_PANEL][GETRS_PANEL + 1];  // X[i][j]: row i of column j
  const int j = threadIdx.x;
  for (int i = 0; i < GETRS_PANEL; i++) X[i][j] = 0.0;
  if (j < jb) {
    if (!upper) {
      X[j][j] = 1.0;
      for (int i = j + 1; i < jb; i++) {
        double s = 0.0;
        for (int q = j; q < i; q++) s = fma(T[i + q * lda], X[q][j], s);
        X[i][j] = -s;
      }
    } else {
      for (int i = j; i >= 0; i--) {
        double s = (i == j) ? 1.0 : 0.0;
        for (int q = i + 1; q <= j; q++) s = fma(-T[i + q * lda], X[q][j], s);
        double d = T[i + i * lda];
        if (d == 0.0) d = 1e-300;
        X[i][j] = s / d;
      }
    }
  }
  __syncthreads();
  double* D = t.dinv + (size_t)(upper * t.nblk + b) * GETRS_PANEL * GETRS_PANEL;
  for (int i = 0; i < GETRS_PANEL; i++) D[i + j * GETRS_PANEL] = X[i][j];
}

// Panel solve.  w1 = P B, then for every panel of GETRS_PANEL columns a
// launch over (row chunks, tasks): each CTA solves the panel's diagonal block
// (one warp, rows in registers, values by shuffle) from `in` and updates its
// chunk of the remaining rows of `in` in place; CTA 0 of a task writes the
// diagonal block's solution to `out`.  Forward: in = w1, out = w2 (unit lower
// L); backward: in = w2, out = B (upper U).  Within a launch the diagonal rows
// of `in` are only read and every other row has one writer.
__global__ void k_getrs_gather(const RsPanel* __restrict__ tasks) {
  const RsPanel t = tasks[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.n) return;
  const int src = t.perm[i];
  for (int c = 0; c < t.ncols; c++) t.w1[i + (long long)c * t.n] = t.B[src + (long long)c * t.ldb];
}

__device__ inline const double* LU_row(const double* LU, int i, int k0, long long lda) {
  return LU + i + k0 * lda;
}

__global__ void __launch_bounds__(GETRS_PROWS) k_getrs_panel(const RsPanel* __restrict__ tasks,
                                                            int k0, int upper) {
  const RsPanel t = tasks[blockIdx.y];
  const int n = t.n;
  if (k0 >= n) return;
  const int jb = min(GETRS_PANEL, n - k0);
  const int r_lo = upper ? 0 : k0 + jb, r_hi = upper ? k0 : n;  // rows to update
  if (blockIdx.x > 0 && r_lo + blockIdx.x * GETRS_PROWS >= r_hi) return;
  const int i = r_lo + blockIdx.x * GETRS_PROWS + threadIdx.x;
  const long long lda = t.lda;
  const double* D = t.dinv + (size_t)(upper * t.nblk + k0 / GETRS_PANEL) * GETRS_PANEL * GETRS_PANEL;
  __shared__ double xin[GETRS_PANEL];
  __shared__ double half[2][GETRS_PANEL];
  __shared__ double xd[GETRS_PANEL];
  const int r = threadIdx.x & (GETRS_PANEL - 1), h = threadIdx.x / GETRS_PANEL;
  for (int c = 0; c < t.ncols; c++) {
    double* in = (upper ? t.w2 : t.w1) + (long long)c * n;
    double* out = upper ? t.B + (long long)c * t.ldb : t.w2 + (long long)c * n;
    if (threadIdx.x < GETRS_PANEL) xin[threadIdx.x] = threadIdx.x < jb ? in[k0 + threadIdx.x] : 0.0;
    __syncthreads();
    {  // xd = D xin: thread (r, h) sums 32 columns in four chains
      const double* d = D + r + (size_t)(h * 32) * GETRS_PANEL;
      const double* x = xin + h * 32;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
      for (int q = 0; q < 32; q += 4) {
        s0 = fma(d[(q + 0) * GETRS_PANEL], x[q + 0], s0);
        s1 = fma(d[(q + 1) * GETRS_PANEL], x[q + 1], s1);
        s2 = fma(d[(q + 2) * GETRS_PANEL], x[q + 2], s2);
        s3 = fma(d[(q + 3) * GETRS_PANEL], x[q + 3], s3);
      }
      half[h][r] = (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
    if (threadIdx.x < GETRS_PANEL) xd[threadIdx.x] = half[0][threadIdx.x] + half[1][threadIdx.x];
    __syncthreads();
    if (blockIdx.x == 0)
      for (int q = threadIdx.x; q < jb; q += blockDim.x) out[k0 + q] = xd[q];
    if (i < r_hi) {
      const double* a = LU_row(t.LU, i, k0, lda);
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      if (jb == GETRS_PANEL) {
#pragma unroll
        for (int q = 0; q < GETRS_PANEL; q += 4) {
          s0 = fma(a[(q + 0) * lda], xd[q + 0], s0);
          s1 = fma(a[(q + 1) * lda], xd[q + 1], s1);
          s2 = fma(a[(q + 2) * lda], xd[q + 2], s2);
          s3 = fma(a[(q + 3) * lda], xd[q + 3], s3);
        }
      } else {
        for (int q = 0; q < jb; q++) s0 = fma(a[q * lda], xd[q], s0);
      }
      in[i] -= (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
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
  if (cmax <= GETRS_SMALL_COLS) {
    std::vector<int*> pm(tasks.size());
    for (size_t i = 0; i < tasks.size(); i++) pm[i] = ar.alloc<int>(std::max(tasks[i].n, 1));
    const int* const* dpm = upload(ar, pm, s);
    k_piv_to_perm<<<(P.nt + 127) / 128, 128, 0, s>>>(P.d, const_cast<int* const*>(dpm), P.nt);
    CK_LAUNCH("k_piv_to_perm");
    P.panel = true;
    std::vector<RsPanel> pt;
    for (size_t i = 0; i < tasks.size(); i++) {
      const RsTask& t = tasks[i];
      const size_t len = (size_t)std::max(t.n, 1) * std::max(t.ncols, 1);
      const int nblk = (t.n + GETRS_PANEL - 1) / GETRS_PANEL;
      P.nblk_max = std::max(P.nblk_max, nblk);
      pt.push_back({t.LU, t.lda, t.n, pm[i], t.B, t.ldb, t.ncols, ar.alloc<double>(len),
                    ar.alloc<double>(len),
                    ar.alloc<double>((size_t)2 * std::max(nblk, 1) * GETRS_PANEL * GETRS_PANEL),
                    nblk});
    }
    P.pd = upload(ar, pt, s);
    k_getrs_dinv<<<dim3(P.nblk_max, P.nt, 2), GETRS_PANEL, 0, s>>>(P.pd);
    CK_LAUNCH("k_getrs_dinv");
    return P;
  }
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
  if (P.panel) {
    Prof pr("phase:getrs_panel", 2.0 * P.nmax * (double)P.nmax * P.nt, 8.0 * P.nmax * (double)P.nmax * P.nt, s);
    k_getrs_gather<<<dim3((P.nmax + 255) / 256, P.nt), 256, 0, s>>>(P.pd);
    CK_LAUNCH("k_getrs_gather");
    const dim3 grid((P.nmax + GETRS_PROWS - 1) / GETRS_PROWS, P.nt);
    for (int k0 = 0; k0 < P.nmax; k0 += GETRS_PANEL) {
      k_getrs_panel<<<grid, GETRS_PROWS, 0, s>>>(P.pd, k0, 0);
      CK_LAUNCH("k_getrs_panel");
    }
    for (int k0 = ((P.nmax - 1) / GETRS_PANEL) * GETRS_PANEL; k0 >= 0; k0 -= GETRS_PANEL) {
      k_getrs_panel<<<grid, GETRS_PROWS, 0, s>>>(P.pd, k0, 1);
      CK_LAUNCH("k_getrs_panel");
    }
    return;
  }
  Prof pr("phase:getrs_blocked", 2.0 * P.nmax * (double)P.nmax * P.nt, 8.0 * P.nmax * (double)P.nmax * P.nt, s);
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
// L (L J = W Sigma).  The LQ keeps L (a x a, lower) and a chunk C of columns
// of M side by side, [L | C], and annihilates C row by row with Householder
// reflectors; after the last chunk L carries the left singular structure of
// M.  Both phases live in shared memory when a <= SVD_SMEM_A, otherwise in
// global scratch.
//
// FP64 throughput is the limit on this part (a few FP64 lanes per SM per
// clock), so the kernels spend FP64 instructions only on the arithmetic:
// G lanes share one row (LQ) or one column pair (Jacobi) so that a warp
// instruction carries 32 / G rows or pairs, reductions take log2(G) adds, the
// reflector and rotation scalars are formed once per row or pair, rotations
// are scaled (two FMAs per element, column scales kept aside) and the column
// norms are carried through each rotation instead of being recomputed.
// ---------------------------------------------------------------------------
constexpr int SVD_CW = 16;  // chunk width of the global-memory path

struct SvdView {
  double* L;    // a x a, ld = lda
  double* C;    // a x cw, ld = ldc
  int lda, ldc;
};

// H = I - beta v v^T with v = [v0, C[k, :]] (v0 on L[k, k]); the row
// [L[k, k], C[k, :]] maps to [alpha, 0]; beta = 2 / (v^T v) = -1 / (alpha v0).
struct Refl { double alpha, v0, beta; };

template <int G>
__device__ inline double group_sum(double v) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline Refl make_refl(double x0, double sq) {
  Refl r;
  // nothing to annihilate (or entries so small that beta = -1 / (alpha v0)
  // would overflow: below 1e-140 in norm they cannot matter): identity
  if (!(sq > 1e-280)) {
    r.alpha = x0; r.v0 = 0.0; r.beta = 0.0;
    return r;
  }
  const double nrm = sqrt(fma(x0, x0, sq));
  r.alpha = (x0 >= 0.0) ? -nrm : nrm;
  r.v0 = x0 - r.alpha;  // same sign as x0: no cancellation
  r.beta = -1.0 / (r.alpha * r.v0);
  return r;
}

// Annihilate the chunk C (a x cw) against L, rows 0..a-1 in order.  The group
// that updates row k + 1 during step k also forms that row's reflector, so a
// step costs one barrier; refl[2] alternates between steps.
template <int G>
__device__ void lq_chunk(SvdView v, int a, int cw, Refl* refl) {
  constexpr int RPW = 32 / G;  // rows per warp instruction
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int grp = lane / G, q = lane % G;
  if (wid == 0) {
    double sq = 0.0;
    for (int c = lane; c < cw; c += 32) {
      const double x = v.C[(size_t)c * v.ldc];
      sq = fma(x, x, sq);
    }
    sq = warp_sum(sq);
    if (lane == 0) refl[0] = make_refl(v.L[0], sq);
  }
  __syncthreads();
  for (int k = 0; k < a; k++) {
    const Refl R = refl[k & 1];
    const double* ck = v.C + k;
    for (int base = k + 1 + wid * RPW; base < a; base += nw * RPW) {  // warp-uniform
      const int i = base + grp;
      const bool act = i < a;
      const bool next = (base == k + 1);  // this pass holds row k + 1 (group 0)
      double* ci = v.C + i;
      double* li = v.L + i + (size_t)k * v.lda;
      double d = 0.0;
      if (act) {
        for (int c = q; c < cw; c += G) d = fma(ci[(size_t)c * v.ldc], ck[(size_t)c * v.ldc], d);
        if (q == 0) d = fma(*li, R.v0, d);
      }
      d = group_sum<G>(d);
      double sq = 0.0;
      if (act) {
        const double f = R.beta * d;
        for (int c = q; c < cw; c += G) {
          const double x = fma(-f, ck[(size_t)c * v.ldc], ci[(size_t)c * v.ldc]);
          ci[(size_t)c * v.ldc] = x;
          if (next) sq = fma(x, x, sq);
        }
        if (q == 0) *li = fma(-f, R.v0, *li);
      }
      if (next) {
        sq = group_sum<G>(sq);
        if (lane == 0) refl[(k + 1) & 1] = make_refl(v.L[(k + 1) + (size_t)(k + 1) * v.lda], sq);
      }
    }
    if (threadIdx.x == 0) v.L[k + (size_t)k * v.lda] = R.alpha;
    __syncthreads();
  }
}

// Squared column norms of L (a x a) into nr, folding the column scales dsc
// into the data first when `fold` is set; scales reset to one.
template <int G>
__device__ void jacobi_norms(double* L, int lda, int a, double* nr, double* dsc, double* dinv,
                             bool fold) {
  constexpr int PPW = 32 / G;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int grp = lane / G, q = lane % G;
  for (int base = wid * PPW; base < a; base += nw * PPW) {  // warp-uniform
    const int j = base + grp;
    const bool act = j < a;
    double s = 0.0;
    if (act) {
      const double dj = fold ? dsc[j] : 1.0;
      double* x = L + (size_t)j * lda;
      for (int r = q; r < a; r += G) {
        double e = x[r];
        if (fold) { e *= dj; x[r] = e; }
        s = fma(e, e, s);
      }
    }
    s = group_sum<G>(s);
    if (act && q == 0) { nr[j] = s; dsc[j] = 1.0; dinv[j] = 1.0; }
  }
}

// One-sided Jacobi on the columns of L (a x a, ld lda), round-robin pairing;
// on return L = W Sigma (columns orthogonal).  Column j is stored as X_j with
// the true column dsc[j] X_j; a rotation of (p, q) with tangent t becomes
// X_p -= t (d_q / d_p) X_q, X_q += t (d_p / d_q) X_p, d_p, d_q *= cos.
// nr carries the true squared norms (||x_p||^2 -= t g, ||x_q||^2 += t g).
// Returns the FP64 flops it performed: 2a per pair product and 4a per rotation
// (the counted work of the launch profiler; the iteration count is data dependent).
template <int G>
__device__ unsigned long long jacobi_columns(double* L, int lda, int a, double* nr, double* dsc,
                                             double* dinv, int* flag, unsigned int* nrot) {
  constexpr int PPW = 32 / G;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int grp = lane / G, q = lane % G;
  const int n = (a + 1) & ~1;
  int sweeps = 0;
  if (threadIdx.x == 0) *nrot = 0;
  for (int sweep = 0; sweep < 40; sweep++) {
    jacobi_norms<G>(L, lda, a, nr, dsc, dinv, sweep > 0);
    if (threadIdx.x == 0) *flag = 0;
    sweeps++;
    __syncthreads();
    for (int round = 0; round < n - 1; round++) {
      for (int base = wid * PPW; base < n / 2; base += nw * PPW) {  // warp-uniform
        // round-robin tournament: seat 0 fixed, seats 1..n-1 rotate by `round`;
        // seat m plays seat n-1-m, so every pair meets once per sweep
        const int pr = base + grp;
        int p = 0, r2 = 0;
        bool act = pr < n / 2;
        if (act) {
          const int ma = pr, mb = n - 1 - pr;
          const int pa = (ma == 0) ? 0 : ((ma - 1 + round) % (n - 1)) + 1;
          const int pb = (mb == 0) ? 0 : ((mb - 1 + round) % (n - 1)) + 1;
          p = min(pa, pb);
          r2 = max(pa, pb);
          act = (r2 < a) && (p != r2);
        }
        double* xp = L + (size_t)p * lda;
        double* xq = L + (size_t)r2 * lda;
        double g = 0.0, dp = 1.0, dq = 1.0, ip = 1.0, iq = 1.0, al = 0.0, be = 0.0;
        if (act) {
          for (int r = q; r < a; r += G) g = fma(xp[r], xq[r], g);
          dp = dsc[p]; dq = dsc[r2]; ip = dinv[p]; iq = dinv[r2]; al = nr[p]; be = nr[r2];
        }
        g = group_sum<G>(g);  // identical in every lane of the group
        if (act) {
          g *= dp * dq;
          if (g != 0.0 && g * g > 1e-30 * (al * be)) {
            // t = tan(theta), the smaller root of t^2 + 2 zeta t - 1 = 0 with
            // zeta = (be - al) / (2 g), written without the division by g
            const double del = be - al;
            const double h = sqrt(fma(del, del, 4.0 * g * g));
            const double t = (del >= 0.0 ? 2.0 * g : -2.0 * g) / (fabs(del) + h);
            const double tt1 = fma(t, t, 1.0);
            const double c = rsqrt(tt1);
            const double t1 = t * dq * ip, t2 = t * dp * iq;
            for (int r = q; r < a; r += G) {
              const double x = xp[r], y = xq[r];
              xp[r] = fma(-t1, y, x);
              xq[r] = fma(t2, x, y);
            }
            if (q == 0) {
              const double ic = tt1 * c;  // 1 / cos
              dsc[p] = dp * c;
              dsc[r2] = dq * c;
              dinv[p] = ip * ic;
              dinv[r2] = iq * ic;
              // carried squared norms: exact arithmetic keeps both >= 0, rounding
              // can push a nearly zero column's below zero
              nr[p] = fmax(fma(-t, g, al), 0.0);
              nr[r2] = fmax(fma(t, g, be), 0.0);
              *flag = 1;
              atomicAdd(nrot, 1u);
            }
          }
        }
      }
      __syncthreads();
      if ((round & 63) == 63 && round + 1 < n - 1) {
        // long sweeps: fold the scales back before they drift far from one
        jacobi_norms<G>(L, lda, a, nr, dsc, dinv, true);
        __syncthreads();
      }
    }
    const bool again = *flag != 0;
    __syncthreads();
    if (!again) break;
  }
  jacobi_norms<G>(L, lda, a, nr, dsc, dinv, true);
  __syncthreads();
  const unsigned long long pairs = (unsigned long long)a * (a - 1) / 2;
  return (unsigned long long)sweeps * pairs * 2ull * a + (unsigned long long)(*nrot) * 4ull * a;
}

// FP64 flops of the Jacobi phases since the last svd_jacobi_flops_take()
__device__ unsigned long long g_svd_jacobi_flops = 0;

template <int G>
__global__ void __launch_bounds__(512) k_svd_left(const SvdTask* __restrict__ tasks, int use_smem,
                                                  int cw_max) {
  const SvdTask t = tasks[blockIdx.x];
  const int a = t.a;
  if (a <= 0) return;
  if ((a <= SVD_SMEM_A) != (use_smem != 0)) return;
  extern __shared__ double sm[];
  __shared__ Refl refl[2];
  __shared__ int flag;
  __shared__ unsigned int nrot;
  SvdView v;
  double* aux;  // nr, dsc, dinv: 3a doubles
  int cwm;
  if (use_smem) {
    v.L = sm;
    v.lda = a + 1;                 // odd stride: no bank conflicts on row access
    v.C = sm + (size_t)(a + 1) * a;
    v.ldc = a + 1;
    aux = v.C + (size_t)(a + 1) * cw_max;
    cwm = cw_max;
  } else {
    v.L = t.work;
    v.lda = a;
    v.C = t.work + (size_t)a * a;
    v.ldc = a;
    aux = sm;
    cwm = SVD_CW;
  }
  // L starts at zero; every column of M is streamed through the chunk C and
  // annihilated against L (the reflector treats L[k,k] as its first entry).
  for (int e = threadIdx.x; e < a * a; e += blockDim.x) v.L[(e % a) + (size_t)(e / a) * v.lda] = 0.0;
  __syncthreads();
  for (int c0 = 0; c0 < t.w; c0 += cwm) {
    const int cw = min(cwm, t.w - c0);
    for (int e = threadIdx.x; e < a * cw; e += blockDim.x) {
      const int r = e % a, c = e / a;
      v.C[r + (size_t)c * v.ldc] = t.M[r + (long long)(c0 + c) * t.ldm];
    }
    __syncthreads();
    lq_chunk<G>(v, a, cw, refl);
  }
  const unsigned long long jfl =
      jacobi_columns<G>(v.L, v.lda, a, aux, aux + a, aux + 2 * a, &flag, &nrot);
  if (threadIdx.x == 0) atomicAdd(&g_svd_jacobi_flops, jfl);
  // sigma_j = |L_j|; order by decreasing sigma (ties: lower column first).
  // The chunk area (>= a doubles) is free now and holds the column norms.
  double* sg = v.C;
  for (int j = threadIdx.x; j < a; j += blockDim.x) sg[j] = sqrt(fmax(aux[j], 0.0));
  __syncthreads();
  double smax = 0.0;
  for (int j = 0; j < a; j++) smax = fmax(smax, sg[j]);
  for (int j = threadIdx.x; j < a; j += blockDim.x) {
    int pos = 0;
    for (int k = 0; k < a; k++) pos += (sg[k] > sg[j]) || (sg[k] == sg[j] && k < j);
    t.sigma[pos] = sg[j];
    const double inv = sg[j] > 0.0 ? 1.0 / sg[j] : 0.0;
    for (int r = 0; r < a; r++) t.W[r + (long long)pos * a] = v.L[r + (size_t)j * v.lda] * inv;
  }
  __syncthreads();
  // complete the basis where sigma is negligible: Gram-Schmidt (twice) against
  // the preceding columns, starting from the column or from unit vectors
  double* red = aux;  // the Jacobi scratch is free now (>= 3a >= 33 doubles for a >= 11)
  __shared__ double red_small[40];
  if (3 * a < 40) red = red_small;
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

unsigned long long svd_jacobi_flops_take() {
  unsigned long long v = 0, z = 0;
  CK(cudaMemcpyFromSymbol(&v, g_svd_jacobi_flops, sizeof(v)));
  CK(cudaMemcpyToSymbol(g_svd_jacobi_flops, &z, sizeof(z)));
  return v;
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

void run_svd_left(Arena& ar, const std::vector<SvdTask>& tasks_in, cudaStream_t s) {
  if (tasks_in.empty()) return;
  std::chrono::steady_clock::time_point t0;
  if (svd_tracing()) {
    CK(cudaStreamSynchronize(s));
    t0 = std::chrono::steady_clock::now();
  }
  std::vector<SvdTask> tasks(tasks_in);
  // Longest tasks first (one CTA per task, blocks start in index order): the
  // streaming LQ costs ~ a^2 w and the Jacobi sweeps ~ a^3, so starting the
  // expensive ones first keeps the last wave from waiting on one big task.
  std::stable_sort(tasks.begin(), tasks.end(), [](const SvdTask& x, const SvdTask& y) {
    const double cx = (double)x.a * x.a * (x.w + 10.0 * x.a);
    const double cy = (double)y.a * y.a * (y.w + 10.0 * y.a);
    return cx > cy;
  });
  for (auto& t : tasks) {
    if (t.a <= 0) continue;
    if (t.a > SVD_SMEM_A && !t.work)
      t.work = ar.alloc<double>((size_t)t.a * t.a + (size_t)t.a * SVD_CW);
    Ranges::check(t.M, mat_bytes(t.a, t.w, t.ldm), "svd M");
    Ranges::check(t.W, mat_bytes(t.a, t.a, t.a), "svd W");
    Ranges::check(t.sigma, sizeof(double) * t.a, "svd sigma");
    if (t.a > SVD_SMEM_A)
      Ranges::check(t.work, sizeof(double) * ((size_t)t.a * t.a + (size_t)t.a * SVD_CW), "svd work");
  }
  const SvdTask* d = upload(ar, tasks, s);
  int amax_s = 0, amax_g = 0, wmax = 0;
  for (auto& t : tasks) {
    if (t.a <= SVD_SMEM_A) {
      amax_s = std::max(amax_s, t.a);
      wmax = std::max(wmax, t.w);
    } else {
      amax_g = std::max(amax_g, t.a);
    }
  }
  double fl = 0.0;
  for (auto& t : tasks) fl += 2.0 * t.a * (double)t.a * t.w;
  Prof p("k_svd_left", fl, 0.0, s);
  set_max_dynamic_smem((const void*)k_svd_left<4>, SVD_SMEM_BUDGET * 8);
  set_max_dynamic_smem((const void*)k_svd_left<8>, SVD_SMEM_BUDGET * 8);
  if (amax_s > 0) {
    // shared memory: L ((a+1) x a), chunk ((a+1) x cw), 3a doubles of Jacobi
    // state.  Small blocks take a smaller budget so several CTAs share an SM.
    const long long a = amax_s;
    const long long budget = a <= 32 ? SVD_SMEM_BUDGET / 4 : (a <= 80 ? SVD_SMEM_BUDGET / 2
                                                                        : SVD_SMEM_BUDGET);
    long long cw = (budget - (a + 1) * a - 3 * a) / (a + 1);
    cw = std::min<long long>(cw, std::max(wmax, 1));
    if (cw < 1) throw Error(IFMM_ERR_CUDA, "internal: SVD shared-memory budget too small");
    const size_t smem = sizeof(double) * (size_t)((a + 1) * (a + cw) + 3 * a);
    if (a <= 32) {
      k_svd_left<4><<<(int)tasks.size(), 128, smem, s>>>(d, 1, (int)cw);
    } else {
      k_svd_left<8><<<(int)tasks.size(), a <= 64 ? 256 : 512, smem, s>>>(d, 1, (int)cw);
    }
    CK_LAUNCH("k_svd_left(smem)");
  }
  if (amax_g > 0) {
    k_svd_left<8><<<(int)tasks.size(), 512, sizeof(double) * 3 * (size_t)amax_g, s>>>(d, 0, SVD_CW);
    CK_LAUNCH("k_svd_left(global)");
  }
  if (svd_tracing()) {
    CK(cudaStreamSynchronize(s));
    int amax = 0, wm = 0;
    double wsum = 0.0;
    for (auto& t : tasks) { amax = std::max(amax, t.a); wm = std::max(wm, t.w); wsum += t.w; }
    std::fprintf(stderr, "[svd] tasks %zu, max a %d, max w %d, avg w %.0f, %.4f s\n", tasks.size(),
                 amax, wm, wsum / tasks.size(),
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
// directions (above the SVD's basis-completion threshold 1e-13 a s[0] for the
// k <= 1000 rows these products have)
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
    if (t.k != k || t.k < 1 || t.k > t.a)
      throw Error(IFMM_ERR_CUDA, "internal: randomised SVD tasks need a common k, 1 <= k <= a");
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
