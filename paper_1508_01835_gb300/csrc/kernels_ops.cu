// kernels_ops.cu -- kernel evaluation, Chebyshev operators and block-sparse
// products of the IFMM library.
//
// Operators (Sec. 2.1, Sec. 3): the leaf interpolation U_i = V_i (L2P / P2M),
// the child-to-parent transfer T_c (L2L, its transpose M2M), the M2L blocks
// K_iq between Chebyshev nodes of well-separated boxes, and the exact
// near-field blocks S_ij (P2P).  The interpolant of the black-box FMM the
// paper cites is S_n(x, t) = 1/n + (2/n) sum_{k=1}^{n-1} T_k(x) T_k(t).
#include "kernels_ops.cuh"

namespace ifmm {

__device__ __forceinline__ double kernel_value(const KSpec& k, double r) {
  if (r == 0.0) return k.diag;
  if (k.kind == IFMM_K_INV_R) return 1.0 / r;
  if (k.kind == IFMM_K_GAUSSIAN) return exp(-(r * r) / (2.0 * k.param * k.param));
  return (r < k.param) ? r / k.param : k.param / r;  // Eq. (K_ij)
}

__device__ __forceinline__ double dist(const double* x, const double* y, int dim) {
  double s = 0.0;
  for (int d = 0; d < dim; d++) {
    const double t = x[d] - y[d];
    s += t * t;
  }
  return sqrt(s);
}

// one-dimensional interpolant S_n(x, t_a)
__device__ double cheb_S1(const ChebSpec& c, double x, int a) {
  const double t = c.t[a];
  double s = 1.0 / c.n;
  if (c.n > 1) {
    double tx0 = 1.0, tx1 = x, tt0 = 1.0, tt1 = t;
    s += (2.0 / c.n) * tx1 * tt1;
    for (int k = 2; k < c.n; k++) {
      const double tx2 = 2.0 * x * tx1 - tx0, tt2 = 2.0 * t * tt1 - tt0;
      s += (2.0 / c.n) * tx2 * tt2;
      tx0 = tx1; tx1 = tx2; tt0 = tt1; tt1 = tt2;
    }
  }
  return s;
}

// U[p, a] of every leaf: one thread per (point, node)
__global__ void k_leaf_interp(ChebSpec c, int dim, const double* __restrict__ pts_tree,
                              const LeafGeom* __restrict__ leaves, int nleaves,
                              double* __restrict__ U) {
  const int i = blockIdx.x;
  if (i >= nleaves) return;
  const LeafGeom g = leaves[i];
  const int m = g.p1 - g.p0;
  for (int e = threadIdx.x; e < m * c.nd; e += blockDim.x) {
    const int p = e % m, a = e / m;
    const double* x = pts_tree + (size_t)(g.p0 + p) * dim;
    double v = 1.0;
    int aa = a;
    for (int d = 0; d < dim; d++) {
      const double xi = (x[d] - g.centre[d]) / g.h;
      v *= cheb_S1(c, xi, aa % c.n);
      aa /= c.n;
    }
    U[g.uoff + e] = v;
  }
}

// T_c[a, b] = prod_d S_n(shift_d + t_{a_d} / 2, t_{b_d}), shift = +-1/2
__global__ void k_transfer(ChebSpec c, int dim, double* __restrict__ T) {
  const int child = blockIdx.x;
  const int nd = c.nd;
  for (int e = threadIdx.x; e < nd * nd; e += blockDim.x) {
    const int a = e % nd, b = e / nd;
    int aa = a, bb = b;
    double v = 1.0;
    for (int d = 0; d < dim; d++) {
      const double shift = ((child >> d) & 1) ? 0.5 : -0.5;
      v *= cheb_S1(c, shift + 0.5 * c.t[aa % c.n], bb % c.n);
      aa /= c.n;
      bb /= c.n;
    }
    T[(size_t)child * nd * nd + e] = v;
  }
}

// M2L table of one level: K_off[a, b] = K(|x_a - y_b|) with x_a = h t_a and
// y_b = 2 h delta + h t_b, delta in [-3, 3]^dim (offset index sum (delta_d+3) 7^d)
__global__ void k_m2l_table(ChebSpec c, int dim, KSpec ks, double h, double* __restrict__ K) {
  const int o = blockIdx.x;
  int delta[3] = {0, 0, 0};
  int oo = o;
  for (int d = 0; d < dim; d++) { delta[d] = oo % 7 - 3; oo /= 7; }
  const int nd = c.nd;
  for (int e = threadIdx.x; e < nd * nd; e += blockDim.x) {
    const int a = e % nd, b = e / nd;
    double xa[3], yb[3];
    int aa = a, bb = b;
    for (int d = 0; d < dim; d++) {
      xa[d] = h * c.t[aa % c.n];
      yb[d] = 2.0 * h * delta[d] + h * c.t[bb % c.n];
      aa /= c.n;
      bb /= c.n;
    }
    K[(size_t)o * nd * nd + e] = kernel_value(ks, dist(xa, yb, dim));
  }
}

// near-field blocks S_ij, one CTA per (i, j) pair
__global__ void k_p2p_blocks(KSpec ks, int dim, const double* __restrict__ pts_tree,
                             const P2PTask* __restrict__ tasks, double* __restrict__ S) {
  const P2PTask t = tasks[blockIdx.x];
  const int mi = t.i1 - t.i0, mj = t.j1 - t.j0;
  for (int e = threadIdx.x; e < mi * mj; e += blockDim.x) {
    const int r = e % mi, c = e / mi;
    const int gi = t.i0 + r, gj = t.j0 + c;
    const double v = (gi == gj) ? ks.diag
                                : kernel_value(ks, dist(pts_tree + (size_t)gi * dim,
                                                        pts_tree + (size_t)gj * dim, dim));
    S[t.off + e] = v;
  }
}

// y = A x over all points (direct sum), user order, one thread per target
__global__ void __launch_bounds__(256) k_direct(KSpec ks, int dim, const double* __restrict__ pts,
                                                long long N, const double* __restrict__ x,
                                                long long ldx, double* __restrict__ y,
                                                long long ldy, int col) {
  __shared__ double sp[256 * 3];
  __shared__ double sx[256];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double xi[3] = {0, 0, 0};
  if (i < N)
    for (int d = 0; d < dim; d++) xi[d] = pts[i * dim + d];
  double acc = 0.0;
  const double* xc = x + (long long)col * ldx;
  for (long long j0 = 0; j0 < N; j0 += 256) {
    const long long j = j0 + threadIdx.x;
    if (j < N) {
      for (int d = 0; d < dim; d++) sp[threadIdx.x * 3 + d] = pts[j * dim + d];
      sx[threadIdx.x] = xc[j];
    }
    __syncthreads();
    const int nj = (int)min((long long)256, N - j0);
    if (i < N) {
      for (int q = 0; q < nj; q++) {
        const long long gj = j0 + q;
        const double v = (gj == i) ? ks.diag : kernel_value(ks, dist(xi, sp + q * 3, dim));
        acc += v * sx[q];
      }
    }
    __syncthreads();
  }
  if (i < N) y[(long long)col * ldy + i] = acc;
}

// Block-row sparse product, one warp per job (SpJob), for FP64 and FP32.
// A job is one tile of MR rows of a row (MR = 8, 16 or 32 from the row's
// height; taller rows are several tiles) over a contiguous range of its
// concatenated entry columns.  A pass serves up to NBT right-hand sides (4 or
// 32) from one read of the job's matrix entries: for every chunk of KC entry
// columns the warp copies the x values (NBT columns, [k][column] with row
// stride NBT + 16 / sizeof(T)) and the tile's A values ([k][row]) into its
// shared memory with cp.async, all of the chunk's copies in flight together;
// lane (r, g) then keeps row r of the tile for the columns g*CPL ..
// g*CPL+CPL-1 in registers (32 / MR column groups), reading one A value and
// CPL x values (16-byte loads) per k.  Sums run over the job's segments in
// order; a tile cut along k meets its partial sums in k_spmm_reduce /
// k_spmm_f32_reduce in job order, so results do not depend on scheduling.
constexpr int SW_WARPS = 8, SW_NB = 32;
// k values per staged chunk: 32 (FP32) or 16 (FP64), so that a warp's stage
// (x: KC x (NBT + pad), A: KC x MR) stays near 8 KB
template <class T>
__host__ __device__ constexpr int sw_kc() {
  return sizeof(T) == 4 ? 32 : 16;
}

template <class T>
struct SpT;
template <>
struct SpT<double> {
  using Row = SpRow;
  using Ent = SpEnt;
  __device__ static bool trans(const SpEnt& e) { return e.transA != 0; }
};
template <>
struct SpT<float> {
  using Row = SpRowF;
  using Ent = SpEntF;
  __device__ static bool trans(const SpEntF&) { return false; }
};
// staged x row stride (elements) for passes of NBT columns
template <class T, int NBT>
__host__ __device__ constexpr int sw_xs() {
  return NBT + 16 / (int)sizeof(T);
}
// elements of one warp's stage: x (KC rows of sw_xs) then A (KC x MR)
template <class T, int MR, int NBT>
__host__ __device__ constexpr int sw_stage() {
  return sw_kc<T>() * (sw_xs<T, NBT>() + MR);
}

// asynchronous element copy global -> shared (cp.async); a false `ok` copies
// no bytes and zero-fills the element
template <class T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem, bool ok) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem),
                 "r"(ok ? 4 : 0)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem),
                 "r"(ok ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_drain() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// n consecutive values, with 16-byte loads where n * sizeof(T) allows
template <class T, int N>
__device__ __forceinline__ void vload(const T* p, T (&v)[N]) {
  if constexpr (N * sizeof(T) % 16 == 0) {
    constexpr int VN = 16 / (int)sizeof(T);
#pragma unroll
    for (int q = 0; q < N / VN; q++) {
      if constexpr (sizeof(T) == 4) {
        const float4 u = reinterpret_cast<const float4*>(p)[q];
        v[4 * q] = u.x; v[4 * q + 1] = u.y; v[4 * q + 2] = u.z; v[4 * q + 3] = u.w;
      } else {
        const double2 u = reinterpret_cast<const double2*>(p)[q];
        v[2 * q] = u.x; v[2 * q + 1] = u.y;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = p[i];
  }
}

template <class T, int MR, int NBT>
__device__ __forceinline__ void spmm_warp_job(const typename SpT<T>::Row& R,
                                              const typename SpT<T>::Ent* __restrict__ ents,
                                              const SpJob& J, const SpSeg* __restrict__ segs,
                                              T* __restrict__ part, long long pld, int c0,
                                              int nb, T* xs, int lane) {
  constexpr int CPL = NBT * MR / 32;  // columns per lane: 32 / MR column groups
  constexpr int XS = sw_xs<T, NBT>();
  constexpr int KC = sw_kc<T>();
  T* as = xs + KC * XS;  // staged A: as[k * MR + row of the tile]
  const int rl = lane % MR, g = lane / MR;
  {  // the job's tile: rows J.r0 .. J.r0 + J.mt - 1 (J.mt <= MR)
    const int r = J.r0 + rl;
    const bool rin = rl < J.mt;
    T acc[CPL];
#pragma unroll
    for (int j = 0; j < CPL; j++) acc[j] = T(0);
    for (int si = J.s0; si < J.s0 + J.ns; si++) {
      const SpSeg S = segs[si];
      const typename SpT<T>::Ent E = ents[S.ent];
      const bool tr = SpT<T>::trans(E);
      for (int kc0 = S.k0; kc0 < S.k1; kc0 += KC) {
        const int kk = min(KC, S.k1 - kc0);
        __syncwarp();  // the previous chunk has been read
        // the chunk's x and A values are copied with cp.async, all in flight
        // together (padding columns and rows zero-filled)
        for (int e = lane; e < kk * NBT; e += 32) {
          const int k = e % kk, c = e / kk;
          const bool ok = c < nb;
          cp_async_elem(xs + k * XS + c, E.x + kc0 + k + (ok ? (long long)(c0 + c) * E.ldx : 0),
                        ok);
        }
        if (E.A) {
          if (!tr) {  // lanes along the tile's rows (contiguous in a column)
            for (int e = lane; e < kk * MR; e += 32) {
              const int rr = e % MR, k = e / MR;
              const bool ok = rr < J.mt;
              cp_async_elem(as + k * MR + rr,
                            E.A + (ok ? J.r0 + rr : 0) + (long long)(kc0 + k) * E.lda, ok);
            }
          } else {  // lanes along k (contiguous in a stored row)
            for (int e = lane; e < kk * MR; e += 32) {
              const int k = e % kk, rr = e / kk;
              const bool ok = rr < J.mt;
              cp_async_elem(as + k * MR + rr,
                            E.A + (long long)(ok ? J.r0 + rr : 0) * E.lda + kc0 + k, ok);
            }
          }
        }
        cp_async_drain();
        __syncwarp();
        const T* xr = xs + g * CPL;
        if (!E.A) {  // identity: output row r takes x[r] (rows k0 .. k1 of this entry)
          if (rin && r >= kc0 && r < kc0 + kk) {
            const T* xk = xr + (r - kc0) * XS;
#pragma unroll
            for (int j = 0; j < CPL; j++) acc[j] = fma(E.alpha, xk[j], acc[j]);
          }
        } else if (rin) {
#pragma unroll 4
          for (int k = 0; k < kk; k++) {
            const T av = E.alpha * as[k * MR + rl];
            T v[CPL];
            vload<T, CPL>(xr + k * XS, v);
#pragma unroll
            for (int j = 0; j < CPL; j++) acc[j] = fma(av, v[j], acc[j]);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < CPL; j++) {
      const int c = g * CPL + j;
      if (!rin || c >= nb) continue;
      if (J.part < 0) {
        T* y = R.y + (long long)(c0 + c) * R.ldy + r;
        *y = (R.beta == T(0)) ? acc[j] : fma(R.beta, *y, acc[j]);
      } else {
        part[J.part + rl + (long long)c * pld] = acc[j];
      }
    }
  }
}

// jobs[0 .. njobs) all belong to rows of the class MR (m <= 8, <= 16, > 16);
// passes of NBT (4 or 32) columns
template <class T, int MR, int NBT>
__global__ void __launch_bounds__(32 * SW_WARPS, 2)
    k_spmm_warp(const typename SpT<T>::Row* __restrict__ rows,
                const typename SpT<T>::Ent* __restrict__ ents, const SpJob* __restrict__ jobs,
                int njobs, const SpSeg* __restrict__ segs, T* __restrict__ part, long long pld,
                int c0, int nb) {
  extern __shared__ __align__(16) unsigned char sw_smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jb = blockIdx.x * SW_WARPS + w;
  if (jb >= njobs) return;  // warp-uniform; no block-wide barrier in this kernel
  T* xs = reinterpret_cast<T*>(sw_smem) + (size_t)w * sw_stage<T, MR, NBT>();
  const SpJob J = jobs[jb];
  const typename SpT<T>::Row R = rows[J.row];
  spmm_warp_job<T, MR, NBT>(R, ents, J, segs, part, pld, c0, nb, xs, lane);
}

// every row class in one launch: the warp's job picks its tile height (jobs
// are grouped by class, so a CTA's warps mostly take the same branch)
template <class T, int NBT>
__global__ void __launch_bounds__(32 * SW_WARPS, 2)
    k_spmm_warp_any(const typename SpT<T>::Row* __restrict__ rows,
                    const typename SpT<T>::Ent* __restrict__ ents, const SpJob* __restrict__ jobs,
                    int njobs, const SpSeg* __restrict__ segs, T* __restrict__ part,
                    long long pld, int c0, int nb) {
  extern __shared__ __align__(16) unsigned char sw_smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jb = blockIdx.x * SW_WARPS + w;
  if (jb >= njobs) return;  // warp-uniform; no block-wide barrier in this kernel
  T* xs = reinterpret_cast<T*>(sw_smem) + (size_t)w * sw_stage<T, 32, NBT>();
  const SpJob J = jobs[jb];
  const typename SpT<T>::Row R = rows[J.row];
  if (R.m <= 8) spmm_warp_job<T, 8, NBT>(R, ents, J, segs, part, pld, c0, nb, xs, lane);
  else if (R.m <= 16) spmm_warp_job<T, 16, NBT>(R, ents, J, segs, part, pld, c0, nb, xs, lane);
  else spmm_warp_job<T, 32, NBT>(R, ents, J, segs, part, pld, c0, nb, xs, lane);
}

// row class of a job: 0 (m <= 8), 1 (m <= 16), 2 (m > 16)
static int sw_class(int m) { return m <= 8 ? 0 : m <= 16 ? 1 : 2; }

template <class T, int MR, int NBT>
static void launch_sw_tile(const typename SpT<T>::Row* rows, const typename SpT<T>::Ent* ents,
                           const SpJob* jobs, int njobs, const SpSeg* segs, T* part,
                           long long pld, int c0, int nb, cudaStream_t s) {
  const int smem = SW_WARPS * sw_stage<T, MR, NBT>() * (int)sizeof(T);
  set_max_dynamic_smem((const void*)k_spmm_warp<T, MR, NBT>, smem);
  k_spmm_warp<T, MR, NBT><<<(njobs + SW_WARPS - 1) / SW_WARPS, 32 * SW_WARPS, smem, s>>>(
      rows, ents, jobs, njobs, segs, part, pld, c0, nb);
}
template <class T, int MR>
static void launch_sw_class(const typename SpT<T>::Row* rows, const typename SpT<T>::Ent* ents,
                            const SpJob* jobs, int njobs, const SpSeg* segs, T* part,
                            long long pld, int c0, int nb, cudaStream_t s) {
  if (njobs <= 0) return;
  if (nb <= 4) launch_sw_tile<T, MR, 4>(rows, ents, jobs, njobs, segs, part, pld, c0, nb, s);
  else launch_sw_tile<T, MR, 32>(rows, ents, jobs, njobs, segs, part, pld, c0, nb, s);
}

template <class T, int NBT>
static void launch_sw_any(const typename SpT<T>::Row* rows, const typename SpT<T>::Ent* ents,
                          const SpJob* jobs, int njobs, const SpSeg* segs, T* part, long long pld,
                          int c0, int nb, cudaStream_t s) {
  const int smem = SW_WARPS * sw_stage<T, 32, NBT>() * (int)sizeof(T);
  set_max_dynamic_smem((const void*)k_spmm_warp_any<T, NBT>, smem);
  k_spmm_warp_any<T, NBT><<<(njobs + SW_WARPS - 1) / SW_WARPS, 32 * SW_WARPS, smem, s>>>(
      rows, ents, jobs, njobs, segs, part, pld, c0, nb);
}

// Launch of a plan's jobs (grouped by row class at plan time): one kernel for
// a single class, one kernel over all classes otherwise (IFMM_SPMM_SPLIT=1:
// one launch per class)
template <class T>
static void launch_spmm_warp(const typename SpT<T>::Row* rows, const typename SpT<T>::Ent* ents,
                             const SpJob* jobs, const int* ncls, const SpSeg* segs, T* part,
                             long long pld, int c0, int nb, cudaStream_t s) {
  static const bool split = [] {
    const char* e = std::getenv("IFMM_SPMM_SPLIT");
    return e && e[0] == '1';
  }();
  const int classes = (ncls[0] > 0) + (ncls[1] > 0) + (ncls[2] > 0);
  if (classes > 1 && !split) {
    const int njobs = ncls[0] + ncls[1] + ncls[2];
    if (nb <= 4) launch_sw_any<T, 4>(rows, ents, jobs, njobs, segs, part, pld, c0, nb, s);
    else launch_sw_any<T, 32>(rows, ents, jobs, njobs, segs, part, pld, c0, nb, s);
    return;
  }
  launch_sw_class<T, 8>(rows, ents, jobs, ncls[0], segs, part, pld, c0, nb, s);
  launch_sw_class<T, 16>(rows, ents, jobs + ncls[0], ncls[1], segs, part, pld, c0, nb, s);
  launch_sw_class<T, 32>(rows, ents, jobs + ncls[0] + ncls[1], ncls[2], segs, part, pld, c0, nb,
                         s);
}

// jobs grouped by row class (stable); each job keeps its partial-sum slot
template <class Row>
static void group_jobs(const std::vector<Row>& rows, std::vector<SpJob>& jobs, int* ncls) {
  std::vector<SpJob> out;
  out.reserve(jobs.size());
  for (int c = 0; c < 3; c++) {
    ncls[c] = 0;
    for (const SpJob& J : jobs)
      if (sw_class(rows[J.row].m) == c) {
        out.push_back(J);
        ncls[c]++;
      }
  }
  jobs.swap(out);
}

// y = beta y + (sum of the row's partial sums, in job order)
__global__ void __launch_bounds__(256) k_spmm_reduce(const SpRow* __restrict__ rows,
                                                     const SpRed* __restrict__ reds,
                                                     const double* __restrict__ part,
                                                     long long pld, int c0, int nb) {
  const SpRed D = reds[blockIdx.x];
  const SpRow R = rows[D.row];
  // every thread takes (row, column) pairs of the tile
  for (int e = threadIdx.x; e < D.mt * nb; e += blockDim.x) {
    const int r = e % D.mt, c = e / D.mt;
    const double* pp = part + D.base + r + (long long)c * pld;
    double v = 0.0;
    for (int j = 0; j < D.nj; j++) v += pp[(long long)j * D.mt];
    double* y = R.y + (long long)(c0 + c) * R.ldy + D.r0 + r;
    *y = (R.beta == 0.0) ? v : fma(R.beta, *y, v);
  }
}

// Job split shared by the FP64 and FP32 products: every row is cut into tiles
// of 8, 16 or 32 rows (the kernel's class for the row's height); a tile whose
// work exceeds the target (about 32 jobs, one warp each, per SM; at least
// 4096 multiply-adds per right-hand side) is cut into up to 64 contiguous
// column ranges whose partial sums are added by the reduce kernel.
template <class Row, class Ent>
static void split_jobs(const std::vector<Row>& rows, const std::vector<Ent>& ents, int nsm,
                       std::vector<SpJob>& jobs, std::vector<SpSeg>& segs,
                       std::vector<SpRed>& reds, long long& poff) {
  double total = 0.0;
  for (const Row& R : rows)
    for (int e = R.e0; e < R.e0 + R.ne; e++)
      total += (ents[e].A ? (double)R.m : 1.0) * ents[e].k;
  const double target = std::max(4096.0, total / (32.0 * nsm));
  poff = 0;
  for (int ri = 0; ri < (int)rows.size(); ri++) {
    const Row& R = rows[ri];
    long long K = 0;
    for (int e = R.e0; e < R.e0 + R.ne; e++) K += ents[e].k;
    const int mr = R.m <= 8 ? 8 : R.m <= 16 ? 16 : 32;  // rows per tile (the kernel's class)
    for (int r0 = 0; r0 < R.m; r0 += mr) {
      const int mt = std::min(mr, R.m - r0);
      double work = 0.0;
      for (int e = R.e0; e < R.e0 + R.ne; e++)
        work += (ents[e].A ? (double)mt : 1.0) * ents[e].k;
      int ns = (int)std::ceil(work / target);
      if ((long long)ns > std::max(K, 1ll)) ns = (int)std::max(K, 1ll);
      ns = std::max(1, std::min(ns, 64));
      if (ns > 1) reds.push_back({ri, ns, r0, mt, poff});
      for (int j = 0; j < ns; j++) {
        const long long K0 = K * j / ns, K1 = K * (j + 1) / ns;
        SpJob J{ri, (int)segs.size(), 0, r0, mt, ns > 1 ? poff + (long long)j * mt : -1};
        long long base = 0;
        for (int e = R.e0; e < R.e0 + R.ne; e++) {
          const long long lo = std::max(K0, base), hi = std::min(K1, base + ents[e].k);
          if (lo < hi) {
            segs.push_back({e, (int)(lo - base), (int)(hi - base)});
            J.ns++;
          }
          base += ents[e].k;
        }
        jobs.push_back(J);
      }
      if (ns > 1) poff += (long long)ns * mt;
    }
  }
}

static int sm_count() {
  int dev = 0, nsm = 1;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  return nsm;
}

SpmmPlan plan_spmm(Arena& ar, const std::vector<SpRow>& rows, const std::vector<SpEnt>& ents,
                   int cap, cudaStream_t s) {
  SpmmPlan P;
  if (rows.empty()) return P;
  if (cap < 1) cap = 1;
  validate_spmm(rows, ents, cap);
  for (const SpRow& R : rows) {
    P.vbytes += 8.0 * R.m;
    for (int e = R.e0; e < R.e0 + R.ne; e++) {
      const SpEnt& E = ents[e];
      P.flops += 2.0 * R.m * (double)E.k;
      P.vbytes += 8.0 * E.k;
      P.bytes += E.A ? 8.0 * R.m * (double)E.k : 0.0;
    }
  }
  std::vector<SpJob> jobs;
  std::vector<SpSeg> segs;
  std::vector<SpRed> reds;
  long long poff = 0;
  split_jobs(rows, ents, sm_count(), jobs, segs, reds, poff);
  group_jobs(rows, jobs, P.ncls);
  P.rows = upload(ar, rows, s);
  P.ents = upload(ar, ents, s);
  P.jobs = upload(ar, jobs, s);
  P.segs = segs.empty() ? nullptr : upload(ar, segs, s);
  P.reds = reds.empty() ? nullptr : upload(ar, reds, s);
  P.njobs = (int)jobs.size();
  P.nreds = (int)reds.size();
  P.part_ld = poff;
  P.cap = cap;
  if (poff > 0) P.part = ar.alloc<double>((size_t)poff * cap);
  return P;
}

// ---------------------------------------------------------------------------
// FP32 block-row products (reduced-precision sweeps, FP32 far field): the
// same job split and the same warp kernel in FP32.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_spmm_f32_reduce(const SpRowF* __restrict__ rows,
                                                         const SpRed* __restrict__ reds,
                                                         const float* __restrict__ part,
                                                         long long pld, int c0, int nb) {
  const SpRed D = reds[blockIdx.x];
  const SpRowF R = rows[D.row];
  for (int e = threadIdx.x; e < D.mt * nb; e += blockDim.x) {
    const int r = e % D.mt, c = e / D.mt;
    const float* pp = part + D.base + r + (long long)c * pld;
    float v = 0.0f;
    for (int j = 0; j < D.nj; j++) v += pp[(long long)j * D.mt];
    float* y = R.y + (long long)(c0 + c) * R.ldy + D.r0 + r;
    *y = (R.beta == 0.0f) ? v : fmaf(R.beta, *y, v);
  }
}

SpmmPlanF plan_spmm_f32(Arena& ar, const std::vector<SpRowF>& rows,
                        const std::vector<SpEntF>& ents, int cap, cudaStream_t s) {
  SpmmPlanF P;
  if (rows.empty()) return P;
  if (cap < 1) cap = 1;
  for (const SpRowF& R : rows) {
    Ranges::check(R.y, sizeof(float) * ((size_t)(cap - 1) * R.ldy + R.m), "spmm32 y");
    P.vbytes += 4.0 * R.m;
    for (int e = R.e0; e < R.e0 + R.ne; e++) {
      const SpEntF& E = ents[e];
      if (E.A) Ranges::check(E.A, sizeof(float) * ((size_t)(E.k - 1) * E.lda + R.m), "spmm32 A");
      Ranges::check(E.x, sizeof(float) * ((size_t)(cap - 1) * E.ldx + E.k), "spmm32 x");
      P.flops += 2.0 * R.m * (double)E.k;
      P.vbytes += 4.0 * E.k;
      P.bytes += E.A ? 4.0 * R.m * (double)E.k : 0.0;
    }
  }
  std::vector<SpJob> jobs;
  std::vector<SpSeg> segs;
  std::vector<SpRed> reds;
  long long poff = 0;
  split_jobs(rows, ents, sm_count(), jobs, segs, reds, poff);
  group_jobs(rows, jobs, P.ncls);
  P.rows = upload(ar, rows, s);
  P.ents = upload(ar, ents, s);
  P.jobs = upload(ar, jobs, s);
  P.segs = segs.empty() ? nullptr : upload(ar, segs, s);
  P.reds = reds.empty() ? nullptr : upload(ar, reds, s);
  P.njobs = (int)jobs.size();
  P.nreds = (int)reds.size();
  P.part_ld = poff;
  P.cap = cap;
  if (poff > 0) P.part = ar.alloc<float>((size_t)poff * std::min(cap, 32));
  return P;
}

void launch_spmm_f32(const SpmmPlanF& p, int nrhs, cudaStream_t s) {
  if (p.njobs <= 0 || nrhs <= 0) return;
  for (int c0 = 0; c0 < nrhs; c0 += SW_NB) {
    const int nb = std::min(SW_NB, nrhs - c0);
    {
      Prof pr("k_spmm_f32", p.flops * nb, p.bytes + p.vbytes * nb, s);
      launch_spmm_warp<float>(p.rows, p.ents, p.jobs, p.ncls, p.segs, p.part, p.part_ld, c0, nb,
                              s);
      CK_LAUNCH("k_spmm_f32");
    }
    if (p.nreds > 0) {
      Prof pr("k_spmm_f32_reduce", 0.0, 8.0 * p.part_ld * nb, s);
      k_spmm_f32_reduce<<<p.nreds, 256, 0, s>>>(p.rows, p.reds, p.part, p.part_ld, c0, nb);
      CK_LAUNCH("k_spmm_f32_reduce");
    }
  }
}

// FP64 <-> FP32 copies with a row permutation (the reduced-precision sweeps
// read b and write x in FP64, user order; they work in FP32, tree order).
__global__ void k_gather_rows_f32(const long long* __restrict__ perm, long long N,
                                  const double* __restrict__ in, long long ldi,
                                  float* __restrict__ out, long long ldo, int ncols) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const long long src = perm[t];
  for (int c = 0; c < ncols; c++) out[t + c * ldo] = (float)in[src + c * ldi];
}
__global__ void k_scatter_rows_f32(const long long* __restrict__ perm, long long N,
                                   const float* __restrict__ in, long long ldi,
                                   double* __restrict__ out, long long ldo, int ncols) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const long long dst = perm[t];
  for (int c = 0; c < ncols; c++) out[dst + c * ldo] = (double)in[t + c * ldi];
}
void launch_gather_rows_f32(const long long* perm, long long N, const double* in, long long ldi,
                            float* out, long long ldo, int ncols, cudaStream_t s) {
  if (N <= 0) return;
  k_gather_rows_f32<<<(int)((N + 255) / 256), 256, 0, s>>>(perm, N, in, ldi, out, ldo, ncols);
  CK_LAUNCH("k_gather_rows_f32");
}
void launch_scatter_rows_f32(const long long* perm, long long N, const float* in, long long ldi,
                             double* out, long long ldo, int ncols, cudaStream_t s) {
  if (N <= 0) return;
  k_scatter_rows_f32<<<(int)((N + 255) / 256), 256, 0, s>>>(perm, N, in, ldi, out, ldo, ncols);
  CK_LAUNCH("k_scatter_rows_f32");
}

// Element-wise FP64 -> FP32 narrowing of a list of arrays (one CTA per array).
__global__ void k_narrow(const NarrowTask* __restrict__ t) {
  const NarrowTask T = t[blockIdx.x];
  for (long long e = threadIdx.x; e < T.n; e += blockDim.x) T.dst[e] = (float)T.src[e];
}
void launch_narrow(Arena& ar, const std::vector<NarrowTask>& v, cudaStream_t s) {
  std::vector<NarrowTask> keep;
  for (const NarrowTask& t : v)
    if (t.n > 0) {
      Ranges::check(t.src, sizeof(double) * t.n, "narrow src");
      Ranges::check(t.dst, sizeof(float) * t.n, "narrow dst");
      keep.push_back(t);
    }
  if (keep.empty()) return;
  k_narrow<<<(int)keep.size(), 256, 0, s>>>(upload(ar, keep, s));
  CK_LAUNCH("k_narrow");
}

__global__ void k_narrow_t(const NarrowTTask* __restrict__ t) {
  const NarrowTTask T = t[blockIdx.x];
  const long long n = (long long)T.rows * T.cols;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) {
    const int c = (int)(e % T.cols), r = (int)(e / T.cols);  // dst[c + r * cols]
    T.dst[e] = (float)T.src[r + (long long)c * T.rows];
  }
}
void launch_narrow_t(Arena& ar, const std::vector<NarrowTTask>& v, cudaStream_t s) {
  std::vector<NarrowTTask> keep;
  for (const NarrowTTask& t : v)
    if (t.rows > 0 && t.cols > 0) {
      const size_t n = (size_t)t.rows * t.cols;
      Ranges::check(t.src, sizeof(double) * n, "narrow_t src");
      Ranges::check(t.dst, sizeof(float) * n, "narrow_t dst");
      keep.push_back(t);
    }
  for (size_t b = 0; b < keep.size(); b += 65535) {
    const size_t e = std::min(keep.size(), b + 65535);
    std::vector<NarrowTTask> part(keep.begin() + b, keep.begin() + e);
    k_narrow_t<<<(int)part.size(), 128, 0, s>>>(upload(ar, part, s));
    CK_LAUNCH("k_narrow_t");
  }
}

__global__ void k_gather_rows_2(const long long* __restrict__ perm, long long N,
                                const double* __restrict__ in, long long ldi,
                                double* __restrict__ out64, float* __restrict__ out32,
                                long long ldo, int ncols) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const long long src = perm[t];
  for (int c = 0; c < ncols; c++) {
    const double v = in[src + c * ldi];
    out64[t + c * ldo] = v;
    out32[t + c * ldo] = (float)v;
  }
}
void launch_gather_rows_2(const long long* perm, long long N, const double* in, long long ldi,
                          double* out64, float* out32, long long ldo, int ncols, cudaStream_t s) {
  if (N <= 0 || ncols <= 0) return;
  Prof p("k_gather_rows_2", 0.0, (8.0 + 8.0 + 8.0 + 4.0) * N * ncols, s);
  k_gather_rows_2<<<(int)((N + 255) / 256), 256, 0, s>>>(perm, N, in, ldi, out64, out32, ldo,
                                                         ncols);
  CK_LAUNCH("k_gather_rows_2");
}

__global__ void k_scatter_rows_add(const long long* __restrict__ perm, long long N,
                                   const double* __restrict__ in64, const float* __restrict__ in32,
                                   long long ldi, double* __restrict__ out, long long ldo,
                                   int ncols) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const long long dst = perm[t];
  for (int c = 0; c < ncols; c++)
    out[dst + c * ldo] = in64[t + c * ldi] + (double)in32[t + c * ldi];
}
void launch_scatter_rows_add(const long long* perm, long long N, const double* in64,
                             const float* in32, long long ldi, double* out, long long ldo,
                             int ncols, cudaStream_t s) {
  if (N <= 0 || ncols <= 0) return;
  Prof p("k_scatter_rows_add", 0.0, (8.0 + 8.0 + 4.0 + 8.0) * N * ncols, s);
  k_scatter_rows_add<<<(int)((N + 255) / 256), 256, 0, s>>>(perm, N, in64, in32, ldi, out, ldo,
                                                            ncols);
  CK_LAUNCH("k_scatter_rows_add");
}

void launch_spmm(const SpmmPlan& p, int nrhs, cudaStream_t s) {
  if (p.njobs <= 0 || nrhs <= 0) return;
  const int step = std::min(p.cap, SW_NB);  // the partial sums hold cap columns
  for (int c0 = 0; c0 < nrhs; c0 += step) {
    const int nb = std::min(step, nrhs - c0);
    {
      Prof pr("k_spmm_job", p.flops * nb, p.bytes + p.vbytes * nb, s);
      launch_spmm_warp<double>(p.rows, p.ents, p.jobs, p.ncls, p.segs, p.part, p.part_ld, c0, nb,
                               s);
      CK_LAUNCH("k_spmm_job");
    }
    if (p.nreds > 0) {
      Prof pr("k_spmm_reduce", 0.0, 16.0 * p.part_ld * nb, s);
      k_spmm_reduce<<<p.nreds, 256, 0, s>>>(p.rows, p.reds, p.part, p.part_ld, c0, nb);
      CK_LAUNCH("k_spmm_reduce");
    }
  }
}

void validate_spmm(const std::vector<SpRow>& rows, const std::vector<SpEnt>& ents, int nrhs) {
  if (!Ranges::on()) return;
  for (const SpRow& R : rows) {
    Ranges::check(R.y, mat_bytes(R.m, nrhs, R.ldy), "spmm y");
    for (int e = R.e0; e < R.e0 + R.ne; e++) {
      const SpEnt& E = ents.at(e);
      if (!E.A) {
        if (E.k != R.m) throw Error(IFMM_ERR_CUDA, "bounds check failed: identity entry size");
        Ranges::check(E.x, mat_bytes(R.m, nrhs, E.ldx), "spmm x (identity)");
        continue;
      }
      Ranges::check(E.A, E.transA ? mat_bytes(E.k, R.m, E.lda) : mat_bytes(R.m, E.k, E.lda),
                    "spmm A");
      Ranges::check(E.x, mat_bytes(E.k, nrhs, E.ldx), "spmm x");
    }
  }
}


// out[t + c ld_out] = in[perm[t] + c ld_in]   (gather: user -> tree order)
__global__ void k_gather_rows(const long long* __restrict__ perm, long long N,
                              const double* __restrict__ in, long long ldi,
                              double* __restrict__ out, long long ldo, int ncols) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const long long p = perm[t];
  for (int c = 0; c < ncols; c++) out[t + c * ldo] = in[p + c * ldi];
}

// out[perm[t] + c ld_out] = in[t + c ld_in]   (scatter: tree -> user order)
__global__ void k_scatter_rows(const long long* __restrict__ perm, long long N,
                               const double* __restrict__ in, long long ldi,
                               double* __restrict__ out, long long ldo, int ncols) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const long long p = perm[t];
  for (int c = 0; c < ncols; c++) out[p + c * ldo] = in[t + c * ldi];
}

__global__ void k_permute_points(const long long* __restrict__ perm, long long N, int dim,
                                 const double* __restrict__ in, double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const long long p = perm[t];
  for (int d = 0; d < dim; d++) out[t * dim + d] = in[p * dim + d];
}

void launch_permute_points(const long long* perm, long long N, int dim, const double* in,
                           double* out, cudaStream_t s) {
  if (N <= 0) return;
  k_permute_points<<<(int)((N + 255) / 256), 256, 0, s>>>(perm, N, dim, in, out);
  CK_LAUNCH("k_permute_points");
}

void launch_leaf_interp(ChebSpec c, int dim, const double* pts_tree, const LeafGeom* leaves,
                        int nleaves, double* U, cudaStream_t s) {
  if (nleaves <= 0) return;
  k_leaf_interp<<<nleaves, 256, 0, s>>>(c, dim, pts_tree, leaves, nleaves, U);
  CK_LAUNCH("k_leaf_interp");
}
void launch_transfer(ChebSpec c, int dim, double* T, cudaStream_t s) {
  k_transfer<<<1 << dim, 256, 0, s>>>(c, dim, T);
  CK_LAUNCH("k_transfer");
}
void launch_m2l_table(ChebSpec c, int dim, KSpec ks, double h, double* K, cudaStream_t s) {
  int no = 1;
  for (int d = 0; d < dim; d++) no *= 7;
  k_m2l_table<<<no, 256, 0, s>>>(c, dim, ks, h, K);
  CK_LAUNCH("k_m2l_table");
}
void launch_p2p_blocks(KSpec ks, int dim, const double* pts_tree, const P2PTask* tasks, int n,
                       double* S, cudaStream_t s) {
  if (n <= 0) return;
  k_p2p_blocks<<<n, 256, 0, s>>>(ks, dim, pts_tree, tasks, S);
  CK_LAUNCH("k_p2p_blocks");
}
void launch_direct(KSpec ks, int dim, const double* pts, long long N, const double* x,
                   long long ldx, double* y, long long ldy, int nrhs, cudaStream_t s) {
  const int blocks = (int)((N + 255) / 256);
  Prof p("k_direct", 2.0 * (double)N * N * nrhs, 0.0, s);
  for (int c = 0; c < nrhs; c++) {
    k_direct<<<blocks, 256, 0, s>>>(ks, dim, pts, N, x, ldx, y, ldy, c);
    CK_LAUNCH("k_direct");
  }
}
void launch_gather_rows(const long long* perm, long long N, const double* in, long long ldi,
                        double* out, long long ldo, int ncols, cudaStream_t s) {
  if (N <= 0) return;
  k_gather_rows<<<(int)((N + 255) / 256), 256, 0, s>>>(perm, N, in, ldi, out, ldo, ncols);
  CK_LAUNCH("k_gather_rows");
}
void launch_scatter_rows(const long long* perm, long long N, const double* in, long long ldi,
                         double* out, long long ldo, int ncols, cudaStream_t s) {
  if (N <= 0) return;
  k_scatter_rows<<<(int)((N + 255) / 256), 256, 0, s>>>(perm, N, in, ldi, out, ldo, ncols);
  CK_LAUNCH("k_scatter_rows");
}

}  // namespace ifmm
