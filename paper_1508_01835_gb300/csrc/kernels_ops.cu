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

// Block-row sparse product, one CTA per job (SpJob): 32 rows at a time, the
// 8 warps take interleaved columns of each non-transposed segment (coalesced
// 256-byte column pieces of A, one FMA per element); transposed segments go a
// row per warp with the lanes along the column.  Per-warp sums meet in shared
// memory in a fixed order.
constexpr int SPMM_WARPS = 8;

__device__ inline double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) k_spmm_job(const SpRow* __restrict__ rows,
                                                  const SpEnt* __restrict__ ents,
                                                  const SpJob* __restrict__ jobs,
                                                  const SpSeg* __restrict__ segs,
                                                  double* __restrict__ part, long long pld,
                                                  int c0, int nb) {
  const SpJob J = jobs[blockIdx.x];
  const SpRow R = rows[J.row];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ double sacc[SPMM_WARPS][33];
  __shared__ double sacc_t[32];
  for (int c = 0; c < nb; c++) {
    for (int rt = 0; rt < R.m; rt += 32) {
      const int r = rt + lane;
      const bool rin = r < R.m;
      if (threadIdx.x < 32) sacc_t[threadIdx.x] = 0.0;
      __syncthreads();
      double acc = 0.0;
      for (int si = J.s0; si < J.s0 + J.ns; si++) {
        const SpSeg G = segs[si];
        const SpEnt E = ents[G.ent];
        const double* x = E.x + (long long)(c0 + c) * E.ldx;
        if (!E.A) {  // identity: rows k0..k1 of this entry
          if (wid == 0 && rin && r >= G.k0 && r < G.k1) acc = fma(E.alpha, x[r], acc);
        } else if (!E.transA) {
          if (rin) {
            const double* a = E.A + r;
            double s0 = 0.0, s1 = 0.0;
            int col = G.k0 + wid;
            for (; col + SPMM_WARPS < G.k1; col += 2 * SPMM_WARPS) {
              s0 = fma(a[(long long)col * E.lda], x[col], s0);
              s1 = fma(a[(long long)(col + SPMM_WARPS) * E.lda], x[col + SPMM_WARPS], s1);
            }
            if (col < G.k1) s0 = fma(a[(long long)col * E.lda], x[col], s0);
            acc = fma(E.alpha, s0 + s1, acc);
          }
        } else {  // op(A) = A^T with A (k x m): output row r is column r of A
          const int rmax = min(32, R.m - rt);
          for (int rl = wid; rl < rmax; rl += SPMM_WARPS) {  // warp-uniform
            const double* a = E.A + (long long)(rt + rl) * E.lda;
            double d = 0.0;
            for (int col = G.k0 + lane; col < G.k1; col += 32) d = fma(a[col], x[col], d);
            d = warp_sum_d(d);
            if (lane == 0) sacc_t[rl] = fma(E.alpha, d, sacc_t[rl]);
          }
        }
      }
      sacc[wid][lane] = acc;
      __syncthreads();
      if (wid == 0 && rin) {
        double v = sacc_t[lane];
#pragma unroll
        for (int w = 0; w < SPMM_WARPS; w++) v += sacc[w][lane];
        if (J.part < 0) {
          double* y = R.y + (long long)(c0 + c) * R.ldy + r;
          *y = (R.beta == 0.0) ? v : fma(R.beta, *y, v);
        } else {
          part[J.part + r + (long long)c * pld] = v;
        }
      }
      __syncthreads();
    }
  }
}

// y = beta y + (sum of the row's partial sums, in job order)
__global__ void __launch_bounds__(256) k_spmm_reduce(const SpRow* __restrict__ rows,
                                                     const SpRed* __restrict__ reds,
                                                     const double* __restrict__ part,
                                                     long long pld, int c0, int nb) {
  const SpRed D = reds[blockIdx.x];
  const SpRow R = rows[D.row];
  // every thread takes (row, column) pairs: all threads busy for short rows
  for (int e = threadIdx.x; e < R.m * nb; e += blockDim.x) {
    const int r = e % R.m, c = e / R.m;
    const double* pp = part + D.base + r + (long long)c * pld;
    double v = 0.0;
    for (int j = 0; j < D.nj; j++) v += pp[(long long)j * R.m];
    double* y = R.y + (long long)(c0 + c) * R.ldy + r;
    *y = (R.beta == 0.0) ? v : fma(R.beta, *y, v);
  }
}

// Job split shared by the FP64 and FP32 products: about four jobs per SM, no
// job below 8192 multiply-adds per right-hand side; a row whose work exceeds
// the target is cut into up to 64 contiguous column ranges (partial sums).
template <class Row, class Ent>
static void split_jobs(const std::vector<Row>& rows, const std::vector<Ent>& ents, int nsm,
                       std::vector<SpJob>& jobs, std::vector<SpSeg>& segs,
                       std::vector<SpRed>& reds, long long& poff) {
  double total = 0.0;
  for (const Row& R : rows)
    for (int e = R.e0; e < R.e0 + R.ne; e++)
      total += (ents[e].A ? (double)R.m : 1.0) * ents[e].k;
  const double target = std::max(8192.0, total / (4.0 * nsm));
  poff = 0;
  for (int ri = 0; ri < (int)rows.size(); ri++) {
    const Row& R = rows[ri];
    long long K = 0;
    double work = 0.0;
    for (int e = R.e0; e < R.e0 + R.ne; e++) {
      K += ents[e].k;
      work += (ents[e].A ? (double)R.m : 1.0) * ents[e].k;
    }
    int ns = (int)std::ceil(work / target);
    if ((long long)ns > std::max(K, 1ll)) ns = (int)std::max(K, 1ll);
    ns = std::max(1, std::min(ns, 64));
    if (ns > 1) reds.push_back({ri, ns, poff});
    for (int j = 0; j < ns; j++) {
      const long long K0 = K * j / ns, K1 = K * (j + 1) / ns;
      SpJob J{ri, (int)segs.size(), 0, ns > 1 ? poff + (long long)j * R.m : -1};
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
    if (ns > 1) poff += (long long)ns * R.m;
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
    P.bytes += 8.0 * R.m;
    for (int e = R.e0; e < R.e0 + R.ne; e++) {
      const SpEnt& E = ents[e];
      P.flops += 2.0 * R.m * (double)E.k;
      P.bytes += 8.0 * E.k + (E.A ? 8.0 * R.m * (double)E.k : 0.0);
    }
  }
  std::vector<SpJob> jobs;
  std::vector<SpSeg> segs;
  std::vector<SpRed> reds;
  long long poff = 0;
  split_jobs(rows, ents, sm_count(), jobs, segs, reds, poff);
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
// FP32 block-row products for the reduced-precision substitution sweeps: the
// same job split, but every job serves all of its right-hand sides (up to 32
// per pass) from one read of its matrix entries.  The x columns of a chunk of
// 32 matrix columns are staged in shared memory; each warp walks a strided
// subset of the chunk's columns for 32 output rows and keeps NB partial sums
// per row in registers; the eight warps' sums are added through shared memory.
// ---------------------------------------------------------------------------
constexpr int F32_KCH = 32;

template <int NB>
__global__ void __launch_bounds__(256) k_spmm_f32(const SpRowF* __restrict__ rows,
                                                  const SpEntF* __restrict__ ents,
                                                  const SpJob* __restrict__ jobs,
                                                  const SpSeg* __restrict__ segs,
                                                  float* __restrict__ part, long long pld,
                                                  int c0, int nb) {
  const SpJob J = jobs[blockIdx.x];
  const SpRowF R = rows[J.row];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ __align__(16) float xs[F32_KCH][NB + 4];
  __shared__ float red[SPMM_WARPS][32][NB + 1];
  for (int rt = 0; rt < R.m; rt += 32) {
    const int r = rt + lane;
    const bool rin = r < R.m;
    float acc[NB];
#pragma unroll
    for (int c = 0; c < NB; c++) acc[c] = 0.0f;
    for (int si = J.s0; si < J.s0 + J.ns; si++) {
      const SpSeg G = segs[si];
      const SpEntF E = ents[G.ent];
      for (int kc0 = G.k0; kc0 < G.k1; kc0 += F32_KCH) {
        const int kk = min(F32_KCH, G.k1 - kc0);
        __syncthreads();  // the previous chunk has been read
        for (int e = threadIdx.x; e < kk * NB; e += blockDim.x) {
          const int col = e % kk, c = e / kk;
          xs[col][c] = c < nb ? E.x[kc0 + col + (long long)(c0 + c) * E.ldx] : 0.0f;
        }
        __syncthreads();
        if (!E.A) {  // identity: output row r takes x[r] (rows kc0 .. kc0 + kk)
          if (wid == 0 && rin && r >= kc0 && r < kc0 + kk) {
#pragma unroll
            for (int c = 0; c < NB; c++) acc[c] = fmaf(E.alpha, xs[r - kc0][c], acc[c]);
          }
        } else if (rin) {
          const float* a = E.A + r + (long long)kc0 * E.lda;
          for (int col = wid; col < kk; col += SPMM_WARPS) {
            const float av = E.alpha * a[(long long)col * E.lda];
            const float4* xv = reinterpret_cast<const float4*>(&xs[col][0]);
#pragma unroll
            for (int q = 0; q < NB / 4; q++) {
              const float4 v = xv[q];
              acc[4 * q + 0] = fmaf(av, v.x, acc[4 * q + 0]);
              acc[4 * q + 1] = fmaf(av, v.y, acc[4 * q + 1]);
              acc[4 * q + 2] = fmaf(av, v.z, acc[4 * q + 2]);
              acc[4 * q + 3] = fmaf(av, v.w, acc[4 * q + 3]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NB; c++) red[wid][lane][c] = acc[c];
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * nb; e += blockDim.x) {
      const int rl = e % 32, c = e / 32, row = rt + rl;
      if (row < R.m) {
        float v = 0.0f;
#pragma unroll
        for (int w = 0; w < SPMM_WARPS; w++) v += red[w][rl][c];
        if (J.part < 0) {
          float* y = R.y + (long long)(c0 + c) * R.ldy + row;
          *y = (R.beta == 0.0f) ? v : fmaf(R.beta, *y, v);
        } else {
          part[J.part + row + (long long)c * pld] = v;
        }
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_spmm_f32_reduce(const SpRowF* __restrict__ rows,
                                                         const SpRed* __restrict__ reds,
                                                         const float* __restrict__ part,
                                                         long long pld, int c0, int nb) {
  const SpRed D = reds[blockIdx.x];
  const SpRowF R = rows[D.row];
  for (int e = threadIdx.x; e < R.m * nb; e += blockDim.x) {
    const int r = e % R.m, c = e / R.m;
    const float* pp = part + D.base + r + (long long)c * pld;
    float v = 0.0f;
    for (int j = 0; j < D.nj; j++) v += pp[(long long)j * R.m];
    float* y = R.y + (long long)(c0 + c) * R.ldy + r;
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
    P.bytes += 4.0 * R.m;
    for (int e = R.e0; e < R.e0 + R.ne; e++) {
      const SpEntF& E = ents[e];
      if (E.A) Ranges::check(E.A, sizeof(float) * ((size_t)(E.k - 1) * E.lda + R.m), "spmm32 A");
      Ranges::check(E.x, sizeof(float) * ((size_t)(cap - 1) * E.ldx + E.k), "spmm32 x");
      P.flops += 2.0 * R.m * (double)E.k;
      P.bytes += 4.0 * E.k + (E.A ? 4.0 * R.m * (double)E.k : 0.0);
    }
  }
  std::vector<SpJob> jobs;
  std::vector<SpSeg> segs;
  std::vector<SpRed> reds;
  long long poff = 0;
  split_jobs(rows, ents, sm_count(), jobs, segs, reds, poff);
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
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int nb = std::min(32, nrhs - c0);
    {
      Prof pr("k_spmm_f32", p.flops * nb, p.bytes, s);
      if (nb <= 4)
        k_spmm_f32<4><<<p.njobs, 256, 0, s>>>(p.rows, p.ents, p.jobs, p.segs, p.part, p.part_ld, c0, nb);
      else if (nb <= 8)
        k_spmm_f32<8><<<p.njobs, 256, 0, s>>>(p.rows, p.ents, p.jobs, p.segs, p.part, p.part_ld, c0, nb);
      else if (nb <= 16)
        k_spmm_f32<16><<<p.njobs, 256, 0, s>>>(p.rows, p.ents, p.jobs, p.segs, p.part, p.part_ld, c0, nb);
      else
        k_spmm_f32<32><<<p.njobs, 256, 0, s>>>(p.rows, p.ents, p.jobs, p.segs, p.part, p.part_ld, c0, nb);
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
  for (int c0 = 0; c0 < nrhs; c0 += p.cap) {
    const int nb = std::min(p.cap, nrhs - c0);
    {
      Prof pr("k_spmm_job", p.flops * nb, p.bytes * nb, s);
      k_spmm_job<<<p.njobs, 256, 0, s>>>(p.rows, p.ents, p.jobs, p.segs, p.part, p.part_ld, c0,
                                         nb);
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
