// gmres.cu -- GMRES with the IFMM as preconditioner (Sec. 3.2: tolerance on
// ||b - A x|| / ||b||, at most maxit iterations, the black-box FMM for the
// products; Appendix B: the same with left preconditioning, where the
// tolerance applies to ||M^-1 (b - A x)|| / ||M^-1 b||).  Readings: x_0 = 0,
// classical Gram-Schmidt applied twice, Givens rotations; each right-hand
// side is an independent solve, all of them advance in lock step (finished
// columns are frozen).  Right preconditioning recomputes the true residual at
// the end; when rounding leaves it above tol although the Arnoldi estimate
// met tol, GMRES restarts from x (at most `refine` times, iterations counted
// in the same maxit).  Flexible GMRES (right preconditioning that keeps
// z_k = M^-1 v_k and forms x = Z y) is for a preconditioner applied in lower
// precision, which is not one fixed linear operator.
//
// Iterative refinement (mixed-precision GMRES-IR after Carson and Higham,
// 2018; an option, not in the paper): every cycle solves A d = r for the
// current FP64 residual r with GMRES whose products take the FMM's far field
// in FP32 (the near field stays FP64), to a relative reduction of
// IR_INNER_REDUCTION; then x += d and r = b - A x with the FP64 FMM.  The
// column converges when that true residual is <= tol ||b||; a cycle that does
// not halve any column's residual ends the refinement.
#include "factor.cuh"

namespace ifmm {

// The Krylov basis grows in chunks of KCH vectors, allocated as the iteration
// reaches them: basis vector j of right-hand side c is at
// Vtab[j / KCH] + c * N * KCH + (j % KCH) * N.
constexpr int KCH = 16;
__device__ __forceinline__ const double* basis(const double* const* Vtab, long long N, int c,
                                               int j) {
  return Vtab[j / KCH] + (long long)c * N * KCH + (long long)(j % KCH) * N;
}

// h[c * ldh + j] = sum_i V_c[i, j] w_c[i], j = 0..k
__global__ void k_basis_dots(const double* const* __restrict__ Vtab, long long N,
                             const double* __restrict__ w, long long ldw, int k,
                             double* __restrict__ h, int ldh) {
  const int j = blockIdx.x, c = blockIdx.y;
  if (j > k) return;
  const double* v = basis(Vtab, N, c, j);
  const double* x = w + c * ldw;
  double s = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) s += v[i] * x[i];
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int hh = blockDim.x / 2; hh > 0; hh >>= 1) {
    if (threadIdx.x < hh) sh[threadIdx.x] += sh[threadIdx.x + hh];
    __syncthreads();
  }
  if (threadIdx.x == 0) h[c * ldh + j] = sh[0];
}

// w_c -= sum_{j <= k} V_c[:, j] h[c, j]   (or x_c = sum_j V_c[:, j] y[c, j] when beta == 0)
__global__ void k_basis_combine(const double* const* __restrict__ Vtab, long long N,
                                double* __restrict__ w, long long ldw, const int* __restrict__ kc,
                                int k, const double* __restrict__ h, int ldh, double sign,
                                double beta) {
  const int c = blockIdx.y;
  const int kk = kc ? kc[c] - 1 : k;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j <= kk; j++) s += basis(Vtab, N, c, j)[i] * h[c * ldh + j];
    double* o = w + c * ldw + i;
    *o = (beta == 0.0) ? sign * s : beta * (*o) + sign * s;
  }
}

struct GState {
  double beta;   // norm of this cycle's starting residual (g_0)
  double ref;    // the stopping reference: ||b|| (right) or ||M^-1 b|| (left)
  double stop;   // this cycle stops the column once res <= stop
  double res;    // |g_{k+1}|
  int active;    // still iterating
  int iters;     // Arnoldi steps of this cycle
};

// Givens update of column k for every active column (one thread per column)
__global__ void k_givens(int ncols, int k, const double* __restrict__ h, int ldh,
                         const double* __restrict__ hn2, double* __restrict__ H, int ldH,
                         double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                         int ldg, double tol, GState* __restrict__ st, double* __restrict__ inv_hn) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  inv_hn[c] = 0.0;
  if (!st[c].active) return;
  const double hnc = sqrt(hn2[c]);
  double* col = H + (long long)c * ldH * (ldH - 1) + (long long)k * ldH;  // H_c[:, k]
  for (int j = 0; j <= k; j++) col[j] = h[c * ldh + j];
  col[k + 1] = hnc;
  double* csc = cs + (long long)c * ldg;
  double* snc = sn + (long long)c * ldg;
  double* gc = g + (long long)c * ldg;
  for (int j = 0; j < k; j++) {
    const double t = csc[j] * col[j] + snc[j] * col[j + 1];
    col[j + 1] = -snc[j] * col[j] + csc[j] * col[j + 1];
    col[j] = t;
  }
  const double den = hypot(col[k], col[k + 1]);
  csc[k] = den != 0.0 ? col[k] / den : 1.0;
  snc[k] = den != 0.0 ? col[k + 1] / den : 0.0;
  col[k] = den;
  col[k + 1] = 0.0;
  gc[k + 1] = -snc[k] * gc[k];
  gc[k] = csc[k] * gc[k];
  st[c].res = fabs(gc[k + 1]);
  st[c].iters = k + 1;
  if (hnc > 0.0) inv_hn[c] = 1.0 / hnc;
  if (st[c].res <= st[c].stop || hnc == 0.0) st[c].active = 0;
}

// y = H^-1 g (upper triangular, k_c x k_c) per column
__global__ void k_backsolve(int ncols, const double* __restrict__ H, int ldH,
                            const double* __restrict__ g, int ldg, const GState* __restrict__ st,
                            double* __restrict__ y, int* __restrict__ kc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const int k = st[c].iters;
  kc[c] = k;
  const double* Hc = H + (long long)c * ldH * (ldH - 1);
  double* yc = y + (long long)c * ldg;
  for (int i = k - 1; i >= 0; i--) {
    double s = g[(long long)c * ldg + i];
    for (int j = i + 1; j < k; j++) s -= Hc[i + (long long)j * ldH] * yc[j];
    yc[i] = s / Hc[i + (long long)i * ldH];
  }
}

// Start of a cycle: beta = |r_0|; on the first cycle the stopping reference is
// beta itself (||b|| or ||M^-1 b||), later cycles keep it.  A column already
// within tol of its reference does not iterate.  The cycle's stop is tol ref,
// or with iterative refinement (inner > 0) max(tol ref / 2, inner beta).
__global__ void k_init_state(int ncols, const double* __restrict__ bn2, GState* __restrict__ st,
                             double* __restrict__ g, int ldg, double* __restrict__ inv, int first,
                             double tol, double inner) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const double b = sqrt(bn2[c]);
  if (first) st[c].ref = b;
  st[c].beta = b;
  st[c].res = b;
  st[c].stop = inner > 0.0 ? fmax(0.5 * tol * st[c].ref, inner * b) : tol * st[c].ref;
  st[c].active = b > 0.0 && !(b <= tol * st[c].ref);
  st[c].iters = 0;
  g[(long long)c * ldg] = b;
  inv[c] = b > 0.0 ? 1.0 / b : 0.0;
}

static inline int gblocks(long long n) { return (int)std::min<long long>(1024, (n + 255) / 256); }

// Chunked Krylov basis (V, or the preconditioned vectors Z of flexible GMRES):
// chunks of KCH vectors are allocated as the iteration reaches them.
struct Basis {
  Arena& ar;
  long long N, ldV;
  int nrhs;
  cudaStream_t s;
  std::vector<double*> tab;
  double** d_tab;
  Basis(Arena& a, long long n, int k, int m, cudaStream_t st)
      : ar(a), N(n), ldV(n * KCH), nrhs(k), s(st), tab(m / KCH + 1, nullptr) {
    d_tab = ar.alloc<double*>(tab.size());
  }
  double* vec(int j) {
    const int ch = j / KCH;
    if (!tab[ch]) {
      tab[ch] = ar.alloc<double>((size_t)ldV * nrhs);
      CK(cudaMemcpyAsync(d_tab + ch, &tab[ch], sizeof(double*), cudaMemcpyHostToDevice, s));
    }
    return tab[ch] + (long long)(j % KCH) * N;
  }
};

ifmm_status gmres_run(ifmm_system* sys, ifmm_factorization* fac, int mode, const double* b,
                      double* x, int nrhs, long long ld, double tol, int maxit,
                      ifmm_gmres_report* rep, cudaStream_t s, Arena* workspace,
                      const GmresOpts& opt) {
  if (opt.block && nrhs > 1) {
    GmresOpts bo = opt;
    bo.block = 0;  // the per-column finish of block GMRES
    return block_gmres_run(sys, fac, mode, b, x, nrhs, ld, tol, maxit, rep, s, bo);
  }
  const long long N = sys->N;
  const int m = maxit;
  const int side = fac ? opt.side : IFMM_GMRES_RIGHT;  // no preconditioner: plain GMRES
  if (fac && opt.precond_fp32 && side != IFMM_GMRES_FLEXIBLE)
    throw Error(IFMM_ERR_INVALID_ARG, "FP32 substitution sweeps need flexible GMRES");
  const bool ir = opt.mv_fp32 != 0;
  if (ir && (mode != IFMM_MV_FMM || side == IFMM_GMRES_LEFT))
    throw Error(IFMM_ERR_INVALID_ARG,
                "iterative refinement takes the FMM matvec and right or flexible GMRES");
  // Arnoldi products: FP64, or with iterative refinement the FP32 far field
  auto amv = [&](const double* in, long long ldi, double* out, long long ldo) {
    if (ir) system_matvec_f32far(sys, in, ldi, out, ldo, nrhs, s);
    else system_matvec(sys, mode, in, ldi, out, ldo, nrhs, s);
  };
  // workspace: the caller's arena, rewound and reused across calls (no device
  // allocation once it has grown, so no implicit device-wide synchronisation
  // of cudaMalloc / cudaFree between concurrent solves), or a private one
  Arena own;
  own.chunk_bytes = size_t(64) << 20;
  Arena& ar = workspace ? *workspace : own;
  ar.reset();
  Basis V(ar, N, nrhs, m, s);
  std::unique_ptr<Basis> Zb;
  if (side == IFMM_GMRES_FLEXIBLE) Zb.reset(new Basis(ar, N, nrhs, m, s));
  const long long ldV = V.ldV;
  double* Z = ar.alloc<double>((size_t)N * nrhs);
  double* Wv = ar.alloc<double>((size_t)N * nrhs);
  double* R = ar.alloc<double>((size_t)N * nrhs);
  const int ldH = m + 1;
  double* H = ar.alloc<double>((size_t)ldH * m * nrhs + 1);
  double* cs = ar.alloc<double>((size_t)(m + 1) * nrhs);
  double* sn = ar.alloc<double>((size_t)(m + 1) * nrhs);
  double* g = ar.alloc<double>((size_t)(m + 1) * nrhs);
  double* y = ar.alloc<double>((size_t)(m + 1) * nrhs);
  double* h = ar.alloc<double>((size_t)(m + 1) * nrhs);
  double* h2 = ar.alloc<double>((size_t)(m + 1) * nrhs);
  double* hn = ar.alloc<double>(nrhs);
  double* inv = ar.alloc<double>(nrhs);
  double* part = ar.alloc<double>((size_t)256 * nrhs);
  int* kc = ar.alloc<int>(nrhs);
  GState* st = ar.alloc<GState>(nrhs);
  auto precond = [&](const double* in, long long ldi, double* out, long long ldo) {
    if (opt.precond_fp32) factor_solve_f32(fac, in, ldi, out, ldo, nrhs, s);  // out ~ M^-1 in
    else factor_solve(fac, in, ldi, out, ldo, nrhs, s);                       // out = M^-1 in
  };
  std::vector<GState> hs(nrhs);
  std::vector<int> total(nrhs, 0);
  std::vector<double> rn(nrhs), prev_t(nrhs, 1.0), bn(nrhs);
  int used = 0;  // Arnoldi steps so far (all cycles)
  const int cycles = 1 + std::max(0, opt.refine);
  for (int cyc = 0; cyc < cycles && used < m; cyc++) {
    const bool first = cyc == 0;
    const int mc = m - used;  // steps left for this cycle
    CK(cudaMemsetAsync(g, 0, sizeof(double) * (m + 1) * nrhs, s));
    CK(cudaMemsetAsync(H, 0, sizeof(double) * ((size_t)ldH * m * nrhs + 1), s));
    // r_0: b (first cycle, x_0 = 0) or b - A x, which the previous cycle left
    // in R; left preconditioning applies M^-1
    const double* r0 = first ? b : R;
    long long ldr = first ? ld : N;
    if (side == IFMM_GMRES_LEFT) {
      precond(r0, ldr, Z, N);
      r0 = Z;
      ldr = N;
    }
    launch_dots(r0, ldr, r0, ldr, N, nrhs, hn, part, s);
    k_init_state<<<(nrhs + 63) / 64, 64, 0, s>>>(nrhs, hn, st, g, m + 1, inv, first ? 1 : 0, tol,
                                                  ir ? IR_INNER_REDUCTION : 0.0);
    CK_LAUNCH("k_init_state");
    launch_axpby(N, nrhs, inv, 1.0, r0, ldr, 0.0, V.vec(0), ldV, s);
    CK(cudaMemcpyAsync(hs.data(), st, nrhs * sizeof(GState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool any = false;
    for (auto& q : hs) any |= q.active != 0;
    int k = 0;
    for (k = 0; any && k < mc; k++) {
      double* vk = V.vec(k);
      if (side == IFMM_GMRES_RIGHT) {  // w = A M^-1 v_k
        if (fac) precond(vk, ldV, Z, N);
        else launch_axpby(N, nrhs, nullptr, 1.0, vk, ldV, 0.0, Z, N, s);
        amv(Z, N, Wv, N);
      } else if (side == IFMM_GMRES_FLEXIBLE) {  // z_k = M^-1 v_k kept, w = A z_k
        double* zk = Zb->vec(k);
        precond(vk, ldV, zk, ldV);
        amv(zk, ldV, Wv, N);
      } else {  // left: w = M^-1 A v_k
        system_matvec(sys, mode, vk, ldV, Z, N, nrhs, s);
        precond(Z, N, Wv, N);
      }
      // CGS2
      const double* const* Vt = V.d_tab;
      k_basis_dots<<<dim3(k + 1, nrhs), 256, 0, s>>>(Vt, N, Wv, N, k, h, m + 1);
      CK_LAUNCH("k_basis_dots");
      k_basis_combine<<<dim3(gblocks(N), nrhs), 256, 0, s>>>(Vt, N, Wv, N, nullptr, k, h, m + 1,
                                                             -1.0, 1.0);
      CK_LAUNCH("k_basis_combine");
      k_basis_dots<<<dim3(k + 1, nrhs), 256, 0, s>>>(Vt, N, Wv, N, k, h2, m + 1);
      CK_LAUNCH("k_basis_dots");
      k_basis_combine<<<dim3(gblocks(N), nrhs), 256, 0, s>>>(Vt, N, Wv, N, nullptr, k, h2,
                                                             m + 1, -1.0, 1.0);
      CK_LAUNCH("k_basis_combine");
      launch_axpby((long long)(k + 1), nrhs, nullptr, 1.0, h2, m + 1, 1.0, h, m + 1, s);
      launch_dots(Wv, N, Wv, N, N, nrhs, hn, part, s);  // ||w||^2
      k_givens<<<(nrhs + 63) / 64, 64, 0, s>>>(nrhs, k, h, m + 1, hn, H, ldH, cs, sn, g, m + 1,
                                               tol, st, inv);
      CK_LAUNCH("k_givens");
      if (k + 1 < mc) launch_axpby(N, nrhs, inv, 1.0, Wv, N, 0.0, V.vec(k + 1), ldV, s);
      CK(cudaMemcpyAsync(hs.data(), st, nrhs * sizeof(GState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      any = false;
      for (auto& q : hs) any |= q.active != 0;
    }
    used += k;
    for (int c = 0; c < nrhs; c++) total[c] += hs[c].iters;
    // update u = M^-1 (V y) (right), Z y (flexible) or V y (left); x = u or x + u
    k_backsolve<<<(nrhs + 63) / 64, 64, 0, s>>>(nrhs, H, ldH, g, m + 1, st, y, kc);
    CK_LAUNCH("k_backsolve");
    const double xb = first ? 0.0 : 1.0;
    if (side == IFMM_GMRES_FLEXIBLE) {
      k_basis_combine<<<dim3(gblocks(N), nrhs), 256, 0, s>>>(Zb->d_tab, N, x, ld, kc, 0, y, m + 1,
                                                             1.0, xb);
      CK_LAUNCH("k_basis_combine");
    } else if (side == IFMM_GMRES_LEFT) {
      k_basis_combine<<<dim3(gblocks(N), nrhs), 256, 0, s>>>(V.d_tab, N, x, ld, kc, 0, y, m + 1,
                                                             1.0, xb);
      CK_LAUNCH("k_basis_combine");
    } else {
      k_basis_combine<<<dim3(gblocks(N), nrhs), 256, 0, s>>>(V.d_tab, N, Z, N, kc, 0, y, m + 1,
                                                             1.0, 0.0);
      CK_LAUNCH("k_basis_combine");
      if (fac) precond(Z, N, Wv, N);
      else launch_axpby(N, nrhs, nullptr, 1.0, Z, N, 0.0, Wv, N, s);
      launch_axpby(N, nrhs, nullptr, 1.0, Wv, N, xb, x, ld, s);
    }
    // true residual R = b - A x (FP64; the next cycle starts from it)
    system_matvec(sys, mode, x, ld, Wv, N, nrhs, s);
    launch_axpby(N, nrhs, nullptr, 1.0, b, ld, 0.0, R, N, s);
    launch_axpby(N, nrhs, nullptr, -1.0, Wv, N, 1.0, R, N, s);
    launch_dots(R, N, R, N, N, nrhs, hn, part, s);
    CK(cudaMemcpyAsync(rn.data(), hn, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (first) {
      launch_dots(b, ld, b, ld, N, nrhs, hn, part, s);
      CK(cudaMemcpyAsync(bn.data(), hn, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaMemcpyAsync(hs.data(), st, nrhs * sizeof(GState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // refinement: another cycle from x while a column's recomputed residual is
    // above tol although its Arnoldi estimate met it (right and flexible GMRES;
    // left GMRES stops on the preconditioned residual, as the paper states it);
    // with iterative refinement while a column is above tol and some column's
    // residual at least halved in this cycle
    bool again = false, progress = false;
    for (int c = 0; c < nrhs; c++) {
      const double t = bn[c] > 0 ? std::sqrt(rn[c] / bn[c]) : 0.0;
      rep[c].iters = total[c];
      rep[c].rel_residual = hs[c].ref > 0 ? hs[c].res / hs[c].ref : 0.0;
      rep[c].true_rel_residual = t;
      const bool est_ok = hs[c].ref == 0.0 || hs[c].res <= tol * hs[c].ref;
      if (ir) {
        if (t > tol) again = true;
        if (t <= 0.5 * prev_t[c]) progress = true;
      } else if (side != IFMM_GMRES_LEFT && est_ok && t > tol) {
        again = true;
      }
      prev_t[c] = t;
    }
    if (!again || (ir && !progress)) break;
  }
  ifmm_status out = IFMM_OK;
  for (int c = 0; c < nrhs; c++) {
    const bool est_ok = hs[c].ref == 0.0 || hs[c].res <= tol * hs[c].ref;
    const bool conv = ir ? rep[c].true_rel_residual <= tol
                         : side == IFMM_GMRES_LEFT ? est_ok
                                                   : (est_ok && rep[c].true_rel_residual <= tol);
    rep[c].status = conv ? IFMM_OK : IFMM_ERR_NOT_CONVERGED;
    if (!conv) out = IFMM_ERR_NOT_CONVERGED;
  }
  return out;
}


// ---------------------------------------------------------------------------
// Block GMRES over the nrhs columns (one Krylov space shared by all right-hand
// sides; right or flexible preconditioning): block Arnoldi with block CGS2 and
// Cholesky QR (applied twice) of each new block, the block Hessenberg reduced
// by Givens rotations on the host (it is at most a few thousand entries
// wide), x = M^-1 V Y (right) or Z Y (flexible).  A column's residual is the
// norm of its part of the rotated right-hand side below the triangle.  If a
// new block loses rank (Cholesky breaks down, e.g. after some columns have
// converged) the block iteration stops and the columns still above tol finish
// with the per-column GMRES from the current x.
// ---------------------------------------------------------------------------
__global__ void k_sum_parts(const double* __restrict__ part, int nparts, long long n,
                            double* __restrict__ out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nparts; c++) s += part[(long long)c * n + e];
    out[e] = s;
  }
}

// D (m x k, ld m) = X^T Y, X: N x m (ld ldx), Y: N x k (ld ldy); split over
// row chunks of N, partial products summed in chunk order (deterministic)
static void gram(Arena& ar, const double* X, long long ldx, int m, const double* Y, long long ldy,
                 int k, long long N, double* D, cudaStream_t s) {
  const long long chunk = std::max<long long>(2048, (N + 63) / 64);
  const int nparts = (int)((N + chunk - 1) / chunk);
  double* part = ar.alloc<double>((size_t)nparts * m * k);
  std::vector<GemmTask> g;
  for (int c = 0; c < nparts; c++) {
    const long long r0 = (long long)c * chunk, r1 = std::min(N, r0 + chunk);
    g.push_back(GemmTask{X + r0, Y + r0, part + (size_t)c * m * k, (int)ldx, (int)ldy, m, m, k,
                         (int)(r1 - r0), 1, 0, 1.0, 0.0});
  }
  run_gemms(ar, g, s);
  const long long n = (long long)m * k;
  k_sum_parts<<<(int)std::min<long long>(1024, (n + 255) / 256), 256, 0, s>>>(part, nparts, n, D);
  CK_LAUNCH("k_sum_parts");
}

// Cholesky G = R^T R (k x k, column-major); false if not positive definite
static bool chol_upper(const std::vector<double>& G, int k, std::vector<double>& R) {
  R.assign((size_t)k * k, 0.0);
  for (int j = 0; j < k; j++) {
    double d = G[j + (size_t)j * k];
    for (int i = 0; i < j; i++) d -= R[i + (size_t)j * k] * R[i + (size_t)j * k];
    if (!(d > 1e-300)) return false;
    const double rjj = std::sqrt(d);
    R[j + (size_t)j * k] = rjj;
    for (int c = j + 1; c < k; c++) {
      double v = G[j + (size_t)c * k];
      for (int i = 0; i < j; i++) v -= R[i + (size_t)j * k] * R[i + (size_t)c * k];
      R[j + (size_t)c * k] = v / rjj;
    }
  }
  return true;
}

static std::vector<double> inv_upper(const std::vector<double>& R, int k) {
  std::vector<double> X((size_t)k * k, 0.0);
  for (int c = 0; c < k; c++) {  // solve R x = e_c
    for (int i = c; i >= 0; i--) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int j = i + 1; j <= c; j++) v -= R[i + (size_t)j * k] * X[j + (size_t)c * k];
      X[i + (size_t)c * k] = v / R[i + (size_t)i * k];
    }
  }
  return X;
}

ifmm_status block_gmres_run(ifmm_system* sys, ifmm_factorization* fac, int mode, const double* b,
                            double* x, int k, long long ld, double tol, int maxit,
                            ifmm_gmres_report* rep, cudaStream_t s, const GmresOpts& opt) {
  const long long N = sys->N;
  const bool flex = fac && opt.side == IFMM_GMRES_FLEXIBLE;
  if (fac && opt.side == IFMM_GMRES_LEFT)
    throw Error(IFMM_ERR_INVALID_ARG, "block GMRES takes right or flexible preconditioning");
  const int m = maxit;  // block steps
  Arena ar;
  ar.chunk_bytes = size_t(64) << 20;
  Arena scratch;
  double* V = ar.alloc<double>((size_t)N * (m + 1) * k);      // basis blocks, ld N
  double* Zall = flex ? ar.alloc<double>((size_t)N * m * k) : nullptr;
  double* Zt = ar.alloc<double>((size_t)N * k);
  double* W = ar.alloc<double>((size_t)N * k);
  double* D = ar.alloc<double>((size_t)(m + 1) * k * k);
  double* D2 = ar.alloc<double>((size_t)(m + 1) * k * k);
  double* Gk = ar.alloc<double>((size_t)k * k);
  double* Ri = ar.alloc<double>((size_t)k * k);
  auto precond = [&](const double* in, long long ldi, double* out, long long ldo) {
    if (!fac) launch_axpby(N, k, nullptr, 1.0, in, ldi, 0.0, out, ldo, s);
    else if (opt.precond_fp32) factor_solve_f32(fac, in, ldi, out, ldo, k, s);
    else factor_solve(fac, in, ldi, out, ldo, k, s);
  };
  // column norms of b (stopping references)
  std::vector<double> bn(k);
  {
    double* hn = scratch.alloc<double>(k);
    double* part = scratch.alloc<double>((size_t)256 * k);
    launch_dots(b, ld, b, ld, N, k, hn, part, s);
    CK(cudaMemcpyAsync(bn.data(), hn, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (auto& v : bn) v = std::sqrt(v);
  }
  // Cholesky QR twice of the block at W into V_j, returning R (k x k) = R2 R1
  auto cholqr2 = [&](double* Vj, std::vector<double>& Rtot) -> bool {
    std::vector<double> R1, R2, Gh((size_t)k * k);
    for (int pass = 0; pass < 2; pass++) {
      scratch.reset();
      gram(scratch, W, N, k, W, N, k, N, Gk, s);
      CK(cudaMemcpyAsync(Gh.data(), Gk, sizeof(double) * k * k, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      std::vector<double>& R = pass == 0 ? R1 : R2;
      if (!chol_upper(Gh, k, R)) return false;
      std::vector<double> Rinv = inv_upper(R, k);
      CK(cudaMemcpyAsync(Ri, Rinv.data(), sizeof(double) * k * k, cudaMemcpyHostToDevice, s));
      double* dst = pass == 0 ? Zt : Vj;  // W R1^-1 -> Zt -> (copy back) ; second pass -> V_j
      run_gemms(scratch, {GemmTask{W, Ri, dst, (int)N, k, (int)N, (int)N, k, k, 0, 0, 1.0, 0.0}}, s);
      if (pass == 0) launch_axpby(N, k, nullptr, 1.0, Zt, N, 0.0, W, N, s);
      CK(cudaStreamSynchronize(s));
    }
    Rtot.assign((size_t)k * k, 0.0);  // R2 R1
    for (int c = 0; c < k; c++)
      for (int r = 0; r <= c; r++) {
        double v = 0.0;
        for (int q = r; q <= c; q++) v += R2[r + (size_t)q * k] * R1[q + (size_t)c * k];
        Rtot[r + (size_t)c * k] = v;
      }
    return true;
  };
  // host state of the least-squares problem: rotated block Hessenberg columns
  const int rows = (m + 1) * k;
  std::vector<double> Hh((size_t)rows * m * k, 0.0);  // column-major, ld rows
  std::vector<double> G((size_t)rows * k, 0.0);       // rotated right-hand side
  struct Rot { int r; double c, s; };
  std::vector<Rot> rots;
  std::vector<int> first_ok(k, -1);
  // V_0 S_0 = b
  launch_axpby(N, k, nullptr, 1.0, b, ld, 0.0, W, N, s);
  std::vector<double> S0;
  if (!cholqr2(V, S0)) throw Error(IFMM_ERR_INVALID_ARG, "block GMRES: the right-hand sides are linearly dependent");
  for (int c = 0; c < k; c++)
    for (int r = 0; r <= c; r++) G[r + (size_t)c * rows] = S0[r + (size_t)c * k];
  int steps = 0;
  bool broke = false;
  for (int j = 0; j < m; j++) {
    double* Vj = V + (size_t)j * k * N;
    double* Zj = flex ? Zall + (size_t)j * k * N : Zt;
    precond(Vj, N, Zj, N);
    system_matvec(sys, mode, Zj, N, W, N, k, s);
    // block CGS2 against V_0 .. V_j
    const int mj = (j + 1) * k;
    scratch.reset();
    gram(scratch, V, N, mj, W, N, k, N, D, s);
    run_gemms(scratch, {GemmTask{V, D, W, (int)N, mj, (int)N, (int)N, k, mj, 0, 0, -1.0, 1.0}}, s);
    gram(scratch, V, N, mj, W, N, k, N, D2, s);
    run_gemms(scratch, {GemmTask{V, D2, W, (int)N, mj, (int)N, (int)N, k, mj, 0, 0, -1.0, 1.0}}, s);
    std::vector<double> h1((size_t)mj * k), h2((size_t)mj * k);
    CK(cudaMemcpyAsync(h1.data(), D, sizeof(double) * mj * k, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h2.data(), D2, sizeof(double) * mj * k, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<double> Rn;
    const bool ok = cholqr2(V + (size_t)(j + 1) * k * N, Rn);
    // new block column of H: [h1 + h2 ; R_{j+1,j}]
    for (int c = 0; c < k; c++) {
      double* col = Hh.data() + (size_t)(j * k + c) * rows;
      for (int r = 0; r < mj; r++) col[r] = h1[r + (size_t)c * mj] + h2[r + (size_t)c * mj];
      for (int r = 0; r < k; r++) col[mj + r] = ok ? Rn[r + (size_t)c * k] : 0.0;
    }
    // apply the earlier blocks' rotations (in creation order) to the whole new
    // block column, then zero its subdiagonal entries column by column
    for (int c = 0; c < k; c++) {
      double* col = Hh.data() + (size_t)(j * k + c) * rows;
      for (const Rot& q : rots) {
        const double a = col[q.r], bb = col[q.r + 1];
        col[q.r] = q.c * a + q.s * bb;
        col[q.r + 1] = -q.s * a + q.c * bb;
      }
    }
    for (int c = 0; c < k; c++) {
      double* col = Hh.data() + (size_t)(j * k + c) * rows;
      const int dg = j * k + c;  // diagonal row of this column
      for (int r = mj + c; r > dg; r--) {
        const double a = col[r - 1], bb = col[r];
        const double den = std::hypot(a, bb);
        const double cc = den != 0.0 ? a / den : 1.0, ss = den != 0.0 ? bb / den : 0.0;
        col[r - 1] = den;
        col[r] = 0.0;
        rots.push_back({r - 1, cc, ss});
        for (int q = 0; q < k; q++) {
          double* g = G.data() + (size_t)q * rows;
          const double ga = g[r - 1], gb = g[r];
          g[r - 1] = cc * ga + ss * gb;
          g[r] = -ss * ga + cc * gb;
        }
        // the rotation also acts on the later columns of this block
        for (int c2 = c + 1; c2 < k; c2++) {
          double* o = Hh.data() + (size_t)(j * k + c2) * rows;
          const double oa = o[r - 1], ob = o[r];
          o[r - 1] = cc * oa + ss * ob;
          o[r] = -ss * oa + cc * ob;
        }
      }
    }
    steps = j + 1;
    // residuals of the columns: their parts of G below row (j + 1) k
    bool all = true;
    for (int q = 0; q < k; q++) {
      double rr = 0.0;
      for (int r = (j + 1) * k; r < (j + 2) * k; r++) rr += G[r + (size_t)q * rows] * G[r + (size_t)q * rows];
      const double res = std::sqrt(rr);
      rep[q].rel_residual = bn[q] > 0 ? res / bn[q] : 0.0;
      if (bn[q] == 0.0 || res <= tol * bn[q]) {
        if (first_ok[q] < 0) first_ok[q] = steps;
      } else {
        all = false;
      }
    }
    if (all) break;
    if (!ok) { broke = true; break; }
  }
  // rotations above were applied within each block column as the zeros were
  // made, so Hh[0:n, 0:n] is upper triangular; Y = H^-1 G[0:n, :]
  const int n = steps * k;
  std::vector<double> Y((size_t)n * k, 0.0);
  for (int q = 0; q < k; q++)
    for (int i = n - 1; i >= 0; i--) {
      double v = G[i + (size_t)q * rows];
      for (int c = i + 1; c < n; c++) v -= Hh[i + (size_t)c * rows] * Y[c + (size_t)q * n];
      const double d = Hh[i + (size_t)i * rows];
      Y[i + (size_t)q * n] = d != 0.0 ? v / d : 0.0;
    }
  double* Yd = scratch.alloc<double>((size_t)n * k);
  CK(cudaMemcpyAsync(Yd, Y.data(), sizeof(double) * n * k, cudaMemcpyHostToDevice, s));
  if (flex) {
    run_gemms(scratch, {GemmTask{Zall, Yd, x, (int)N, n, (int)ld, (int)N, k, n, 0, 0, 1.0, 0.0}}, s);
  } else {
    run_gemms(scratch, {GemmTask{V, Yd, W, (int)N, n, (int)N, (int)N, k, n, 0, 0, 1.0, 0.0}}, s);
    precond(W, N, x, ld);
  }
  CK(cudaStreamSynchronize(s));
  // true residuals; columns still above tol finish with per-column GMRES from x
  double* R = W;
  system_matvec(sys, mode, x, ld, R, N, k, s);
  launch_axpby(N, k, nullptr, 1.0, b, ld, -1.0, R, N, s);
  std::vector<double> rn(k);
  {
    double* hn = scratch.alloc<double>(k);
    double* part = scratch.alloc<double>((size_t)256 * k);
    launch_dots(R, N, R, N, N, k, hn, part, s);
    CK(cudaMemcpyAsync(rn.data(), hn, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  ifmm_status out = IFMM_OK;
  bool finish = false;
  for (int q = 0; q < k; q++) {
    rep[q].iters = first_ok[q] > 0 ? first_ok[q] : steps;
    rep[q].true_rel_residual = bn[q] > 0 ? std::sqrt(rn[q]) / bn[q] : 0.0;
    if (rep[q].true_rel_residual > tol) finish = true;
  }
  if (finish && steps < m && opt.refine > 0) {
    // dx from the residual R (= b - A x), one column group, per-column GMRES
    std::vector<ifmm_gmres_report> r2(k);
    GmresOpts o2 = opt;
    o2.side = flex ? IFMM_GMRES_FLEXIBLE : IFMM_GMRES_RIGHT;
    double* dx = Zt;
    gmres_run(sys, fac, mode, R, dx, k, N, tol * 0.999, m - steps, r2.data(), s, nullptr, o2);
    (void)broke;
    launch_axpby(N, k, nullptr, 1.0, dx, N, 1.0, x, ld, s);
    system_matvec(sys, mode, x, ld, R, N, k, s);
    launch_axpby(N, k, nullptr, 1.0, b, ld, -1.0, R, N, s);
    double* hn = scratch.alloc<double>(k);
    double* part = scratch.alloc<double>((size_t)256 * k);
    launch_dots(R, N, R, N, N, k, hn, part, s);
    CK(cudaMemcpyAsync(rn.data(), hn, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int q = 0; q < k; q++) {
      rep[q].iters += r2[q].iters;
      rep[q].true_rel_residual = bn[q] > 0 ? std::sqrt(rn[q]) / bn[q] : 0.0;
    }
  }
  for (int q = 0; q < k; q++) {
    const bool conv = rep[q].true_rel_residual <= tol;
    rep[q].status = conv ? IFMM_OK : IFMM_ERR_NOT_CONVERGED;
    if (!conv) out = IFMM_ERR_NOT_CONVERGED;
  }
  return out;
}

}  // namespace ifmm
