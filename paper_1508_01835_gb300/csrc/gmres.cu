// gmres.cu -- non-restarted GMRES with the IFMM as right preconditioner
// (Sec. 3.2: tolerance on ||b - A x|| / ||b||, at most maxit iterations, the
// black-box FMM for the products).  Readings: x_0 = 0, classical Gram-Schmidt
// applied twice, Givens rotations; each right-hand side is an independent
// solve, all of them advance in lock step (finished columns are frozen).
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
  double beta;   // ||b||
  double res;    // |g_{k+1}|
  int active;    // still iterating
  int iters;
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
  if (st[c].res <= tol * st[c].beta || hnc == 0.0) st[c].active = 0;
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

__global__ void k_init_state(int ncols, const double* __restrict__ bn2, GState* __restrict__ st,
                             double* __restrict__ g, int ldg, double* __restrict__ inv) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const double b = sqrt(bn2[c]);
  st[c].beta = b;
  st[c].res = b;
  st[c].active = b > 0.0;
  st[c].iters = 0;
  g[(long long)c * ldg] = b;
  inv[c] = b > 0.0 ? 1.0 / b : 0.0;
}

static inline int gblocks(long long n) { return (int)std::min<long long>(1024, (n + 255) / 256); }

ifmm_status gmres_run(ifmm_system* sys, ifmm_factorization* fac, int mode, const double* b,
                      double* x, int nrhs, long long ld, double tol, int maxit,
                      ifmm_gmres_report* rep, cudaStream_t s, Arena* workspace) {
  const long long N = sys->N;
  const int m = maxit;
  // workspace: the caller's arena, rewound and reused across calls (no device
  // allocation once it has grown, so no implicit device-wide synchronisation
  // of cudaMalloc / cudaFree between concurrent solves), or a private one
  Arena own;
  own.chunk_bytes = size_t(64) << 20;
  Arena& ar = workspace ? *workspace : own;
  ar.reset();
  // Krylov basis: chunks of KCH vectors (ld N * KCH between right-hand sides)
  const long long ldV = N * KCH;
  const int nchunks = m / KCH + 1;
  std::vector<double*> vtab(nchunks, nullptr);
  double** d_vtab = ar.alloc<double*>(nchunks);
  auto vec = [&](int j) -> double* {  // basis vector j (allocating its chunk)
    const int ch = j / KCH;
    if (!vtab[ch]) {
      vtab[ch] = ar.alloc<double>((size_t)ldV * nrhs);
      CK(cudaMemcpyAsync(d_vtab + ch, &vtab[ch], sizeof(double*), cudaMemcpyHostToDevice, s));
    }
    return vtab[ch] + (long long)(j % KCH) * N;
  };
  const double* const* Vt = d_vtab;
  double* Z = ar.alloc<double>((size_t)N * nrhs);
  double* Wv = ar.alloc<double>((size_t)N * nrhs);
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
  CK(cudaMemsetAsync(g, 0, sizeof(double) * (m + 1) * nrhs, s));
  CK(cudaMemsetAsync(H, 0, sizeof(double) * ((size_t)ldH * m * nrhs + 1), s));
  // beta = ||b||, v_0 = b / beta
  launch_dots(b, ld, b, ld, N, nrhs, hn, part, s);
  k_init_state<<<(nrhs + 63) / 64, 64, 0, s>>>(nrhs, hn, st, g, m + 1, inv);
  CK_LAUNCH("k_init_state");
  launch_axpby(N, nrhs, inv, 1.0, b, ld, 0.0, vec(0), ldV, s);
  std::vector<GState> hs(nrhs);
  int k = 0;
  for (k = 0; k < m; k++) {
    double* vk = vec(k);
    if (fac) factor_solve(fac, vk, ldV, Z, N, nrhs, s);  // Z = M^-1 v_k
    else launch_axpby(N, nrhs, nullptr, 1.0, vk, ldV, 0.0, Z, N, s);
    system_matvec(sys, mode, Z, N, Wv, N, nrhs, s);
    // CGS2
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
    k_givens<<<(nrhs + 63) / 64, 64, 0, s>>>(nrhs, k, h, m + 1, hn, H, ldH, cs, sn, g, m + 1, tol,
                                             st, inv);
    CK_LAUNCH("k_givens");
    if (k + 1 < m + 1)
      launch_axpby(N, nrhs, inv, 1.0, Wv, N, 0.0, vec(k + 1), ldV, s);
    CK(cudaMemcpyAsync(hs.data(), st, nrhs * sizeof(GState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool any = false;
    for (auto& q : hs) any |= q.active != 0;
    if (!any) break;
  }
  // x = M^-1 (V y)
  k_backsolve<<<(nrhs + 63) / 64, 64, 0, s>>>(nrhs, H, ldH, g, m + 1, st, y, kc);
  CK_LAUNCH("k_backsolve");
  k_basis_combine<<<dim3(gblocks(N), nrhs), 256, 0, s>>>(Vt, N, Z, N, kc, 0, y, m + 1, 1.0,
                                                         0.0);
  CK_LAUNCH("k_basis_combine");
  if (fac) factor_solve(fac, Z, N, x, ld, nrhs, s);
  else launch_axpby(N, nrhs, nullptr, 1.0, Z, N, 0.0, x, ld, s);
  // true residual ||b - A x|| / ||b||
  system_matvec(sys, mode, x, ld, Wv, N, nrhs, s);
  launch_axpby(N, nrhs, nullptr, 1.0, b, ld, -1.0, Wv, N, s);
  launch_dots(Wv, N, Wv, N, N, nrhs, hn, part, s);
  std::vector<double> rn(nrhs);
  CK(cudaMemcpyAsync(rn.data(), hn, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hs.data(), st, nrhs * sizeof(GState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  ifmm_status out = IFMM_OK;
  for (int c = 0; c < nrhs; c++) {
    const double bb = hs[c].beta;
    rep[c].iters = hs[c].iters;
    rep[c].rel_residual = bb > 0 ? hs[c].res / bb : 0.0;
    rep[c].true_rel_residual = bb > 0 ? std::sqrt(rn[c]) / bb : 0.0;
    const bool conv = bb == 0.0 || hs[c].res <= tol * bb || hs[c].active == 0;
    rep[c].status = conv ? IFMM_OK : IFMM_ERR_NOT_CONVERGED;
    if (!conv) out = IFMM_ERR_NOT_CONVERGED;
  }
  return out;
}

}  // namespace ifmm
