// factor.cu -- IFMM elimination (Algorithms 1-3 of the paper) on the GPU.
//
// Level by level (l = L .. 2) the factorisation
//   1. builds weighted bases for the level (footnote to Eq. U_j_recomp):
//      left SVD of U_i [K_iq V_q^T]_{q in I_i}, truncated at tau (reading R6);
//   2. eliminates the level colour by colour (colour = box index mod 3 per
//      dimension; boxes of one colour have disjoint neighbour lists, so all of
//      them are eliminated in the same launches):
//        gather E(P,P), E(P,C), E(R,P) of every box  -> batched LU (FP64)
//        -> G = E(P,P)^-1 E(P,C) -> S = E(R,P) G (Schur product)
//        -> scatter -S into neighbour / M2L edges, keep well-separated fill;
//   3. recompresses the bases of the boxes that received well-separated fill
//      (Eqs. U_j_recomp, V_j_recomp; aggregated per box, reading R4) and
//      redirects every edge of those boxes (Algorithm 3, Eq. K_kj_update);
//   4. merges the level into its parent (Eqs. y_merge - K_merge).
// The top system for y^(2) is factorised densely.
#include <chrono>
#include <cstdio>
#include <memory>
#include <map>
#include <set>

#include "factor.cuh"

namespace ifmm {

using Clock = std::chrono::steady_clock;
static double since(Clock::time_point t) {
  return std::chrono::duration<double>(Clock::now() - t).count();
}
// IFMM_TRACE=1: one line per phase on stderr (sizes, ranks, seconds);
// IFMM_TRACE=2 adds one line per SVD launch
static bool tracing() {
  static const bool v = [] {
    const char* e = std::getenv("IFMM_TRACE");
    return e && (e[0] == '1' || e[0] == '2' || e[0] == '3');
  }();
  return v;
}
#define TRACE(...) \
  do {                                  \
    if (tracing()) {                    \
      std::fprintf(stderr, __VA_ARGS__); \
      std::fflush(stderr);              \
    }                                   \
  } while (0)

// IFMM_TRACE=3: after each stage of a colour, copy the blocks it produced to
// the host and report the first one holding a non-finite value (debugging aid;
// synchronises and is slow).
static bool checking() {
  static const bool v = [] {
    const char* e = std::getenv("IFMM_TRACE");
    return e && e[0] == '3';
  }();
  return v;
}
static void check_finite(const char* stage, int l, const std::vector<int>& boxes,
                         const std::vector<std::pair<const double*, size_t>>& arrays,
                         cudaStream_t s) {
  if (!checking()) return;
  CK(cudaStreamSynchronize(s));
  for (size_t k = 0; k < arrays.size(); k++) {
    if (!arrays[k].first || arrays[k].second == 0) continue;
    std::vector<double> h(arrays[k].second);
    CK(cudaMemcpy(h.data(), arrays[k].first, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    size_t bad = 0;
    double mx = 0.0;
    for (double v : h) {
      if (!std::isfinite(v)) bad++;
      else mx = std::max(mx, std::fabs(v));
    }
    if (bad) {
      std::fprintf(stderr, "[ifmm-check] level %d %s: array %zu of %zu has %zu non-finite of %zu (boxes",
                   l, stage, k, arrays.size(), bad, h.size());
      for (int b : boxes) std::fprintf(stderr, " %d", b);
      std::fprintf(stderr, ")\n");
      return;
    }
    if (mx > 1e100)
      std::fprintf(stderr, "[ifmm-check] level %d %s: array %zu max |v| %.3g\n", l, stage, k, mx);
  }
}

static inline GemmTask gm(const double* A, int lda, int tA, const double* B, int ldb, int tB,
                          double* C, int ldc, int M, int N, int K, double alpha, double beta) {
  return GemmTask{A, B, C, lda, ldb, ldc, M, N, K, tA, tB, alpha, beta};
}
static inline CopyTask cp(const double* src, int lds, double* dst, int ldd, int rows, int cols,
                          int trans = 0, double alpha = 1.0, double beta = 0.0,
                          const double* cscale = nullptr, int kind = 0) {
  return CopyTask{src, dst, cscale, lds, ldd, rows, cols, trans, kind, alpha, beta};
}
static inline CopyTask cp_eye(double* dst, int ldd, int n, double alpha) {
  return CopyTask{nullptr, dst, nullptr, 1, ldd, n, n, 0, 1, alpha, 0.0};
}
static inline CopyTask cp_zero(double* dst, int ldd, int rows, int cols) {
  return CopyTask{nullptr, dst, nullptr, 1, ldd, rows, cols, 0, 2, 0.0, 0.0};
}

static void run_copies(Arena& ar, const std::vector<CopyTask>& v, cudaStream_t s) {
  std::vector<CopyTask> keep;
  keep.reserve(v.size());
  for (const CopyTask& c : v)
    if (c.rows > 0 && c.cols > 0) {
      validate(c);
      keep.push_back(c);
    }
  if (keep.empty()) return;
  const CopyTask* d = upload(ar, keep, s);
  launch_copy(d, (int)keep.size(), s);
}

struct FLevel {
  int l = 0, nb = 0;
  std::vector<int> a, r, rcap;
  std::vector<char> elim;
  std::vector<double*> X, Y;  // per neighbour slot (ld a_i) / per N u I slot (ld rcap_i)
  std::vector<double*> U, V, SU, SV, Upar, Vpar;
  std::vector<double*> Uraw, Vraw;  // raw bases of this level (a_i x nd, ld a_i)
  EdgeLevel edge{};                  // device copies of the lists for k_edge_redirect
  Arena mem;
};

// Blocks taller than rsvd_rows (default 160) are recompressed with the
// randomised SVD of Sec. 2.4 when the rank cap is below the block height and
// truncation is on (tau > 0): the top k = min(a, cap + 16) singular triplets
// decide the rank (oversampling 16, one power iteration).
static int rsvd_k(int a, int rcap) { return std::min(a, rcap + RSVD_OVERSAMPLE); }

struct Factorizer {
  ifmm_system* sys;
  ifmm_factorization* f;
  cudaStream_t s;
  const ChebOps& ops;
  int nd, dim;
  double tau = 0.0;
  int cap_global = 0;
  Arena scratch;
  int* d_counters = nullptr;  // [0]: rank cap hits, [1]: tensor-core wait timeouts
  int rsvd_rows = RSVD_ROWS_DEFAULT;

  bool use_rsvd(int a, int rcap) const { return tau > 0.0 && a > rsvd_rows && rcap < a; }

  Factorizer(ifmm_system* sy, ifmm_factorization* fa, cudaStream_t st)
      : sys(sy), f(fa), s(st), ops(sy->ops_f), nd(sy->ops_f.nd), dim(sy->dim) {}

  double* X(FLevel& st, const LevelTopo& lv, int i, int j) {
    const int k = lv.nslot(i, j);
    if (k < 0) throw Error(IFMM_ERR_CUDA, "internal: missing near block");
    return st.X[k];
  }
  double* Y(FLevel& st, const LevelTopo& lv, int i, int j) {
    const int k = lv.yslot(i, j);
    if (k < 0) throw Error(IFMM_ERR_CUDA, "internal: missing far block");
    return st.Y[k];
  }

  void alloc_level(FLevel& st, const LevelTopo& lv) {
    st.l = lv.l;
    st.nb = lv.nb;
    st.rcap.resize(st.nb);
    for (int i = 0; i < st.nb; i++) st.rcap[i] = std::min(st.a[i], cap_global);
    st.r.assign(st.nb, 0);
    st.elim.assign(st.nb, 0);
    long long nx = 0, ny = 0, nu = 0, ns = 0, np = 0;
    for (int i = 0; i < st.nb; i++) {
      for (int k = lv.nbr_ptr[i]; k < lv.nbr_ptr[i + 1]; k++)
        nx += (long long)st.a[i] * st.a[lv.nbr[k]];
      for (int k = lv.yl_ptr[i]; k < lv.yl_ptr[i + 1]; k++)
        ny += (long long)st.rcap[i] * st.rcap[lv.yl[k]];
      nu += (long long)st.a[i] * st.rcap[i];
      ns += st.rcap[i];
      np += (long long)st.rcap[i] * nd;
    }
    double* bx = st.mem.alloc<double>(std::max(nx, 1ll));
    double* by = st.mem.alloc<double>(std::max(ny, 1ll));
    CK(cudaMemsetAsync(by, 0, sizeof(double) * std::max(ny, 1ll), s));
    double* bu = st.mem.alloc<double>(std::max(2 * nu, 1ll));
    double* bs = st.mem.alloc<double>(std::max(2 * ns, 1ll));
    double* bp = st.mem.alloc<double>(std::max(2 * np, 1ll));
    st.X.assign(lv.nbr.size(), nullptr);
    st.Y.assign(lv.yl.size(), nullptr);
    st.U.resize(st.nb); st.V.resize(st.nb); st.SU.resize(st.nb); st.SV.resize(st.nb);
    st.Upar.resize(st.nb); st.Vpar.resize(st.nb);
    long long ox = 0, oy = 0, ou = 0, os = 0, op = 0;
    for (int i = 0; i < st.nb; i++) {
      for (int k = lv.nbr_ptr[i]; k < lv.nbr_ptr[i + 1]; k++) {
        st.X[k] = bx + ox;
        ox += (long long)st.a[i] * st.a[lv.nbr[k]];
      }
      for (int k = lv.yl_ptr[i]; k < lv.yl_ptr[i + 1]; k++) {
        st.Y[k] = by + oy;
        oy += (long long)st.rcap[i] * st.rcap[lv.yl[k]];
      }
      st.U[i] = bu + ou;
      st.V[i] = bu + nu + ou;
      ou += (long long)st.a[i] * st.rcap[i];
      st.SU[i] = bs + os;
      st.SV[i] = bs + ns + os;
      os += st.rcap[i];
      st.Upar[i] = bp + op;
      st.Vpar[i] = bp + np + op;
      op += (long long)st.rcap[i] * nd;
    }
    // interaction lists and edge blocks for the device-side edge redirection
    std::vector<double*> yo(lv.far.size()), yi(lv.far.size());
    for (int i = 0; i < st.nb; i++)
      for (int k = lv.far_ptr[i]; k < lv.far_ptr[i + 1]; k++) {
        yo[k] = Y(st, lv, i, lv.far[k]);
        yi[k] = Y(st, lv, lv.far[k], i);
      }
    st.edge.far_ptr = upload(st.mem, lv.far_ptr, s);
    st.edge.far = upload(st.mem, lv.far, s);
    st.edge.y_out = upload(st.mem, yo, s);
    st.edge.y_in = upload(st.mem, yi, s);
    st.edge.rcap = upload(st.mem, st.rcap, s);
  }

  // sync and read ranks written by rank tasks
  std::vector<int> read_ints(const int* d, int n) {
    std::vector<int> h(n);
    if (n > 0) CK(cudaMemcpyAsync(h.data(), d, n * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return h;
  }

  // -------------------------------------------------------------------------
  // weighted initial bases of a level (footnote to Eq. U_j_recomp, reading R6)
  //
  // Small boxes (a <= n^D): left SVD of M = U_i [K_iq V_q^T]_{q in I_i}
  // (a x sum a_q).  Tall boxes (a > n^D): the same subspace from the reduced
  // form C = R_i [K_iq R_q^T]_q (n^D x n^D |I_i|), where U_i = Q_i R_i comes
  // from the SVD of U_i (R_i = Sigma_i W_i^T) and likewise R_q for V_q; then
  // U_hat = U_i W_i Sigma_i^-1 W_C and r_i = W_C^T R_i.
  // -------------------------------------------------------------------------
  struct Side {
    std::vector<double*> W, sg;      // small boxes: W (a x a), sigma (a); tall: W_C, sigma_C (nd)
    std::vector<double*> R, T2;      // all boxes: R (nd x nd); tall boxes: T2 = W Sigma^-1 W_C
  };

  // R_i (nd x nd) = diag(sigma) W^T from the SVD of raw^T (nd x a), for every box;
  // T_i = W diag(1/sigma) (nd x nd) for the tall boxes
  void raw_factors(FLevel& st, const std::vector<double*>& raw, std::vector<double*>& R,
                   std::vector<double*>& Winv, Arena& keep) {
    const int nb = st.nb;
    std::vector<CopyTask> tr, sc;
    std::vector<SvdTask> sv;
    std::vector<double*> XT(nb), W(nb), sg(nb), P(nb);
    R.assign(nb, nullptr);
    Winv.assign(nb, nullptr);
    for (int i = 0; i < nb; i++) {
      const int a = st.a[i];
      XT[i] = scratch.alloc<double>((size_t)nd * std::max(a, 1));
      W[i] = scratch.alloc<double>((size_t)nd * nd);
      sg[i] = keep.alloc<double>(nd);
      P[i] = scratch.alloc<double>((size_t)nd * nd);
      R[i] = keep.alloc<double>((size_t)nd * nd);
      tr.push_back(cp(raw[i], a, XT[i], nd, nd, a, 1));
      sv.push_back({XT[i], nd, nd, a, W[i], sg[i], nullptr});
    }
    run_copies(scratch, tr, s);
    run_svd_left(scratch, sv, s);
    std::vector<CopyTask> c2;
    for (int i = 0; i < nb; i++) {
      c2.push_back(cp(W[i], nd, P[i], nd, nd, nd, 0, 1.0, 0.0, sg[i]));  // W diag(sigma)
    }
    run_copies(scratch, c2, s);
    c2.clear();
    for (int i = 0; i < nb; i++) c2.push_back(cp(P[i], nd, R[i], nd, nd, nd, 1));  // R = (W S)^T
    run_copies(scratch, c2, s);
    // inverse sigma (dropping null directions) for the tall boxes
    c2.clear();
    std::vector<int> tall;
    for (int i = 0; i < nb; i++)
      if (st.a[i] > nd) tall.push_back(i);
    if (!tall.empty()) {
      std::vector<double*> inv(nb, nullptr);
      std::vector<InvSigma> iv;
      for (int i : tall) {
        inv[i] = scratch.alloc<double>(nd);
        Winv[i] = keep.alloc<double>((size_t)nd * nd);
        iv.push_back({sg[i], inv[i], nd});
      }
      run_inv_sigma(scratch, iv, s);
      for (int i : tall) c2.push_back(cp(W[i], nd, Winv[i], nd, nd, nd, 0, 1.0, 0.0, inv[i]));
      run_copies(scratch, c2, s);
    }
  }

  void init_basis(FLevel& st, const LevelTopo& lv) {
    const int nb = st.nb;
    const double s0 = std::isnan(sys->sigma0) ? 1.0 : sys->sigma0;
    Arena keep;  // per-box factors until ranks are known
    scratch.reset();
    std::vector<double*> RU, RV, TU, TV;
    bool any_tall = false;
    for (int i = 0; i < nb; i++) any_tall |= st.a[i] > nd;
    const bool sym = sys->opt.symmetric != 0;  // reading S: V side = U side
    if (any_tall) {
      raw_factors(st, st.Uraw, RU, TU, keep);
      if (sym) { RV = RU; TV = TU; }
      else raw_factors(st, st.Vraw, RV, TV, keep);
    }
    std::vector<double*> WU(nb), WV(nb), sU(nb), sV(nb);
    std::vector<int> full(nb);
    for (int i = 0; i < nb; i++) {
      const int a = st.a[i];
      const int dimW = a > nd ? nd : a;  // rows of the matrix whose SVD decides the rank
      WU[i] = keep.alloc<double>((size_t)dimW * dimW);
      sU[i] = keep.alloc<double>(dimW);
      WV[i] = sym ? WU[i] : keep.alloc<double>((size_t)dimW * dimW);
      sV[i] = sym ? sU[i] : keep.alloc<double>(dimW);
      full[i] = std::min(a, nd);
    }
    int* d_r = keep.alloc<int>(nb);
    CK(cudaStreamSynchronize(s));
    int i0 = 0;
    while (i0 < nb) {
      scratch.reset();
      long long budget = 0;
      int i1 = i0;
      while (i1 < nb) {
        long long w = 0;
        for (int k = lv.far_ptr[i1]; k < lv.far_ptr[i1 + 1]; k++)
          w += st.a[i1] > nd ? nd : st.a[lv.far[k]];
        if (w == 0) w = nd;
        const long long need = 2 * ((long long)std::min(st.a[i1], nd) * w + (long long)nd * w);
        if (i1 > i0 && budget + need > (256ll << 20)) break;
        budget += need;
        i1++;
      }
      std::vector<GemmTask> g1, g2;
      std::vector<CopyTask> cps;
      std::vector<SvdTask> svd;
      for (int i = i0; i < i1; i++) {
        const int a = st.a[i];
        const bool tall = a > nd;
        const int rows = tall ? nd : a;
        long long w = 0;
        for (int k = lv.far_ptr[i]; k < lv.far_ptr[i + 1]; k++) w += tall ? nd : st.a[lv.far[k]];
        double *MU, *MV;
        int wcols;
        if (w == 0) {
          // empty interaction list: weight the raw basis by sigma_0 (reading R6)
          wcols = nd;
          MU = scratch.alloc<double>((size_t)rows * nd);
          MV = sym ? nullptr : scratch.alloc<double>((size_t)rows * nd);
          if (tall) {
            cps.push_back(cp(RU[i], nd, MU, nd, nd, nd, 0, s0));
            if (!sym) cps.push_back(cp(RV[i], nd, MV, nd, nd, nd, 0, s0));
          } else {
            cps.push_back(cp(st.Uraw[i], a, MU, a, a, nd, 0, s0));
            if (!sym) cps.push_back(cp(st.Vraw[i], a, MV, a, a, nd, 0, s0));
          }
        } else {
          wcols = (int)w;
          double* BU = scratch.alloc<double>((size_t)nd * w);
          double* BV = sym ? nullptr : scratch.alloc<double>((size_t)nd * w);
          MU = scratch.alloc<double>((size_t)rows * w);
          MV = sym ? nullptr : scratch.alloc<double>((size_t)rows * w);
          long long off = 0;
          for (int k = lv.far_ptr[i]; k < lv.far_ptr[i + 1]; k++) {
            const int q = lv.far[k];
            const int aq = st.a[q];
            const double* Kiq = ops.m2l[lv.l] + (size_t)lv.m2l_offset(i, q, dim) * nd * nd;
            const double* Kqi = ops.m2l[lv.l] + (size_t)lv.m2l_offset(q, i, dim) * nd * nd;
            if (tall) {
              // BU[:, off] = K_iq R_q^T ; BV[:, off] = K_qi^T R_q(U)^T   (nd x nd)
              g1.push_back(gm(Kiq, nd, 0, RV[q], nd, 1, BU + off * nd, nd, nd, nd, nd, 1.0, 0.0));
              if (!sym)
                g1.push_back(gm(Kqi, nd, 1, RU[q], nd, 1, BV + off * nd, nd, nd, nd, nd, 1.0, 0.0));
              off += nd;
            } else {
              // BU[:, off] = K_iq V_q^T ; BV[:, off] = K_qi^T U_q^T
              g1.push_back(gm(Kiq, nd, 0, st.Vraw[q], aq, 1, BU + off * nd, nd, nd, aq, nd, 1.0, 0.0));
              if (!sym)
                g1.push_back(gm(Kqi, nd, 1, st.Uraw[q], aq, 1, BV + off * nd, nd, nd, aq, nd, 1.0, 0.0));
              off += aq;
            }
          }
          if (tall) {
            g2.push_back(gm(RU[i], nd, 0, BU, nd, 0, MU, nd, nd, (int)w, nd, 1.0, 0.0));
            if (!sym) g2.push_back(gm(RV[i], nd, 0, BV, nd, 0, MV, nd, nd, (int)w, nd, 1.0, 0.0));
          } else {
            g2.push_back(gm(st.Uraw[i], a, 0, BU, nd, 0, MU, a, a, (int)w, nd, 1.0, 0.0));
            if (!sym) g2.push_back(gm(st.Vraw[i], a, 0, BV, nd, 0, MV, a, a, (int)w, nd, 1.0, 0.0));
          }
        }
        svd.push_back({MU, rows, rows, wcols, WU[i], sU[i], nullptr});
        if (!sym) svd.push_back({MV, rows, rows, wcols, WV[i], sV[i], nullptr});
        f->info.flops_lowrank += (sym ? 2.0 : 4.0) * rows * (double)rows * wcols;
      }
      run_copies(scratch, cps, s);
      run_gemms(scratch, g1, s);
      run_gemms(scratch, g2, s);
      run_svd_left(scratch, svd, s);
      std::vector<RankTask> rt;
      for (int i = i0; i < i1; i++)
        rt.push_back({sU[i], sV[i], full[i], std::min(full[i], st.rcap[i]), d_r + i, d_counters});
      const RankTask* drt = upload(scratch, rt, s);
      launch_rank(drt, (int)rt.size(), tau, s);
      CK(cudaStreamSynchronize(s));
      i0 = i1;
    }
    std::vector<int> r = read_ints(d_r, nb);
    scratch.reset();
    // new bases U_hat, V_hat (a x r) and the transforms r_i, t_i (r x nd)
    std::vector<double*> rt(nb), tt(nb);
    std::vector<GemmTask> g, g2;
    std::vector<CopyTask> cps;
    for (int i = 0; i < nb; i++) {
      const int a = st.a[i];
      st.r[i] = r[i];
      const int ldr = std::max(r[i], 1);
      rt[i] = scratch.alloc<double>((size_t)ldr * nd);
      tt[i] = scratch.alloc<double>((size_t)ldr * nd);
      if (a > nd) {
        double* T2U = scratch.alloc<double>((size_t)nd * nd);
        double* T2V = scratch.alloc<double>((size_t)nd * nd);
        g.push_back(gm(TU[i], nd, 0, WU[i], nd, 0, T2U, nd, nd, r[i], nd, 1.0, 0.0));
        g.push_back(gm(TV[i], nd, 0, WV[i], nd, 0, T2V, nd, nd, r[i], nd, 1.0, 0.0));
        g2.push_back(gm(st.Uraw[i], a, 0, T2U, nd, 0, st.U[i], a, a, r[i], nd, 1.0, 0.0));
        g2.push_back(gm(st.Vraw[i], a, 0, T2V, nd, 0, st.V[i], a, a, r[i], nd, 1.0, 0.0));
        g.push_back(gm(WU[i], nd, 1, RU[i], nd, 0, rt[i], ldr, r[i], nd, nd, 1.0, 0.0));
        g.push_back(gm(WV[i], nd, 1, RV[i], nd, 0, tt[i], ldr, r[i], nd, nd, 1.0, 0.0));
      } else {
        g.push_back(gm(WU[i], a, 1, st.Uraw[i], a, 0, rt[i], ldr, r[i], nd, a, 1.0, 0.0));
        g.push_back(gm(WV[i], a, 1, st.Vraw[i], a, 0, tt[i], ldr, r[i], nd, a, 1.0, 0.0));
        cps.push_back(cp(WU[i], a, st.U[i], a, a, r[i]));
        cps.push_back(cp(WV[i], a, st.V[i], a, a, r[i]));
      }
      cps.push_back(cp(sU[i], 1, st.SU[i], 1, r[i], 1));
      cps.push_back(cp(sV[i], 1, st.SV[i], 1, r[i], 1));
    }
    run_gemms(scratch, g, s);
    run_gemms(scratch, g2, s);
    run_copies(scratch, cps, s);
    g.clear();
    g2.clear();
    for (int i = 0; i < nb; i++) {
      const int ri = st.r[i];
      const int ldr = std::max(ri, 1);
      for (int k = lv.far_ptr[i]; k < lv.far_ptr[i + 1]; k++) {
        const int q = lv.far[k];
        const double* Kiq = ops.m2l[lv.l] + (size_t)lv.m2l_offset(i, q, dim) * nd * nd;
        double* T1 = scratch.alloc<double>((size_t)ldr * nd);
        g.push_back(gm(rt[i], ldr, 0, Kiq, nd, 0, T1, ldr, ri, nd, nd, 1.0, 0.0));
        g2.push_back(gm(T1, ldr, 0, tt[q], std::max(st.r[q], 1), 1, Y(st, lv, i, q), st.rcap[i],
                        ri, st.r[q], nd, 1.0, 0.0));
      }
      if (lv.l > 2) {
        const double* Tc = ops.transfer + (size_t)lv.child_pos(i, dim) * nd * nd;
        g.push_back(gm(rt[i], ldr, 0, Tc, nd, 0, st.Upar[i], st.rcap[i], ri, nd, nd, 1.0, 0.0));
        g.push_back(gm(tt[i], ldr, 0, Tc, nd, 0, st.Vpar[i], st.rcap[i], ri, nd, nd, 1.0, 0.0));
      }
    }
    run_gemms(scratch, g, s);
    run_gemms(scratch, g2, s);
    CK(cudaStreamSynchronize(s));
    scratch.reset();
  }

  // -------------------------------------------------------------------------
  // elimination of one colour class (Algorithm 2, aggregated reading R4)
  // -------------------------------------------------------------------------
  void eliminate_colour(FLevel& st, const LevelTopo& lv, const std::vector<int>& boxes) {
    scratch.reset();
    const int nbx = (int)boxes.size();
    std::vector<FRec> recs(nbx);
    std::vector<double*> S(nbx), LU(nbx), ERP(nbx), G(nbx);
    std::vector<int*> piv(nbx);
    std::vector<CopyTask> cps;
    std::vector<LuTask> lus;
    std::vector<RsTask> rss;
    std::vector<GemmTask> gs;
    for (int b = 0; b < nbx; b++) {
      const int i = boxes[b];
      FRec& R = recs[b];
      R.l = lv.l;
      R.i = i;
      R.a = st.a[i];
      R.r = st.r[i];
      R.p = R.a + R.r;
      R.colour = lv.colour[i];
      int off = 0;
      for (int k = lv.nbr_ptr[i]; k < lv.nbr_ptr[i + 1]; k++) {
        const int j = lv.nbr[k];
        if (j == i) continue;
        const char kind = st.elim[j] ? 'y' : 'x';
        const int d = kind == 'x' ? st.a[j] : st.r[j];
        R.blk.push_back({kind, j, d, off});
        off += d;
      }
      R.blk.push_back({'y', i, R.r, off});
      off += R.r;
      R.nC = off;
      const int p = R.p, nC = R.nC, a = R.a, r = R.r;
      LU[b] = scratch.alloc<double>((size_t)p * p);
      piv[b] = scratch.alloc<int>(p);
      R.info = f->store.alloc<int>(1);
      ERP[b] = scratch.alloc<double>((size_t)nC * p);
      G[b] = scratch.alloc<double>((size_t)p * nC);
      CK(cudaMemsetAsync(ERP[b], 0, sizeof(double) * (size_t)nC * p, s));
      CK(cudaMemsetAsync(G[b], 0, sizeof(double) * (size_t)p * nC, s));
      double* amax = scratch.alloc<double>(1);
      // E(P,P) = [[X(i,i), U_i], [V_i^T, 0]]
      cps.push_back(cp(X(st, lv, i, i), a, LU[b], p, a, a));
      cps.push_back(cp(st.U[i], a, LU[b] + (size_t)a * p, p, a, r));
      cps.push_back(cp(st.V[i], a, LU[b] + a, p, r, a, 1));
      cps.push_back(cp_zero(LU[b] + a + (size_t)a * p, p, r, r));
      for (const BlockRef& B : R.blk) {
        if (B.kind == 'y' && B.box == i) {
          cps.push_back(cp_eye(G[b] + a + (size_t)B.off * p, p, r, -1.0));
          cps.push_back(cp_eye(ERP[b] + B.off + (size_t)a * nC, nC, r, -1.0));
        } else {
          cps.push_back(cp(X(st, lv, i, B.box), a, G[b] + (size_t)B.off * p, p, a, B.dim));
          const int ldj = st.a[B.box];
          cps.push_back(cp(X(st, lv, B.box, i), ldj, ERP[b] + B.off, nC, B.dim, a));
        }
      }
      // W starts as [I_a; 0] and is solved in place with the LU
      R.W = f->store.alloc<double>((size_t)p * std::max(a, 1));
      R.F = f->store.alloc<double>((size_t)nC * std::max(a, 1));
      R.Ga = f->store.alloc<double>((size_t)std::max(a, 1) * nC);
      cps.push_back(cp_eye(R.W, p, a, 1.0));
      cps.push_back(cp_zero(R.W + a, p, r, a));
      lus.push_back({LU[b], p, p, piv[b], R.info, amax});
      rss.push_back({LU[b], p, p, piv[b], G[b], p, nC});
      rss.push_back({LU[b], p, p, piv[b], R.W, p, a});
      S[b] = scratch.alloc<double>((size_t)nC * nC);
      gs.push_back(gm(ERP[b], nC, 0, G[b], p, 0, S[b], nC, nC, nC, p, 1.0, 0.0));
      f->info.flops_lu += 2.0 / 3.0 * p * (double)p * p;
      f->info.flops_trsm += 2.0 * p * (double)p * (nC + a);
      f->info.flops_schur += 2.0 * nC * (double)p * (nC + a);
    }
    run_copies(scratch, cps, s);
    if (checking()) {
      std::vector<std::pair<const double*, size_t>> v;
      for (int b = 0; b < nbx; b++) {
        v.push_back({LU[b], (size_t)recs[b].p * recs[b].p});
        v.push_back({G[b], (size_t)recs[b].p * recs[b].nC});
        v.push_back({ERP[b], (size_t)recs[b].nC * recs[b].p});
      }
      check_finite("pivot inputs", lv.l, boxes, v, s);
    }
    run_getrf(scratch, lus, s);
    run_getrs(scratch, rss, s);
    if (checking()) {
      std::vector<std::pair<const double*, size_t>> v;
      for (int b = 0; b < nbx; b++) {
        v.push_back({LU[b], (size_t)recs[b].p * recs[b].p});
        v.push_back({G[b], (size_t)recs[b].p * recs[b].nC});
      }
      check_finite("LU and G", lv.l, boxes, v, s);
    }
    // the substitution blocks: F = E(R,P) W, Ga = G[0:a, :]
    {
      std::vector<GemmTask> fg;
      std::vector<CopyTask> gc;
      for (int b = 0; b < nbx; b++) {
        const FRec& R = recs[b];
        fg.push_back(gm(ERP[b], R.nC, 0, R.W, R.p, 0, R.F, R.nC, R.nC, R.a, R.p, 1.0, 0.0));
        gc.push_back(cp(G[b], R.p, R.Ga, std::max(R.a, 1), R.a, R.nC));
      }
      run_gemms(scratch, fg, s);
      run_copies(scratch, gc, s);
    }
    // Schur products S = E(R,P) G: FP64, or the tensor cores in the
    // mixed-precision modes (a wait that runs out counts in d_counters[1])
    const int prec = sys->opt.schur;
    if (prec == IFMM_P_TF32 || prec == IFMM_P_FP32 || prec == IFMM_P_BF16)
      run_gemms_tc(scratch, gs, prec, d_counters + 1, s);
    else
      run_gemms(scratch, gs, s);
    if (checking()) {
      std::vector<std::pair<const double*, size_t>> v;
      for (int b = 0; b < nbx; b++) v.push_back({S[b], (size_t)recs[b].nC * recs[b].nC});
      check_finite("Schur products", lv.l, boxes, v, s);
    }
    // scatter -S into edges; collect well-separated fill
    struct Fill { int b, rb, cb; };
    std::vector<Fill> fills;
    cps.clear();
    for (int b = 0; b < nbx; b++) {
      const FRec& R = recs[b];
      const int i = R.i, nC = R.nC;
      for (int x = 0; x < (int)R.blk.size(); x++) {
        const BlockRef& rb = R.blk[x];
        for (int y = 0; y < (int)R.blk.size(); y++) {
          const BlockRef& cb = R.blk[y];
          const double* src = S[b] + rb.off + (size_t)cb.off * nC;
          const int rj = rb.box, cj = cb.box;
          if (rb.kind == 'y' && cb.kind == 'y') {
            cps.push_back(cp(src, nC, Y(st, lv, rj, cj), st.rcap[rj], rb.dim, cb.dim, 0, -1.0, 1.0));
          } else if (rb.kind == 'x' && cb.kind == 'y' && cj == i) {
            cps.push_back(cp(src, nC, X(st, lv, rj, i), st.a[rj], rb.dim, cb.dim, 0, -1.0, 0.0));
          } else if (rb.kind == 'y' && rj == i && cb.kind == 'x') {
            cps.push_back(cp(src, nC, X(st, lv, i, cj), st.a[i], rb.dim, cb.dim, 0, -1.0, 0.0));
          } else if (lv.is_nbr(rj, cj)) {
            cps.push_back(cp(src, nC, X(st, lv, rj, cj), st.a[rj], rb.dim, cb.dim, 0, -1.0, 1.0));
          } else {
            fills.push_back({b, x, y});
          }
        }
      }
    }
    run_copies(scratch, cps, s);
    for (int b = 0; b < nbx; b++) st.elim[boxes[b]] = 1;
    if (!fills.empty()) compress(st, lv, recs, S, fills);
    for (auto& R : recs) f->recs.push_back(std::move(R));
  }

  template <class Fill>
  void compress(FLevel& st, const LevelTopo& lv, const std::vector<FRec>& recs,
                const std::vector<double*>& S, const std::vector<Fill>& fills) {
    // recompressed boxes (uneliminated, with well-separated fill), in Morton order
    std::map<int, int> slot;  // box -> index in J
    std::vector<int> J;
    for (const Fill& F : fills) {
      const FRec& R = recs[F.b];
      const int ks[2] = {F.rb, F.cb};
      for (int k : ks)
        if (R.blk[k].kind == 'x' && !slot.count(R.blk[k].box)) slot[R.blk[k].box] = 0;
    }
    for (auto& kv : slot) { kv.second = (int)J.size(); J.push_back(kv.first); }
    const int nJ = (int)J.size();
    std::vector<int> wU(nJ, 0), wV(nJ, 0);
    for (int t = 0; t < nJ; t++) wU[t] = wV[t] = st.r[J[t]];
    for (const Fill& F : fills) {
      const FRec& R = recs[F.b];
      const BlockRef &rb = R.blk[F.rb], &cb = R.blk[F.cb];
      if (rb.kind == 'x') wU[slot[rb.box]] += cb.dim;
      if (cb.kind == 'x') wV[slot[cb.box]] += rb.dim;
    }
    const bool sym = sys->opt.symmetric != 0;  // reading S: V side = U side
    std::vector<double*> MU(nJ), MV(nJ), WU(nJ), WV(nJ), sU(nJ), sV(nJ);
    std::vector<int> cU(nJ), cV(nJ), kk(nJ);
    std::vector<CopyTask> cps;
    std::vector<SvdTask> svd;
    std::vector<RsvdTask> rsvd;
    int* d_r = scratch.alloc<int>(nJ);
    for (int t = 0; t < nJ; t++) {
      const int j = J[t], a = st.a[j], r = st.r[j];
      kk[t] = use_rsvd(a, st.rcap[j]) ? rsvd_k(a, st.rcap[j]) : a;  // singular values kept
      MU[t] = scratch.alloc<double>((size_t)a * wU[t]);
      WU[t] = scratch.alloc<double>((size_t)a * kk[t]);
      sU[t] = scratch.alloc<double>(kk[t]);
      MV[t] = sym ? nullptr : scratch.alloc<double>((size_t)a * wV[t]);
      WV[t] = sym ? WU[t] : scratch.alloc<double>((size_t)a * kk[t]);
      sV[t] = sym ? sU[t] : scratch.alloc<double>(kk[t]);
      cps.push_back(cp(st.U[j], a, MU[t], a, a, r, 0, 1.0, 0.0, st.SU[j]));
      if (!sym) cps.push_back(cp(st.V[j], a, MV[t], a, a, r, 0, 1.0, 0.0, st.SV[j]));
      cU[t] = cV[t] = r;
    }
    for (const Fill& F : fills) {  // [U Sigma_U | F_j1 | ..], [V Sigma_V | F_1j^T | ..]
      const FRec& R = recs[F.b];
      const BlockRef &rb = R.blk[F.rb], &cb = R.blk[F.cb];
      const double* src = S[F.b] + rb.off + (size_t)cb.off * R.nC;
      if (rb.kind == 'x') {
        const int t = slot[rb.box];
        const int a = st.a[rb.box];
        cps.push_back(cp(src, R.nC, MU[t] + (size_t)cU[t] * a, a, rb.dim, cb.dim, 0, -1.0));
        cU[t] += cb.dim;
      }
      if (cb.kind == 'x' && !sym) {
        const int t = slot[cb.box];
        const int a = st.a[cb.box];
        cps.push_back(cp(src, R.nC, MV[t] + (size_t)cV[t] * a, a, cb.dim, rb.dim, 1, -1.0));
        cV[t] += rb.dim;
      }
    }
    run_copies(scratch, cps, s);
    std::vector<RankTask> rt;
    for (int t = 0; t < nJ; t++) {
      const int j = J[t], a = st.a[j];
      const double wsum = wU[t] + (sym ? 0.0 : (double)wV[t]);
      if (kk[t] < a) {
        rsvd.push_back({MU[t], a, a, wU[t], kk[t], rsvd_seed(lv.l, j, 0), WU[t], sU[t]});
        if (!sym) rsvd.push_back({MV[t], a, a, wV[t], kk[t], rsvd_seed(lv.l, j, 1), WV[t], sV[t]});
        f->info.flops_lowrank += 8.0 * a * (double)kk[t] * wsum;
      } else {
        svd.push_back({MU[t], a, a, wU[t], WU[t], sU[t], nullptr});
        if (!sym) svd.push_back({MV[t], a, a, wV[t], WV[t], sV[t], nullptr});
        f->info.flops_lowrank += 4.0 * a * (double)a * wsum;
      }
      rt.push_back({sU[t], sV[t], kk[t], st.rcap[j], d_r + t, d_counters});
    }
    if (checking()) {
      std::vector<std::pair<const double*, size_t>> v;
      for (int t = 0; t < nJ; t++) {
        v.push_back({MU[t], (size_t)st.a[J[t]] * wU[t]});
        if (!sym) v.push_back({MV[t], (size_t)st.a[J[t]] * wV[t]});
      }
      check_finite("recompression inputs", lv.l, J, v, s);
    }
    run_svd_left(scratch, svd, s);
    // randomised tasks, grouped by their common k
    std::map<int, std::vector<RsvdTask>> byk;
    for (auto& T : rsvd) byk[T.k].push_back(T);
    for (auto& kv : byk) run_rsvd_left(scratch, kv.second, s);
    if (checking()) {
      std::vector<std::pair<const double*, size_t>> v;
      for (int t = 0; t < nJ; t++) {
        v.push_back({WU[t], (size_t)st.a[J[t]] * kk[t]});
        v.push_back({sU[t], (size_t)kk[t]});
      }
      check_finite("recompression SVD", lv.l, J, v, s);
    }
    const RankTask* drt = upload(scratch, rt, s);
    launch_rank(drt, nJ, tau, s);
    std::vector<int> rn = read_ints(d_r, nJ);
    if (tracing() && checking())
      for (int t = 0; t < nJ; t++)
        TRACE("[ifmm-check] level %d box %d: a %d, rank %d -> %d, width %d\n", lv.l, J[t],
              st.a[J[t]], st.r[J[t]], rn[t], wU[t]);
    // r_j = U_hat^T U_old, t_j = V_hat^T V_old
    std::vector<double*> rm(nJ), tm(nJ);
    std::vector<GemmTask> g;
    for (int t = 0; t < nJ; t++) {
      const int j = J[t], a = st.a[j];
      rm[t] = scratch.alloc<double>((size_t)std::max(rn[t], 1) * std::max(st.r[j], 1));
      g.push_back(gm(WU[t], a, 1, st.U[j], a, 0, rm[t], std::max(rn[t], 1), rn[t], st.r[j], a, 1.0, 0.0));
      if (sym) {
        tm[t] = rm[t];  // V_hat = U_hat and V = U: t_j = r_j
      } else {
        tm[t] = scratch.alloc<double>((size_t)std::max(rn[t], 1) * std::max(st.r[j], 1));
        g.push_back(gm(WV[t], a, 1, st.V[j], a, 0, tm[t], std::max(rn[t], 1), rn[t], st.r[j], a, 1.0, 0.0));
      }
    }
    run_gemms(scratch, g, s);
    // Algorithm 3: K(j, q) <- r_j K(j, q), K(q, j) <- K(q, j) t_j^T (q in I_j).
    // Each edge once: (j, q) from j's list; (q, j) from j's list only when q is
    // not recompressed itself (otherwise q's list adds it).
    std::vector<std::pair<int, int>> edges;
    std::vector<char> isR(st.nb, 0);
    for (int j : J) isR[j] = 1;
    auto rold = [&](int b) { return st.r[b]; };
    auto rnew = [&](int b) { auto it = slot.find(b); return it == slot.end() ? st.r[b] : rn[it->second]; };
    std::vector<GemmTask> p1, p2;
    std::vector<CopyTask> c1, c2;
    int rmax = 0;
    for (int b = 0; b < st.nb; b++) rmax = std::max(rmax, std::max(rold(b), rnew(b)));
    const bool on_device = rmax <= 64;
    if (on_device) {
      // one CTA per recompressed box walks its interaction list
      std::vector<int> r0(st.nb), r1(st.nb);
      std::vector<const double*> pm(st.nb, nullptr), pt(st.nb, nullptr);
      for (int b = 0; b < st.nb; b++) { r0[b] = rold(b); r1[b] = rnew(b); }
      double fl = 0.0;
      for (int t = 0; t < nJ; t++) {
        pm[J[t]] = rm[t];
        pt[J[t]] = tm[t];
      }
      for (int j : J)
        for (int k = lv.far_ptr[j]; k < lv.far_ptr[j + 1]; k++) {
          const int q = lv.far[k];
          fl += 2.0 * r1[j] * r0[q] * r0[j];
          fl += isR[q] ? 2.0 * r1[j] * r1[q] * r0[q] : 2.0 * r0[q] * r1[j] * r0[j];
        }
      if (Ranges::on())  // host-side check of every block the kernel will touch
        for (int t = 0; t < nJ; t++) {
          const int j = J[t];
          Ranges::check(rm[t], mat_bytes(r1[j], r0[j], std::max(r1[j], 1)), "edge r_j");
          Ranges::check(tm[t], mat_bytes(r1[j], r0[j], std::max(r1[j], 1)), "edge t_j");
          for (int k = lv.far_ptr[j]; k < lv.far_ptr[j + 1]; k++) {
            const int q = lv.far[k];
            Ranges::check(Y(st, lv, j, q),
                          mat_bytes(std::max(r0[j], r1[j]), std::max(r0[q], r1[q]), st.rcap[j]),
                          "edge K(j,q)");
            if (!isR[q])
              Ranges::check(Y(st, lv, q, j), mat_bytes(r0[q], std::max(r0[j], r1[j]), st.rcap[q]),
                            "edge K(q,j)");
          }
        }
      EdgeColour E{upload(scratch, r0, s), upload(scratch, r1, s), upload(scratch, pm, s),
                   upload(scratch, pt, s), upload(scratch, J, s), std::max(rmax, 1)};
      launch_edge_redirect(st.edge, E, nJ, s, fl);
    } else {
      for (int j : J)
        for (int k = lv.far_ptr[j]; k < lv.far_ptr[j + 1]; k++) {
          const int q = lv.far[k];
          edges.push_back({j, q});
          if (!isR[q]) edges.push_back({q, j});
        }
    }
    for (auto& e : edges) {
      const int a = e.first, b = e.second;
      double* Yab = Y(st, lv, a, b);
      const int lda = st.rcap[a];
      const int ra0 = rold(a), ra1 = rnew(a), rb0 = rold(b), rb1 = rnew(b);
      double* T1 = scratch.alloc<double>((size_t)std::max(ra1, 1) * std::max(rb0, 1));
      const int ldt = std::max(ra1, 1);
      auto ia = slot.find(a), ib = slot.find(b);
      if (ia != slot.end())
        p1.push_back(gm(rm[ia->second], std::max(ra1, 1), 0, Yab, lda, 0, T1, ldt, ra1, rb0, ra0, 1.0, 0.0));
      else
        c1.push_back(cp(Yab, lda, T1, ldt, ra0, rb0));
      if (ib != slot.end())
        p2.push_back(gm(T1, ldt, 0, tm[ib->second], std::max(rb1, 1), 1, Yab, lda, ra1, rb1, rb0, 1.0, 0.0));
      else
        c2.push_back(cp(T1, ldt, Yab, lda, ra1, rb0));
    }
    // parent transfers: U(j, j-dagger) <- r_j U, V(j, j-dagger) <- t_j V (Eqs. U/V_parent_j_update)
    if (lv.l > 2)
      for (int t = 0; t < nJ; t++) {
        const int j = J[t];
        const int r0 = st.r[j], r1 = rn[t];
        double* TU = scratch.alloc<double>((size_t)std::max(r1, 1) * nd);
        double* TV = scratch.alloc<double>((size_t)std::max(r1, 1) * nd);
        p1.push_back(gm(rm[t], std::max(r1, 1), 0, st.Upar[j], st.rcap[j], 0, TU, std::max(r1, 1), r1, nd, r0, 1.0, 0.0));
        p1.push_back(gm(tm[t], std::max(r1, 1), 0, st.Vpar[j], st.rcap[j], 0, TV, std::max(r1, 1), r1, nd, r0, 1.0, 0.0));
        c2.push_back(cp(TU, std::max(r1, 1), st.Upar[j], st.rcap[j], r1, nd));
        c2.push_back(cp(TV, std::max(r1, 1), st.Vpar[j], st.rcap[j], r1, nd));
      }
    run_gemms(scratch, p1, s);
    run_copies(scratch, c1, s);
    run_gemms(scratch, p2, s);
    run_copies(scratch, c2, s);
    // redirect the fill through the new bases (Eq. K_kj_update)
    std::vector<GemmTask> q1, q2;
    for (const Fill& F : fills) {
      const FRec& R = recs[F.b];
      const BlockRef &rb = R.blk[F.rb], &cb = R.blk[F.cb];
      const double* src = S[F.b] + rb.off + (size_t)cb.off * R.nC;
      const int nC = R.nC;
      double* Yt = Y(st, lv, rb.box, cb.box);
      const int ldy = st.rcap[rb.box];
      if (rb.kind == 'x' && cb.kind == 'x') {
        const int tj = slot[rb.box], tk = slot[cb.box];
        const int rj = rn[tj], rk = rn[tk];
        double* T = scratch.alloc<double>((size_t)std::max(rj, 1) * cb.dim);
        q1.push_back(gm(WU[tj], st.a[rb.box], 1, src, nC, 0, T, std::max(rj, 1), rj, cb.dim, rb.dim, -1.0, 0.0));
        q2.push_back(gm(T, std::max(rj, 1), 0, WV[tk], st.a[cb.box], 0, Yt, ldy, rj, rk, cb.dim, 1.0, 1.0));
      } else if (rb.kind == 'x') {
        const int tj = slot[rb.box];
        q1.push_back(gm(WU[tj], st.a[rb.box], 1, src, nC, 0, Yt, ldy, rn[tj], cb.dim, rb.dim, -1.0, 1.0));
      } else {
        const int tk = slot[cb.box];
        q1.push_back(gm(src, nC, 0, WV[tk], st.a[cb.box], 0, Yt, ldy, rb.dim, rn[tk], cb.dim, -1.0, 1.0));
      }
    }
    run_gemms(scratch, q1, s);
    run_gemms(scratch, q2, s);
    // new bases and weights (the first step of Algorithm 3)
    cps.clear();
    for (int t = 0; t < nJ; t++) {
      const int j = J[t], a = st.a[j], r1 = rn[t];
      cps.push_back(cp(WU[t], a, st.U[j], a, a, r1));
      cps.push_back(cp(WV[t], a, st.V[j], a, a, r1));
      cps.push_back(cp(sU[t], 1, st.SU[j], 1, r1, 1));
      cps.push_back(cp(sV[t], 1, st.SV[j], 1, r1, 1));
    }
    run_copies(scratch, cps, s);
    for (int t = 0; t < nJ; t++) st.r[J[t]] = rn[t];
  }

  // -------------------------------------------------------------------------
  // merge (Eqs. y_merge, U_merge, V_merge, K_merge)
  // -------------------------------------------------------------------------
  void merge(FLevel& st, const LevelTopo& lv, FLevel& nst, const LevelTopo& pv) {
    nst.a.assign(pv.nb, 0);
    std::vector<std::vector<int>> coff(pv.nb);
    for (int p = 0; p < pv.nb; p++) {
      int off = 0;
      for (int c = pv.cb[p]; c < pv.ce[p]; c++) { coff[p].push_back(off); off += st.r[c]; }
      nst.a[p] = off;
    }
    alloc_level(nst, pv);
    nst.Uraw.resize(pv.nb);
    nst.Vraw.resize(pv.nb);
    std::vector<CopyTask> cps;
    for (int p = 0; p < pv.nb; p++) {
      const int ap = nst.a[p];
      nst.Uraw[p] = nst.mem.alloc<double>((size_t)std::max(ap, 1) * nd);
      nst.Vraw[p] = nst.mem.alloc<double>((size_t)std::max(ap, 1) * nd);
      for (int c = pv.cb[p]; c < pv.ce[p]; c++) {
        const int o = coff[p][c - pv.cb[p]];
        cps.push_back(cp(st.Upar[c], st.rcap[c], nst.Uraw[p] + o, ap, st.r[c], nd));
        cps.push_back(cp(st.Vpar[c], st.rcap[c], nst.Vraw[p] + o, ap, st.r[c], nd));
      }
      for (int k = pv.nbr_ptr[p]; k < pv.nbr_ptr[p + 1]; k++) {
        const int q = pv.nbr[k];
        double* Xpq = nst.X[k];
        for (int c = pv.cb[p]; c < pv.ce[p]; c++)
          for (int d = pv.cb[q]; d < pv.ce[q]; d++) {
            const int oc = coff[p][c - pv.cb[p]], od = coff[q][d - pv.cb[q]];
            cps.push_back(cp(Y(st, lv, c, d), st.rcap[c], Xpq + oc + (size_t)od * ap, ap, st.r[c], st.r[d]));
          }
      }
    }
    scratch.reset();
    run_copies(scratch, cps, s);
    CK(cudaStreamSynchronize(s));
    scratch.reset();
  }

  void top(FLevel& st, const LevelTopo& lv) {
    std::vector<int> off(st.nb + 1, 0);
    for (int i = 0; i < st.nb; i++) off[i + 1] = off[i] + st.r[i];
    const int n = off[st.nb];
    f->top_n = n;
    f->info.top_size = n;
    if (n == 0) return;
    f->top_LU = f->store.alloc<double>((size_t)n * n);
    f->top_piv = f->store.alloc<int>(n);
    f->top_info = f->store.alloc<int>(1);
    std::vector<CopyTask> cps;
    for (int i = 0; i < st.nb; i++)
      for (int j = 0; j < st.nb; j++) {
        const int k = lv.yslot(i, j);
        if (k < 0) throw Error(IFMM_ERR_CUDA, "internal: top system is not dense");
        cps.push_back(cp(st.Y[k], st.rcap[i], f->top_LU + off[i] + (size_t)off[j] * n, n, st.r[i], st.r[j]));
      }
    scratch.reset();
    run_copies(scratch, cps, s);
    double* amax = scratch.alloc<double>(1);
    run_getrf(scratch, {LuTask{f->top_LU, n, n, f->top_piv, f->top_info, amax}}, s);
    f->info.flops_top += 2.0 / 3.0 * n * (double)n * n;
    CK(cudaStreamSynchronize(s));
  }

  void run() {
    const ifmm_options& o = sys->opt;
    auto t0 = Clock::now();
    const int L = sys->L;
    f->info.levels = L;
    d_counters = f->store.alloc<int>(4);
    CK(cudaMemsetAsync(d_counters, 0, 4 * sizeof(int), s));
    if (L == 0) {  // no tree: one dense LU of A
      const int N = (int)sys->N;
      f->dense_LU = f->store.alloc<double>((size_t)N * N);
      f->dense_piv = f->store.alloc<int>(N);
      f->dense_info = f->store.alloc<int>(1);
      P2PTask t{0, N, 0, N, 0};
      const P2PTask* d = upload(scratch, std::vector<P2PTask>{t}, s);
      launch_p2p_blocks(sys->ks, sys->dim, sys->pts_tree, d, 1, f->dense_LU, s);
      double* amax = scratch.alloc<double>(1);
      run_getrf(scratch, {LuTask{f->dense_LU, N, N, f->dense_piv, f->dense_info, amax}}, s);
      CK(cudaStreamSynchronize(s));
      f->info.flops_top = 2.0 / 3.0 * N * (double)N * N;
      f->info.seconds_top = since(t0);
      return;
    }
    if (o.tau_override > 0.0) {
      tau = o.tau_override;
    } else if (o.eps == 0.0) {
      tau = 0.0;
    } else {
      auto ts = Clock::now();
      if (std::isnan(sys->sigma0)) sys->sigma0 = system_sigma0(sys, s, &sys->sigma0_iters);
      f->info.seconds_sigma0 = since(ts);
      TRACE("[ifmm] sigma0 = %.6g (%d iterations), %.3f s\n", sys->sigma0, sys->sigma0_iters,
            f->info.seconds_sigma0);
      tau = o.eps * sys->sigma0;
    }
    f->info.sigma0 = sys->sigma0;
    f->info.sigma0_iters = sys->sigma0_iters;
    f->info.tau = tau;
    rsvd_rows = o.rsvd_rows > 0 ? o.rsvd_rows : RSVD_ROWS_DEFAULT;
    cap_global = o.rank_cap > 0 ? o.rank_cap : (tau == 0.0 ? (1 << 30) : nd);
    f->rank.assign(L + 1, {});
    f->yoff.assign(L + 1, {});
    auto st = std::make_unique<FLevel>();
    const LevelTopo& leaf = sys->lv[L];
    st->a.resize(leaf.nb);
    for (int i = 0; i < leaf.nb; i++) st->a[i] = leaf.p1[i] - leaf.p0[i];
    alloc_level(*st, leaf);
    // X blocks of the leaves are the near-field blocks (same slot order and ld)
    {
      long long tot = 0;
      for (int i = 0; i < leaf.nb; i++)
        for (int k = leaf.nbr_ptr[i]; k < leaf.nbr_ptr[i + 1]; k++)
          tot += (long long)st->a[i] * st->a[leaf.nbr[k]];
      if (tot > 0)
        CK(cudaMemcpyAsync(st->X[0], sys->p2p, tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    st->Uraw.resize(leaf.nb);
    st->Vraw.resize(leaf.nb);
    for (int i = 0; i < leaf.nb; i++) st->Uraw[i] = st->Vraw[i] = ops.leafU + ops.uoff[i];
    for (int l = L; l >= 2; l--) {
      const LevelTopo& lv = sys->lv[l];
      auto ti = Clock::now();
      init_basis(*st, lv);
      f->info.seconds_init += since(ti);
      if (tracing()) {
        int amax = 0, rmax = 0;
        double rs = 0;
        for (int i = 0; i < lv.nb; i++) { amax = std::max(amax, st->a[i]); rmax = std::max(rmax, st->r[i]); rs += st->r[i]; }
        TRACE("[ifmm] level %d init: %d boxes, max a %d, max r %d, avg r %.1f, %.3f s\n", l, lv.nb,
              amax, rmax, rs / std::max(lv.nb, 1), since(ti));
      }
      auto te = Clock::now();
      int ncol = 1;
      for (int d = 0; d < dim; d++) ncol *= 3;
      for (int c = 0; c < ncol; c++) {
        std::vector<int> boxes;
        for (int i = 0; i < lv.nb; i++)
          if (lv.colour[i] == c) boxes.push_back(i);
        if (boxes.empty()) continue;
        auto tc = Clock::now();
        eliminate_colour(*st, lv, boxes);
        if (tracing()) {
          CK(cudaStreamSynchronize(s));
          int amax = 0, rmax = 0;
          for (int i : boxes) { amax = std::max(amax, st->a[i]); rmax = std::max(rmax, st->r[i]); }
          TRACE("[ifmm] level %d colour %2d: %4zu boxes, max a %d, max r %d, %.3f s\n", l, c,
                boxes.size(), amax, rmax, since(tc));
        }
      }
      CK(cudaStreamSynchronize(s));
      f->info.seconds_elim += since(te);
      f->rank[l] = st->r;
      f->yoff[l].assign(lv.nb + 1, 0);
      for (int i = 0; i < lv.nb; i++) f->yoff[l][i + 1] = f->yoff[l][i] + st->r[i];
      int mx = 0;
      double av = 0.0;
      for (int v : st->r) { mx = std::max(mx, v); av += v; }
      if (l < 32) {
        f->info.max_rank[l] = mx;
        f->info.avg_rank[l] = lv.nb ? av / lv.nb : 0.0;
      }
      if (l > 2) {
        auto tm = Clock::now();
        auto nst = std::make_unique<FLevel>();
        merge(*st, lv, *nst, sys->lv[l - 1]);
        st = std::move(nst);
        f->info.seconds_elim += since(tm);
        TRACE("[ifmm] merge %d -> %d: %.3f s\n", l, l - 1, since(tm));
      }
    }
    auto tt = Clock::now();
    top(*st, sys->lv[2]);
    f->info.seconds_top = since(tt);
    TRACE("[ifmm] top: n = %d, %.3f s\n", f->top_n, f->info.seconds_top);
    std::vector<int> cnt = read_ints(d_counters, 4);
    f->info.rank_capped = cnt[0];
    if (cnt[1] != 0)
      throw Error(IFMM_ERR_TIMEOUT, "tensor-core Schur product: a bounded wait ran out");
  }
};

ifmm_factorization* factor_create(ifmm_system* sys, cudaStream_t s) {
  auto* f = new ifmm_factorization();
  f->sys = sys;
  try {
    Factorizer fz(sys, f, s);
    fz.run();
    // singular pivot tests: count the failed blocks in one reduction
    std::vector<const int*> flags;
    for (const FRec& R : f->recs) flags.push_back(R.info);
    for (int* p : {f->top_info, f->dense_info})
      if (p) flags.push_back(p);
    int sing = 0;
    if (!flags.empty()) {
      Arena tmp;
      int* d_count = tmp.alloc<int>(1);
      launch_count_nonzero(upload(tmp, flags, s), (int)flags.size(), d_count, s);
      CK(cudaMemcpyAsync(&sing, d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    f->info.singular_pivots = sing;
    if (sing > 0 && tracing()) {  // which pivot blocks failed, and at which column
      for (const FRec& R : f->recs) {
        int v = 0;
        CK(cudaMemcpy(&v, R.info, sizeof(int), cudaMemcpyDeviceToHost));
        if (v != 0)
          TRACE("[ifmm] singular pivot: level %d box %d (a %d, r %d, p %d) at column %d\n", R.l,
                R.i, R.a, R.r, R.p, v);
      }
      for (int* p : {f->top_info, f->dense_info}) {
        int v = 0;
        if (p) CK(cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost));
        if (v != 0) TRACE("[ifmm] singular pivot in the top / dense LU at column %d\n", v);
      }
    }
    f->info.factor_bytes = (long long)f->store.held;
    return f;
  } catch (...) {
    delete f;
    throw;
  }
}

}  // namespace ifmm
