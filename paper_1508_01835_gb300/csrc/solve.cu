// solve.cu -- substitution phase of the IFMM (the downward pass of Algorithm 1).
//
// Forward sweep in elimination order: for every eliminated box,
//   w = E(P,P)^-1 [b_xtilde_i ; 0] = W b_i,  b_R -= E(R,P) w = F b_i
// (the right-hand-side update of Algorithm 1); then the top dense
// solve for y^(2); then the backward sweep in reverse order:
//   x_P = w - G x_C,  G = E(P,P)^-1 E(P,C),
// of which only the xtilde_i rows are needed: x_i = w[0:a] - Ga x_C.  The
// unknowns xtilde^(l) of depth l < L are the multipoles ybar^(l+1) of the
// children (Eq. y_merge), so they share storage: the children of a box are
// consecutive in Morton order.  Boxes of one colour have disjoint neighbour
// lists, so each colour's forward step (w of every box and every b_R update)
// is one launch of block-row products, and so is its backward step.
#include "factor.cuh"

namespace ifmm {

static void build_plan(ifmm_factorization* f, SolvePlan& P, int nrhs, cudaStream_t s) {
  P.graph.reset();
  P.steps.clear();
  P.mem.release();
  P.task_mem.release();
  P.cap = nrhs;
  ifmm_system* sys = f->sys;
  const long long N = sys->N;
  const int L = sys->L;
  P.xt = P.mem.alloc<double>((size_t)N * nrhs);
  if (L == 0) return;
  P.ybar.assign(L + 2, nullptr);
  P.nybar.assign(L + 2, 0);
  for (int l = 2; l <= L; l++) {
    P.nybar[l] = f->yoff[l].back();
    P.ybar[l] = P.mem.alloc<double>((size_t)std::max(P.nybar[l], 1ll) * nrhs);
  }
  P.w.resize(f->recs.size());
  for (size_t k = 0; k < f->recs.size(); k++)
    P.w[k] = P.mem.alloc<double>((size_t)std::max(f->recs[k].p, 1) * nrhs);
  auto xt_seg = [&](int l, int box, long long& ld) -> double* {
    if (l == L) { ld = N; return P.xt + sys->lv[L].p0[box]; }
    ld = P.nybar[l + 1];
    return P.ybar[l + 1] + f->yoff[l + 1][sys->lv[l].cb[box]];
  };
  auto yb_seg = [&](int l, int box, long long& ld) -> double* {
    ld = P.nybar[l];
    return P.ybar[l] + f->yoff[l][box];
  };
  auto seg = [&](int l, const BlockRef& b, long long& ld) {
    return b.kind == 'x' ? xt_seg(l, b.box, ld) : yb_seg(l, b.box, ld);
  };
  // groups of records with the same (level, colour), in elimination order
  std::vector<std::pair<size_t, size_t>> groups;
  for (size_t k = 0; k < f->recs.size();) {
    size_t e = k;
    while (e < f->recs.size() && f->recs[e].l == f->recs[k].l &&
           f->recs[e].colour == f->recs[k].colour)
      e++;
    groups.push_back({k, e});
    k = e;
  }
  auto add_spmm = [&](std::vector<SpRow>& rows, std::vector<SpEnt>& ents) {
    if (rows.empty()) return;
    SolvePlan::Step st;
    st.kind = 2;
    st.sp = plan_spmm(P.task_mem, rows, ents, nrhs, s);
    P.steps.push_back(std::move(st));
  };
  for (auto& g : groups) {  // forward: w = W b_i, b_R -= F b_i
    std::vector<SpRow> rows;
    std::vector<SpEnt> ents;
    for (size_t k = g.first; k < g.second; k++) {
      const FRec& R = f->recs[k];
      long long ldb;
      const double* bi = xt_seg(R.l, R.i, ldb);
      rows.push_back({P.w[k], R.p, R.p, (int)ents.size(), 0, 0.0});
      if (R.a > 0) {
        ents.push_back({R.W, bi, ldb, R.p, R.a, 0, 1.0});
        rows.back().ne++;
      }
      for (const BlockRef& b : R.blk) {
        long long ld;
        double* y = seg(R.l, b, ld);
        rows.push_back({y, ld, b.dim, (int)ents.size(), 0, 1.0});
        if (R.a > 0) {
          ents.push_back({R.F + b.off, bi, ldb, R.nC, R.a, 0, -1.0});
          rows.back().ne++;
        }
      }
    }
    add_spmm(rows, ents);
  }
  if (f->top_n > 0) {  // top dense solve for ybar^(2)
    SolvePlan::Step rs;
    rs.kind = 1;
    rs.rs = plan_getrs(P.task_mem,
                       {RsTask{f->top_LU, f->top_n, f->top_n, f->top_piv, P.ybar[2], f->top_n, nrhs}},
                       s);
    P.steps.push_back(std::move(rs));
  }
  for (auto it = groups.rbegin(); it != groups.rend(); ++it) {  // backward: x_i = w - Ga x_C
    std::vector<SpRow> rows;
    std::vector<SpEnt> ents;
    for (size_t k = it->first; k < it->second; k++) {
      const FRec& R = f->recs[k];
      if (R.a == 0) continue;
      long long ldx;
      double* xs = xt_seg(R.l, R.i, ldx);
      rows.push_back({xs, ldx, R.a, (int)ents.size(), 1, 0.0});
      ents.push_back({nullptr, P.w[k], R.p, 1, R.a, 0, 1.0});  // identity: w[0:a]
      for (const BlockRef& b : R.blk) {
        long long ld;
        const double* x = seg(R.l, b, ld);
        ents.push_back({R.Ga + (size_t)b.off * R.a, x, ld, R.a, b.dim, 0, -1.0});
        rows.back().ne++;
      }
    }
    add_spmm(rows, ents);
  }
  CK(cudaStreamSynchronize(s));
}

void factor_solve(ifmm_factorization* f, const double* b, long long ldb, double* x,
                  long long ldx, int nrhs, cudaStream_t s) {
  if (nrhs <= 0) return;
  ifmm_system* sys = f->sys;
  const long long N = sys->N;
  std::unique_ptr<SolvePlan>& slot = f->plans[nrhs];
  if (!slot) {
    CK(cudaStreamSynchronize(s));
    auto P = std::make_unique<SolvePlan>();
    build_plan(f, *P, nrhs, s);
    slot = std::move(P);
  }
  SolvePlan& P = *slot;
  launch_gather_rows(sys->perm, N, b, ldb, P.xt, N, nrhs, s);
  if (sys->L == 0) {
    Arena tmp;
    run_getrs(tmp, {RsTask{f->dense_LU, (int)N, (int)N, f->dense_piv, P.xt, (int)N, nrhs}}, s);
    launch_scatter_rows(sys->perm, N, P.xt, N, x, ldx, nrhs, s);
    CK(cudaStreamSynchronize(s));
    return;
  }
  run_graph(P.graph, nrhs, "graph:ifmm_solve", s, [&](cudaStream_t gs) {
    for (int l = 2; l <= sys->L; l++)
      CK(cudaMemsetAsync(P.ybar[l], 0, sizeof(double) * std::max(P.nybar[l], 1ll) * nrhs, gs));
    for (const SolvePlan::Step& st : P.steps) {
      if (st.kind == 0) launch_copy(st.copies, st.ncopies, gs);
      else if (st.kind == 2) launch_spmm(st.sp, nrhs, gs);
      else exec_getrs(st.rs, gs);
    }
  });
  launch_scatter_rows(sys->perm, N, P.xt, N, x, ldx, nrhs, s);
}

// ---------------------------------------------------------------------------
// FP32 substitution (the preconditioner of flexible GMRES in reduced
// precision): the same steps with FP32 blocks, the top system solved with
// its explicit inverse (one product instead of a chain of triangular panels).
// ---------------------------------------------------------------------------
void factor_prepare_f32(ifmm_factorization* f, cudaStream_t s) {
  F32Data& D = f->f32;
  if (D.ready) return;
  ifmm_system* sys = f->sys;
  Arena scratch;
  std::vector<NarrowTask> nt;
  const size_t nr = f->recs.size();
  D.W.assign(nr, nullptr);
  D.F.assign(nr, nullptr);
  D.Ga.assign(nr, nullptr);
  for (size_t k = 0; k < nr; k++) {
    const FRec& R = f->recs[k];
    const long long a = std::max(R.a, 1);
    float* W = D.mem.alloc<float>((size_t)R.p * a);
    float* F = D.mem.alloc<float>((size_t)R.nC * a);
    float* Ga = D.mem.alloc<float>((size_t)a * R.nC);
    nt.push_back({R.W, W, (long long)R.p * R.a});
    nt.push_back({R.F, F, (long long)R.nC * R.a});
    nt.push_back({R.Ga, Ga, (long long)R.a * R.nC});
    D.W[k] = W;
    D.F[k] = F;
    D.Ga[k] = Ga;
  }
  // inverse of the top system (or of the dense system when there is no tree)
  const int n = sys->L == 0 ? (int)sys->N : f->top_n;
  const double* LU = sys->L == 0 ? f->dense_LU : f->top_LU;
  const int* piv = sys->L == 0 ? f->dense_piv : f->top_piv;
  if (n > 0) {
    double* inv = scratch.alloc<double>((size_t)n * n);
    CK(cudaMemsetAsync(inv, 0, sizeof(double) * (size_t)n * n, s));
    std::vector<CopyTask> eye{CopyTask{nullptr, inv, nullptr, 1, n, n, n, 0, 1, 1.0, 0.0}};
    validate(eye[0]);
    launch_copy(upload(scratch, eye, s), 1, s);
    run_getrs(scratch, {RsTask{LU, n, n, piv, inv, n, n}}, s);
    float* ti = D.mem.alloc<float>((size_t)n * n);
    nt.push_back({inv, ti, (long long)n * n});
    D.top_inv = ti;
  }
  launch_narrow(scratch, nt, s);
  CK(cudaStreamSynchronize(s));
  D.ready = true;
}

static void build_plan32(ifmm_factorization* f, SolvePlan32& P, int nrhs, cudaStream_t s) {
  P.graphs.reset();
  P.steps.clear();
  P.mem.release();
  P.task_mem.release();
  P.cap = nrhs;
  const F32Data& D = f->f32;
  ifmm_system* sys = f->sys;
  const long long N = sys->N;
  const int L = sys->L;
  P.xt = P.mem.alloc<float>((size_t)N * nrhs);
  auto add = [&](std::vector<SpRowF>& rows, std::vector<SpEntF>& ents) {
    if (!rows.empty()) P.steps.push_back(plan_spmm_f32(P.task_mem, rows, ents, nrhs, s));
    rows.clear();
    ents.clear();
  };
  std::vector<SpRowF> rows;
  std::vector<SpEntF> ents;
  if (L == 0) {  // x = A^-1 b with the explicit inverse
    P.xt2 = P.mem.alloc<float>((size_t)N * nrhs);
    rows.push_back({P.xt2, N, (int)N, 0, 1, 0.0f});
    ents.push_back({D.top_inv, P.xt, N, (int)N, (int)N, 1.0f});
    add(rows, ents);
    CK(cudaStreamSynchronize(s));
    return;
  }
  P.ybar.assign(L + 2, nullptr);
  P.nybar.assign(L + 2, 0);
  for (int l = 2; l <= L; l++) {
    P.nybar[l] = f->yoff[l].back();
    P.ybar[l] = P.mem.alloc<float>((size_t)std::max(P.nybar[l], 1ll) * nrhs);
  }
  P.w.resize(f->recs.size());
  for (size_t k = 0; k < f->recs.size(); k++)
    P.w[k] = P.mem.alloc<float>((size_t)std::max(f->recs[k].p, 1) * nrhs);
  auto xt_seg = [&](int l, int box, long long& ld) -> float* {
    if (l == L) { ld = N; return P.xt + sys->lv[L].p0[box]; }
    ld = P.nybar[l + 1];
    return P.ybar[l + 1] + f->yoff[l + 1][sys->lv[l].cb[box]];
  };
  auto seg = [&](int l, const BlockRef& b, long long& ld) -> float* {
    if (b.kind == 'x') return xt_seg(l, b.box, ld);
    ld = P.nybar[l];
    return P.ybar[l] + f->yoff[l][b.box];
  };
  std::vector<std::pair<size_t, size_t>> groups;
  for (size_t k = 0; k < f->recs.size();) {
    size_t e = k;
    while (e < f->recs.size() && f->recs[e].l == f->recs[k].l &&
           f->recs[e].colour == f->recs[k].colour)
      e++;
    groups.push_back({k, e});
    k = e;
  }
  for (auto& g : groups) {  // forward: w = W b_i, b_R -= F b_i
    for (size_t k = g.first; k < g.second; k++) {
      const FRec& R = f->recs[k];
      long long ldb;
      const float* bi = xt_seg(R.l, R.i, ldb);
      rows.push_back({P.w[k], R.p, R.p, (int)ents.size(), 0, 0.0f});
      if (R.a > 0) {
        ents.push_back({D.W[k], bi, ldb, R.p, R.a, 1.0f});
        rows.back().ne++;
      }
      for (const BlockRef& b : R.blk) {
        long long ld;
        float* y = seg(R.l, b, ld);
        rows.push_back({y, ld, b.dim, (int)ents.size(), 0, 1.0f});
        if (R.a > 0) {
          ents.push_back({D.F[k] + b.off, bi, ldb, R.nC, R.a, -1.0f});
          rows.back().ne++;
        }
      }
    }
    add(rows, ents);
  }
  if (f->top_n > 0) {  // ybar^(2) = T^-1 ybar^(2), through a copy
    const int n = f->top_n;
    P.top_tmp = P.mem.alloc<float>((size_t)n * nrhs);
    rows.push_back({P.top_tmp, n, n, 0, 1, 0.0f});
    ents.push_back({nullptr, P.ybar[2], n, 1, n, 1.0f});
    add(rows, ents);
    rows.push_back({P.ybar[2], n, n, 0, 1, 0.0f});
    ents.push_back({D.top_inv, P.top_tmp, n, n, n, 1.0f});
    add(rows, ents);
  }
  for (auto it = groups.rbegin(); it != groups.rend(); ++it) {  // backward: x_i = w - Ga x_C
    for (size_t k = it->first; k < it->second; k++) {
      const FRec& R = f->recs[k];
      if (R.a == 0) continue;
      long long ldx;
      float* xs = xt_seg(R.l, R.i, ldx);
      rows.push_back({xs, ldx, R.a, (int)ents.size(), 1, 0.0f});
      ents.push_back({nullptr, P.w[k], R.p, 1, R.a, 1.0f});
      for (const BlockRef& b : R.blk) {
        long long ld;
        const float* x = seg(R.l, b, ld);
        ents.push_back({D.Ga[k] + (size_t)b.off * R.a, x, ld, R.a, b.dim, -1.0f});
        rows.back().ne++;
      }
    }
    add(rows, ents);
  }
  CK(cudaStreamSynchronize(s));
}

constexpr int PLAN32_COLS = 32;

static SolvePlan32& plan32_for(ifmm_factorization* f, int nrhs, cudaStream_t s) {
  const int cap = std::max(nrhs, PLAN32_COLS);
  std::unique_ptr<SolvePlan32>& slot = f->plans32[cap];
  if (!slot) {
    CK(cudaStreamSynchronize(s));
    factor_prepare_f32(f, s);
    auto P = std::make_unique<SolvePlan32>();
    build_plan32(f, *P, cap, s);
    slot = std::move(P);
  }
  return *slot;
}

void factor_prepare_plans_f32(ifmm_factorization* f, int max_cols, cudaStream_t s) {
  plan32_for(f, max_cols, s);
}

void factor_solve_f32(ifmm_factorization* f, const double* b, long long ldb, double* x,
                      long long ldx, int nrhs, cudaStream_t s) {
  if (nrhs <= 0) return;
  ifmm_system* sys = f->sys;
  const long long N = sys->N;
  SolvePlan32& P = plan32_for(f, nrhs, s);
  launch_gather_rows_f32(sys->perm, N, b, ldb, P.xt, N, nrhs, s);
  run_graph(P.graphs.at(nrhs), nrhs, "graph:ifmm_solve_f32", s, [&](cudaStream_t gs) {
    for (int l = 2; l <= sys->L; l++)
      CK(cudaMemsetAsync(P.ybar[l], 0, sizeof(float) * std::max(P.nybar[l], 1ll) * nrhs, gs));
    for (const SpmmPlanF& st : P.steps) launch_spmm_f32(st, nrhs, gs);
  });
  launch_scatter_rows_f32(sys->perm, N, sys->L == 0 ? P.xt2 : P.xt, N, x, ldx, nrhs, s);
}

}  // namespace ifmm
