// solve.cu -- substitution phase of the IFMM (the downward pass of Algorithm 1).
//
// Forward sweep in elimination order: for every eliminated box,
//   w = E(P,P)^-1 [b_xtilde_i ; 0],  b_R -= E(R,P) w
// (the right-hand-side update of Algorithm 1); then the top dense
// solve for y^(2); then the backward sweep in reverse order:
//   x_P = w - G x_C,  G = E(P,P)^-1 E(P,C),
// which recovers xtilde_i (and z_i).  The unknowns xtilde^(l) of depth l < L
// are the multipoles ybar^(l+1) of the children (Eq. y_merge), so they share
// storage: the children of a box are consecutive in Morton order.
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
  auto add_copies = [&](std::vector<CopyTask>& v) {
    SolvePlan::Step st;
    st.kind = 0;
    std::vector<CopyTask> keep;
    for (auto& c : v)
      if (c.rows > 0 && c.cols > 0) {
        validate(c);
        keep.push_back(c);
      }
    st.ncopies = (int)keep.size();
    st.copies = upload(P.task_mem, keep, s);
    if (st.ncopies) P.steps.push_back(std::move(st));
  };
  auto add_spmm = [&](std::vector<SpRow>& rows, std::vector<SpEnt>& ents) {
    if (rows.empty()) return;
    SolvePlan::Step st;
    st.kind = 2;
    st.sp = plan_spmm(P.task_mem, rows, ents, nrhs, s);
    P.steps.push_back(std::move(st));
  };
  for (auto& g : groups) {  // forward
    std::vector<CopyTask> cps;
    SolvePlan::Step rs;
    rs.kind = 1;
    std::vector<RsTask> rst;
    std::vector<SpRow> rows;
    std::vector<SpEnt> ents;
    for (size_t k = g.first; k < g.second; k++) {
      const FRec& R = f->recs[k];
      long long ld;
      double* xs = xt_seg(R.l, R.i, ld);
      cps.push_back({xs, P.w[k], nullptr, (int)ld, R.p, R.a, nrhs, 0, 0, 1.0, 0.0});
      cps.push_back({nullptr, P.w[k] + R.a, nullptr, 1, R.p, R.r, nrhs, 0, 2, 0.0, 0.0});
      rst.push_back({R.LU, R.p, R.p, R.piv, P.w[k], R.p, nrhs});
      for (const BlockRef& b : R.blk) {
        double* y = seg(R.l, b, ld);
        rows.push_back({y, ld, b.dim, (int)ents.size(), 1, 1.0});
        ents.push_back({R.ERP + b.off, P.w[k], R.p, R.nC, R.p, 0, -1.0});
      }
    }
    add_copies(cps);
    rs.rs = plan_getrs(P.task_mem, rst, s);
    P.steps.push_back(std::move(rs));
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
  for (auto it = groups.rbegin(); it != groups.rend(); ++it) {  // backward
    std::vector<SpRow> rows;
    std::vector<SpEnt> ents;
    std::vector<CopyTask> cps;
    for (size_t k = it->first; k < it->second; k++) {
      const FRec& R = f->recs[k];
      rows.push_back({P.w[k], R.p, R.p, (int)ents.size(), 0, 1.0});
      for (const BlockRef& b : R.blk) {
        long long ld;
        const double* x = seg(R.l, b, ld);
        ents.push_back({R.G + (size_t)b.off * R.p, x, ld, R.p, b.dim, 0, -1.0});
        rows.back().ne++;
      }
      long long ld;
      double* xs = xt_seg(R.l, R.i, ld);
      cps.push_back({P.w[k], xs, nullptr, R.p, (int)ld, R.a, nrhs, 0, 0, 1.0, 0.0});
    }
    add_spmm(rows, ents);
    add_copies(cps);
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

}  // namespace ifmm
