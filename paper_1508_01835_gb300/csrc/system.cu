// system.cu -- tree topology, raw H^2 operators, FMM matvec and sigma_0(E).
//
// Sec. 2.1: A = S + U K V^T applied level by level (Eqs. A_decomp_l3,
// A_decomp_l2); the FMM matvec evaluates it as P2M -> M2M -> M2L/L2L -> L2P
// plus P2P.  Sec. 2.4: sigma_0(E) of the extended sparse matrix E of
// Eq. (Ax=b_extended) scales the truncation threshold.
#include <cmath>

#include "system.cuh"

namespace ifmm {

static ChebSpec make_cheb(int n, int dim) {
  ChebSpec c{};
  c.n = n;
  c.nd = 1;
  for (int d = 0; d < dim; d++) c.nd *= n;
  for (int a = 1; a <= n; a++) c.t[a - 1] = std::cos(((2.0 * a - 1.0) * M_PI) / (2.0 * n));
  return c;
}

static void build_ops(ifmm_system* sys, int n, ChebOps& ops, cudaStream_t s) {
  ops.n = n;
  ops.spec = make_cheb(n, sys->dim);
  ops.nd = ops.spec.nd;
  const int nd = ops.nd, dim = sys->dim;
  ops.transfer = sys->mem.alloc<double>((size_t)(1 << dim) * nd * nd);
  launch_transfer(ops.spec, dim, ops.transfer, s);
  ops.m2l.assign(sys->L + 1, nullptr);
  int no = 1;
  for (int d = 0; d < dim; d++) no *= 7;
  for (int l = 2; l <= sys->L; l++) {
    ops.m2l[l] = sys->mem.alloc<double>((size_t)no * nd * nd);
    launch_m2l_table(ops.spec, dim, sys->ks, sys->lv[l].h, ops.m2l[l], s);
  }
  const LevelTopo& leaf = sys->lv[sys->L];
  ops.uoff.assign(leaf.nb, 0);
  long long tot = 0;
  std::vector<LeafGeom> g(leaf.nb);
  for (int i = 0; i < leaf.nb; i++) {
    ops.uoff[i] = tot;
    g[i].p0 = leaf.p0[i];
    g[i].p1 = leaf.p1[i];
    g[i].uoff = tot;
    g[i].h = leaf.h;
    for (int d = 0; d < 3; d++)
      g[i].centre[d] = d < dim ? sys->lo[d] + (2.0 * leaf.coords[i * 3 + d] + 1.0) * leaf.h : 0.0;
    tot += (long long)(leaf.p1[i] - leaf.p0[i]) * nd;
  }
  ops.leafU = sys->mem.alloc<double>(tot);
  Arena tmp;
  const LeafGeom* dg = upload(tmp, g, s);
  launch_leaf_interp(ops.spec, dim, sys->pts_tree, dg, leaf.nb, ops.leafU, s);
  CK(cudaStreamSynchronize(s));
}

static void build_topology(ifmm_system* sys, const TreeOut& T, cudaStream_t s) {
  const int dim = sys->dim, L = T.L;
  std::vector<std::vector<int>> nbr, far;
  build_lists_device(T.keys, dim, nbr, far, s);
  sys->lv.assign(L + 1, LevelTopo{});
  for (int l = 0; l <= L; l++) {
    LevelTopo& v = sys->lv[l];
    v.l = l;
    v.nb = (int)T.keys[l].size();
    v.h = sys->edge / (double)(1ll << (l + 1));
    v.coords.assign((size_t)v.nb * 3, 0);
    v.colour.assign(v.nb, 0);
    for (int i = 0; i < v.nb; i++) {
      int c[3] = {0, 0, 0};
      morton_decode_host(T.keys[l][i], dim, c);
      int col = 0, w = 1;
      for (int d = 0; d < 3; d++) {
        v.coords[i * 3 + d] = c[d];
        if (d < dim) { col += (c[d] % 3) * w; w *= 3; }
      }
      v.colour[i] = col;
    }
    v.nbr_ptr.assign(v.nb + 1, 0);
    v.far_ptr.assign(v.nb + 1, 0);
    v.yl_ptr.assign(v.nb + 1, 0);
    for (int i = 0; i < v.nb; i++) {
      std::vector<int> a, b;
      for (int k = 0; k < 27; k++)
        if (nbr[l][i * 27 + k] >= 0) a.push_back(nbr[l][i * 27 + k]);
      for (int k = 0; k < 189; k++)
        if (far[l][i * 189 + k] >= 0) b.push_back(far[l][i * 189 + k]);
      for (int q : a)
        if (q >= v.nb) throw Error(IFMM_ERR_CUDA, "internal: neighbour index out of range");
      for (int q : b)
        if (q >= v.nb) throw Error(IFMM_ERR_CUDA, "internal: interaction index out of range");
      if (std::find(a.begin(), a.end(), i) == a.end())
        throw Error(IFMM_ERR_CUDA, "internal: a box is missing from its own neighbour list");
      std::sort(a.begin(), a.end());
      std::sort(b.begin(), b.end());
      std::vector<int> u(a);
      u.insert(u.end(), b.begin(), b.end());
      std::sort(u.begin(), u.end());
      v.nbr.insert(v.nbr.end(), a.begin(), a.end());
      v.far.insert(v.far.end(), b.begin(), b.end());
      v.yl.insert(v.yl.end(), u.begin(), u.end());
      v.nbr_ptr[i + 1] = (int)v.nbr.size();
      v.far_ptr[i + 1] = (int)v.far.size();
      v.yl_ptr[i + 1] = (int)v.yl.size();
    }
  }
  for (int l = 1; l <= L; l++) {
    LevelTopo& v = sys->lv[l];
    LevelTopo& p = sys->lv[l - 1];
    v.parent.assign(v.nb, -1);
    p.cb.assign(p.nb, 0);
    p.ce.assign(p.nb, 0);
    int pi = 0;
    for (int i = 0; i < v.nb; i++) {
      const unsigned long long pk = T.keys[l][i] >> dim;
      while (T.keys[l - 1][pi] != pk) pi++;
      v.parent[i] = pi;
    }
    for (int i = v.nb - 1; i >= 0; i--) p.cb[v.parent[i]] = i;
    for (int i = 0; i < v.nb; i++) p.ce[v.parent[i]] = i + 1;
  }
  LevelTopo& leaf = sys->lv[L];
  leaf.cb.assign(leaf.nb, 0);
  leaf.ce.assign(leaf.nb, 0);
  leaf.p0.assign(leaf.nb, 0);
  leaf.p1.assign(leaf.nb, 0);
  for (int i = 0; i < leaf.nb; i++) {
    leaf.p0[i] = T.leaf_begin[i];
    leaf.p1[i] = (i + 1 < leaf.nb) ? T.leaf_begin[i + 1] : (int)sys->N;
    sys->max_leaf = std::max(sys->max_leaf, leaf.p1[i] - leaf.p0[i]);
  }
}

static void build_p2p(ifmm_system* sys, cudaStream_t s) {
  const LevelTopo& leaf = sys->lv[sys->L];
  std::vector<P2PTask> tasks;
  sys->p2p_off.assign(leaf.nbr.size(), 0);
  long long tot = 0;
  for (int i = 0; i < leaf.nb; i++)
    for (int k = leaf.nbr_ptr[i]; k < leaf.nbr_ptr[i + 1]; k++) {
      const int j = leaf.nbr[k];
      sys->p2p_off[k] = tot;
      tasks.push_back({leaf.p0[i], leaf.p1[i], leaf.p0[j], leaf.p1[j], tot});
      tot += (long long)(leaf.p1[i] - leaf.p0[i]) * (leaf.p1[j] - leaf.p0[j]);
    }
  sys->p2p = sys->mem.alloc<double>(tot);
  Arena tmp;
  const P2PTask* d = upload(tmp, tasks, s);
  launch_p2p_blocks(sys->ks, sys->dim, sys->pts_tree, d, (int)tasks.size(), sys->p2p, s);
  CK(cudaStreamSynchronize(s));
}

ifmm_system* system_create(ifmm_ctx* ctx, const double* pts, bool host, long long N,
                           const ifmm_kernel* k, const ifmm_options* opt, cudaStream_t s) {
  require(N >= 1, "N must be >= 1");
  require(k != nullptr && opt != nullptr, "kernel and options must be given");
  require(opt->dim == 2 || opt->dim == 3, "dim must be 2 or 3");
  require(opt->cheb_n >= 1 && opt->cheb_n <= 8, "cheb_n must be in 1..8");
  require(opt->fmm_n >= 0 && opt->fmm_n <= 8, "fmm_n must be in 0..8");
  require(opt->leaf_max >= 1, "leaf_max must be >= 1");
  require(opt->eps >= 0.0 && std::isfinite(opt->eps), "eps must be >= 0");
  require(opt->schur >= IFMM_P_FP64 && opt->schur <= IFMM_P_FP32, "unknown Schur precision");
  // BF16 keeps 8 significant bits: the products are accurate to ~4e-3, so the
  // option is offered only for loose tolerances
  require(opt->schur != IFMM_P_BF16 || opt->eps >= 1e-4,
          "BF16 Schur products need eps >= 1e-4");
  require(opt->rank_cap >= 0, "rank_cap must be >= 0");
  require(opt->symmetric == 0 || opt->symmetric == 1, "symmetric must be 0 or 1");
  require(opt->rsvd_rows >= 0 && opt->rsvd_rows <= 65536, "rsvd_rows must be in 0..65536");
  require(k->kind >= IFMM_K_INV_R && k->kind <= IFMM_K_PAPER_D, "unknown kernel kind");
  require(!(k->kind == IFMM_K_INV_R && std::isnan(k->diag)), "1/r kernel needs a diagonal");
  require(k->kind == IFMM_K_INV_R || k->param > 0.0, "kernel parameter must be > 0");
  require(N < (1ll << 31), "N must be < 2^31");
  auto* sys = new ifmm_system();
  try {
    sys->ctx = ctx;
    sys->N = N;
    sys->dim = opt->dim;
    sys->opt = *opt;
    sys->ks = {k->kind, k->param, std::isnan(k->diag) ? 1.0 : k->diag};
    const size_t pbytes = (size_t)N * opt->dim * sizeof(double);
    sys->pts_user = sys->mem.alloc<double>((size_t)N * opt->dim);
    CK(cudaMemcpyAsync(sys->pts_user, pts, pbytes,
                       host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    {
      std::vector<double> hp((size_t)N * opt->dim);
      CK(cudaMemcpyAsync(hp.data(), sys->pts_user, pbytes, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (double v : hp) require(std::isfinite(v), "points must be finite");
    }
    sys->perm = sys->mem.alloc<long long>(N);
    TreeOut T = build_tree_device(sys->pts_user, N, opt->dim, opt->leaf_max, sys->perm, s);
    sys->L = T.L;
    sys->edge = T.edge;
    for (int d = 0; d < 3; d++) sys->lo[d] = T.lo[d];
    sys->perm_h = T.perm;
    sys->pts_tree = sys->mem.alloc<double>((size_t)N * opt->dim);
    launch_permute_points(sys->perm, N, opt->dim, sys->pts_user, sys->pts_tree, s);
    if (sys->L == 0) {
      sys->max_leaf = (int)N;
      CK(cudaStreamSynchronize(s));
      return sys;
    }
    build_topology(sys, T, s);
    build_p2p(sys, s);
    build_ops(sys, opt->cheb_n, sys->ops_f, s);
    const int fn = opt->fmm_n > 0 ? opt->fmm_n : opt->cheb_n;
    sys->same_ops = (fn == opt->cheb_n);
    if (!sys->same_ops) build_ops(sys, fn, sys->ops_mv, s);
    build_static_lists(sys, s);
    CK(cudaStreamSynchronize(s));
    return sys;
  } catch (...) {
    delete sys;
    throw;
  }
}

// ---------------------------------------------------------------------------
// FMM matvec plan: P2M, M2M per level, M2L + L2L per level, L2P + P2P
// ---------------------------------------------------------------------------
// The nd x nd translations (M2M, M2L + L2L) run as uniform block rows when
// nd <= 64 (coefficient vectors then hold uniform_ndp(nd) entries per box);
// P2M, L2P and the near field as general block-row products.
static void make_padded_tables(ifmm_system* sys, ChebOps& ops, cudaStream_t s) {
  if (ops.transfer_pad) return;
  const int nd = ops.nd, dim = sys->dim, ndp = uniform_ndp(nd);
  const int nt = 1 << dim;
  int no = 1;
  for (int d = 0; d < dim; d++) no *= 7;
  ops.transfer_pad = sys->mem.alloc<double>((size_t)nt * nd * ndp);
  ops.transferT_pad = sys->mem.alloc<double>((size_t)nt * nd * ndp);
  launch_pad_tables<double>(ops.transfer, ops.transfer_pad, nt, nd, false, s);
  launch_pad_tables<double>(ops.transfer, ops.transferT_pad, nt, nd, true, s);
  ops.m2l_pad.assign(sys->L + 1, nullptr);
  for (int l = 2; l <= sys->L; l++) {
    ops.m2l_pad[l] = sys->mem.alloc<double>((size_t)no * nd * ndp);
    launch_pad_tables<double>(ops.m2l[l], ops.m2l_pad[l], no, nd, false, s);
  }
}

static void build_fmm_plan(ifmm_system* sys, int cap, cudaStream_t s) {
  sys->fmm_graphs.reset();
  sys->fmm_plan.phases.clear();
  sys->fmm_plan.mem.reset();
  sys->fmm_uni.clear();
  sys->fmm_order.clear();
  sys->fmm_ws.release();
  sys->fmm_cap = cap;
  ChebOps& ops = sys->same_ops ? sys->ops_f : sys->ops_mv;
  const int nd = ops.nd, L = sys->L, dim = sys->dim;
  const bool uni = uniform_supported(nd);
  const int ndp = uni ? uniform_ndp(nd) : nd;
  if (uni) make_padded_tables(sys, ops, s);
  const long long N = sys->N;
  sys->fmm_x = sys->fmm_ws.alloc<double>((size_t)N * cap);
  sys->fmm_y = sys->fmm_ws.alloc<double>((size_t)N * cap);
  std::vector<double*> mult(L + 1, nullptr), loc(L + 1, nullptr);
  std::vector<long long> ldl(L + 1, 0);
  for (int l = 2; l <= L; l++) {
    ldl[l] = (long long)sys->lv[l].nb * ndp;
    mult[l] = sys->fmm_ws.alloc<double>((size_t)ldl[l] * cap);
    loc[l] = sys->fmm_ws.alloc<double>((size_t)ldl[l] * cap);
    // padding rows are staged by the uniform kernel (never multiplied): keep them finite
    CK(cudaMemsetAsync(mult[l], 0, sizeof(double) * (size_t)ldl[l] * cap, s));
    CK(cudaMemsetAsync(loc[l], 0, sizeof(double) * (size_t)ldl[l] * cap, s));
  }
  const LevelTopo& leaf = sys->lv[L];
  SpBuild b;
  auto flush = [&] {
    if (b.rows.empty()) return;
    b.flush(sys->fmm_plan, s, cap);
    sys->fmm_order.push_back(0);
  };
  std::vector<UniRow<double>> urows;
  std::vector<UniEnt<double>> uents;
  auto urow = [&](double* y, long long ldy) { urows.push_back({y, ldy, (int)uents.size(), 0}); };
  auto uent = [&](const double* A, const double* x, long long ldx) {
    uents.push_back({A, x, ldx});
    urows.back().ne++;
  };
  auto uflush = [&] {
    sys->fmm_uni.push_back(plan_uniform<double>(sys->fmm_plan.mem, urows, uents, nd, cap, s));
    sys->fmm_order.push_back(1);
    urows.clear();
    uents.clear();
  };
  for (int i = 0; i < leaf.nb; i++) {  // P2M
    const int m = leaf.p1[i] - leaf.p0[i];
    b.row(mult[L] + (long long)i * ndp, ldl[L], nd);
    b.ent(ops.leafU + ops.uoff[i], m, m, 1, sys->fmm_x + leaf.p0[i], N);
  }
  flush();
  for (int l = L - 1; l >= 2; l--) {  // M2M
    const LevelTopo& v = sys->lv[l];
    const LevelTopo& c = sys->lv[l + 1];
    for (int p = 0; p < v.nb; p++) {
      if (uni) urow(mult[l] + (long long)p * ndp, ldl[l]);
      else b.row(mult[l] + (long long)p * ndp, ldl[l], nd);
      for (int ch = v.cb[p]; ch < v.ce[p]; ch++) {
        const size_t t = (size_t)c.child_pos(ch, dim) * nd;
        if (uni) uent(ops.transferT_pad + t * ndp, mult[l + 1] + (long long)ch * ndp, ldl[l + 1]);
        else b.ent(ops.transfer + t * nd, nd, nd, 1, mult[l + 1] + (long long)ch * ndp, ldl[l + 1]);
      }
    }
    if (uni) uflush();
    else flush();
  }
  for (int l = 2; l <= L; l++) {  // M2L + L2L
    const LevelTopo& v = sys->lv[l];
    for (int i = 0; i < v.nb; i++) {
      if (uni) urow(loc[l] + (long long)i * ndp, ldl[l]);
      else b.row(loc[l] + (long long)i * ndp, ldl[l], nd);
      for (int k = v.far_ptr[i]; k < v.far_ptr[i + 1]; k++) {
        const int q = v.far[k];
        const size_t t = (size_t)v.m2l_offset(i, q, dim) * nd;
        if (uni) uent(ops.m2l_pad[l] + t * ndp, mult[l] + (long long)q * ndp, ldl[l]);
        else b.ent(ops.m2l[l] + t * nd, nd, nd, 0, mult[l] + (long long)q * ndp, ldl[l]);
      }
      if (l > 2) {
        const size_t t = (size_t)v.child_pos(i, dim) * nd;
        const double* xp = loc[l - 1] + (long long)v.parent[i] * ndp;
        if (uni) uent(ops.transfer_pad + t * ndp, xp, ldl[l - 1]);
        else b.ent(ops.transfer + t * nd, nd, nd, 0, xp, ldl[l - 1]);
      }
    }
    if (uni) uflush();
    else flush();
  }
  for (int i = 0; i < leaf.nb; i++) {  // L2P + P2P
    const int m = leaf.p1[i] - leaf.p0[i];
    b.row(sys->fmm_y + leaf.p0[i], N, m);
    b.ent(ops.leafU + ops.uoff[i], m, nd, 0, loc[L] + (long long)i * ndp, ldl[L]);
    for (int k = leaf.nbr_ptr[i]; k < leaf.nbr_ptr[i + 1]; k++) {
      const int j = leaf.nbr[k];
      b.ent(sys->p2p + sys->p2p_off[k], m, leaf.p1[j] - leaf.p0[j], 0, sys->fmm_x + leaf.p0[j], N);
    }
  }
  flush();
  CK(cudaStreamSynchronize(s));
}

static void run_fmm_phases(const ifmm_system* sys, int nrhs, cudaStream_t s) {
  size_t a = 0, u = 0;
  for (int kind : sys->fmm_order) {
    if (kind == 0) launch_spmm(sys->fmm_plan.phases[a++], nrhs, s);
    else launch_uniform<double>(sys->fmm_uni[u++], nrhs, s);
  }
}

size_t system_fmm_bytes(const ifmm_system* sys, int cap) {
  if (sys->L == 0) return 0;
  const int nd = sys->mv().nd;
  const int ndp = uniform_supported(nd) ? uniform_ndp(nd) : nd;
  size_t b = 2 * sizeof(double) * (size_t)sys->N * cap;  // x, y in tree order
  size_t ents = 0;
  for (int l = 2; l <= sys->L; l++) {
    b += 2 * sizeof(double) * (size_t)sys->lv[l].nb * ndp * cap;  // multipoles, locals
    ents += sys->lv[l].far.size() + 2 * (size_t)sys->lv[l].nb;
  }
  ents += sys->lv[sys->L].nbr.size();
  return b + 64 * ents + (size_t(16) << 20);
}

size_t system_fmm_held(const ifmm_system* sys) {
  return sys->fmm_ws.held + sys->fmm_plan.mem.held + sys->f32.ops.held + sys->f32.ws.held;
}

void system_prepare_fmm(ifmm_system* sys, int cap, cudaStream_t s) {
  if (sys->L == 0 || cap <= sys->fmm_cap) return;
  CK(cudaStreamSynchronize(s));
  build_fmm_plan(sys, cap, s);
}

void system_matvec(ifmm_system* sys, int mode, const double* x, long long ldx, double* y,
                   long long ldy, int nrhs, cudaStream_t s) {
  if (nrhs <= 0) return;
  if (mode == IFMM_MV_DIRECT || sys->L == 0) {
    launch_direct(sys->ks, sys->dim, sys->pts_user, sys->N, x, ldx, y, ldy, nrhs, s);
    return;
  }
  if (nrhs > sys->fmm_cap) {
    CK(cudaStreamSynchronize(s));
    build_fmm_plan(sys, std::max(nrhs, 4), s);
  }
  launch_gather_rows(sys->perm, sys->N, x, ldx, sys->fmm_x, sys->N, nrhs, s);
  run_graph(sys->fmm_graphs.at(nrhs), nrhs, "graph:fmm_matvec", s,
            [&](cudaStream_t gs) { run_fmm_phases(sys, nrhs, gs); });
  launch_scatter_rows(sys->perm, sys->N, sys->fmm_y, sys->N, y, ldy, nrhs, s);
}

// ---------------------------------------------------------------------------
// FMM matvec with the far field in FP32.  FP32 copies of the operators of the
// matvec's Chebyshev order (leaf U_i and its transpose, the 2^D transfers and
// their transposes, the M2L tables); P2M, M2M, M2L + L2L and L2P run in FP32
// on FP32 coefficients, the near field as FP64 products; y = near + far,
// added in FP64 in the scatter back to user order.
// ---------------------------------------------------------------------------
static void build_f32_ops(ifmm_system* sys, cudaStream_t s) {
  Fmm32& f = sys->f32;
  if (f.leafU) return;
  const ChebOps& ops = sys->mv();
  const int nd = ops.nd, dim = sys->dim, L = sys->L;
  const int nt = 1 << dim;
  int no = 1;
  for (int d = 0; d < dim; d++) no *= 7;
  const LevelTopo& leaf = sys->lv[L];
  long long tot = 0;
  for (int i = 0; i < leaf.nb; i++) tot += (long long)(leaf.p1[i] - leaf.p0[i]) * nd;
  // tables: the uniform kernel's padded layout (nd <= 64) or plain nd x nd
  const bool uni = uniform_supported(nd);
  const int ndp = uni ? uniform_ndp(nd) : nd;
  f.leafU = f.ops.alloc<float>((size_t)tot);
  f.leafUT = f.ops.alloc<float>((size_t)tot);
  f.transfer = f.ops.alloc<float>((size_t)nt * nd * ndp);
  f.transferT = f.ops.alloc<float>((size_t)nt * nd * ndp);
  f.m2l.assign(L + 1, nullptr);
  for (int l = 2; l <= L; l++) f.m2l[l] = f.ops.alloc<float>((size_t)no * nd * ndp);
  std::vector<NarrowTask> nt1{{ops.leafU, f.leafU, tot}};
  std::vector<NarrowTTask> nt2;
  for (int i = 0; i < leaf.nb; i++)
    nt2.push_back({ops.leafU + ops.uoff[i], f.leafUT + ops.uoff[i], leaf.p1[i] - leaf.p0[i], nd});
  if (uni) {
    launch_pad_tables<float>(ops.transfer, f.transfer, nt, nd, false, s);
    launch_pad_tables<float>(ops.transfer, f.transferT, nt, nd, true, s);
    for (int l = 2; l <= L; l++) launch_pad_tables<float>(ops.m2l[l], f.m2l[l], no, nd, false, s);
  } else {
    nt1.push_back({ops.transfer, f.transfer, (long long)nt * nd * nd});
    for (int l = 2; l <= L; l++) nt1.push_back({ops.m2l[l], f.m2l[l], (long long)no * nd * nd});
    for (int c = 0; c < nt; c++)
      nt2.push_back({ops.transfer + (size_t)c * nd * nd, f.transferT + (size_t)c * nd * nd, nd, nd});
  }
  Arena tmp;
  launch_narrow(tmp, nt1, s);
  launch_narrow_t(tmp, nt2, s);
  CK(cudaStreamSynchronize(s));
}

struct F32Sizes {
  size_t vec = 0;              // x64, y64, x32, y32
  std::vector<long long> ldl;  // per depth: nb * ndp
};
static F32Sizes f32_sizes(const ifmm_system* sys, int cap) {
  F32Sizes z;
  const int nd = sys->mv().nd;
  const int ndp = uniform_supported(nd) ? uniform_ndp(nd) : nd;
  z.ldl.assign(sys->L + 1, 0);
  for (int l = 2; l <= sys->L; l++) z.ldl[l] = (long long)sys->lv[l].nb * ndp;
  z.vec = (size_t)sys->N * cap;
  return z;
}

static void build_f32_plan(ifmm_system* sys, int cap, cudaStream_t s) {
  build_f32_ops(sys, s);
  Fmm32& f = sys->f32;
  f.graphs.reset();
  f.far.clear();
  f.far_uni.clear();
  f.order.clear();
  f.near.clear();
  f.ws.release();
  f.cap = cap;
  const ChebOps& ops = sys->mv();
  const int nd = ops.nd, L = sys->L, dim = sys->dim;
  const bool uni = uniform_supported(nd);
  const int ndp = uni ? uniform_ndp(nd) : nd;
  const long long N = sys->N;
  const F32Sizes z = f32_sizes(sys, cap);
  f.x64 = f.ws.alloc<double>(z.vec);
  f.y64 = f.ws.alloc<double>(z.vec);
  f.x32 = f.ws.alloc<float>(z.vec);
  f.y32 = f.ws.alloc<float>(z.vec);
  std::vector<float*> mult(L + 1, nullptr), loc(L + 1, nullptr);
  for (int l = 2; l <= L; l++) {
    mult[l] = f.ws.alloc<float>((size_t)z.ldl[l] * cap);
    loc[l] = f.ws.alloc<float>((size_t)z.ldl[l] * cap);
    CK(cudaMemsetAsync(mult[l], 0, sizeof(float) * (size_t)z.ldl[l] * cap, s));
    CK(cudaMemsetAsync(loc[l], 0, sizeof(float) * (size_t)z.ldl[l] * cap, s));
  }
  const std::vector<long long>& ldl = z.ldl;
  std::vector<SpRowF> rows;
  std::vector<SpEntF> ents;
  auto row = [&](float* y, long long ldy, int m) {
    rows.push_back({y, ldy, m, (int)ents.size(), 0, 0.0f});
  };
  auto ent = [&](const float* A, int lda, int k, const float* x, long long ldx) {
    ents.push_back({A, x, ldx, lda, k, 1.0f});
    rows.back().ne++;
  };
  auto flush = [&] {
    if (rows.empty()) return;
    f.far.push_back(plan_spmm_f32(f.ws, rows, ents, cap, s));
    f.order.push_back(0);
    rows.clear();
    ents.clear();
  };
  std::vector<UniRow<float>> urows;
  std::vector<UniEnt<float>> uents;
  auto urow = [&](float* y, long long ldy) { urows.push_back({y, ldy, (int)uents.size(), 0}); };
  auto uent = [&](const float* A, const float* x, long long ldx) {
    uents.push_back({A, x, ldx});
    urows.back().ne++;
  };
  auto uflush = [&] {
    f.far_uni.push_back(plan_uniform<float>(f.ws, urows, uents, nd, cap, s));
    f.order.push_back(1);
    urows.clear();
    uents.clear();
  };
  // a row of nd x nd blocks: the uniform kernel, or general products from the
  // plain tables
  auto trow = [&](float* y, long long ldy) {
    if (uni) urow(y, ldy);
    else row(y, ldy, nd);
  };
  auto tent = [&](const float* table, size_t t, const float* x, long long ldx) {
    if (uni) uent(table + t * nd * ndp, x, ldx);
    else ent(table + t * nd * nd, nd, nd, x, ldx);
  };
  auto tflush = [&] {
    if (uni) uflush();
    else flush();
  };
  const LevelTopo& leaf = sys->lv[L];
  for (int i = 0; i < leaf.nb; i++) {  // P2M: mult_i = U_i^T x_i
    const int m = leaf.p1[i] - leaf.p0[i];
    row(mult[L] + (long long)i * ndp, ldl[L], nd);
    ent(f.leafUT + ops.uoff[i], nd, m, f.x32 + leaf.p0[i], N);
  }
  flush();
  for (int l = L - 1; l >= 2; l--) {  // M2M: mult_p = sum_c T_c^T mult_c
    const LevelTopo& v = sys->lv[l];
    const LevelTopo& c = sys->lv[l + 1];
    for (int p = 0; p < v.nb; p++) {
      trow(mult[l] + (long long)p * ndp, ldl[l]);
      for (int ch = v.cb[p]; ch < v.ce[p]; ch++)
        tent(f.transferT, (size_t)c.child_pos(ch, dim), mult[l + 1] + (long long)ch * ndp,
             ldl[l + 1]);
    }
    tflush();
  }
  for (int l = 2; l <= L; l++) {  // M2L + L2L
    const LevelTopo& v = sys->lv[l];
    for (int i = 0; i < v.nb; i++) {
      trow(loc[l] + (long long)i * ndp, ldl[l]);
      for (int k = v.far_ptr[i]; k < v.far_ptr[i + 1]; k++) {
        const int q = v.far[k];
        tent(f.m2l[l], (size_t)v.m2l_offset(i, q, dim), mult[l] + (long long)q * ndp, ldl[l]);
      }
      if (l > 2)
        tent(f.transfer, (size_t)v.child_pos(i, dim), loc[l - 1] + (long long)v.parent[i] * ndp,
             ldl[l - 1]);
    }
    tflush();
  }
  for (int i = 0; i < leaf.nb; i++) {  // L2P: y_i = U_i loc_i
    const int m = leaf.p1[i] - leaf.p0[i];
    row(f.y32 + leaf.p0[i], N, m);
    ent(f.leafU + ops.uoff[i], m, nd, loc[L] + (long long)i * ndp, ldl[L]);
  }
  flush();
  SpBuild b;  // near field, FP64
  for (int i = 0; i < leaf.nb; i++) {
    const int m = leaf.p1[i] - leaf.p0[i];
    b.row(f.y64 + leaf.p0[i], N, m);
    for (int k = leaf.nbr_ptr[i]; k < leaf.nbr_ptr[i + 1]; k++) {
      const int j = leaf.nbr[k];
      b.ent(sys->p2p + sys->p2p_off[k], m, leaf.p1[j] - leaf.p0[j], 0, f.x64 + leaf.p0[j], N);
    }
  }
  f.near.push_back(plan_spmm(f.ws, b.rows, b.ents, cap, s));
  CK(cudaStreamSynchronize(s));
}

size_t system_f32far_bytes(const ifmm_system* sys, int cap) {
  if (sys->L == 0) return 0;
  const int nd = sys->mv().nd, dim = sys->dim;
  int no = 1;
  for (int d = 0; d < dim; d++) no *= 7;
  const F32Sizes z = f32_sizes(sys, cap);
  const int ndp = uniform_supported(nd) ? uniform_ndp(nd) : nd;
  size_t b = 2 * sizeof(float) * (size_t)sys->N * nd;              // U, U^T
  b += 2 * sizeof(float) * ((size_t)(1 << dim) * nd * ndp);         // transfers
  b += sizeof(float) * (size_t)(sys->L - 1) * no * nd * ndp;         // M2L tables
  b += (2 * sizeof(double) + 2 * sizeof(float)) * z.vec;            // x, y
  for (int l = 2; l <= sys->L; l++) b += 2 * sizeof(float) * (size_t)z.ldl[l] * cap;
  // plan descriptors and split-K partial sums: about 64 bytes per block entry
  size_t ents = 0;
  for (int l = 2; l <= sys->L; l++) ents += sys->lv[l].far.size() + 2 * (size_t)sys->lv[l].nb;
  ents += sys->lv[sys->L].nbr.size();
  return b + 64 * ents + (size_t(16) << 20);
}

void system_prepare_f32far(ifmm_system* sys, int cap, cudaStream_t s) {
  if (sys->L == 0 || cap <= sys->f32.cap) return;
  CK(cudaStreamSynchronize(s));
  build_f32_plan(sys, cap, s);
}

void system_matvec_f32far(ifmm_system* sys, const double* x, long long ldx, double* y,
                          long long ldy, int nrhs, cudaStream_t s) {
  if (nrhs <= 0) return;
  if (sys->L == 0) {
    system_matvec(sys, IFMM_MV_FMM, x, ldx, y, ldy, nrhs, s);
    return;
  }
  Fmm32& f = sys->f32;
  if (nrhs > f.cap) {
    CK(cudaStreamSynchronize(s));
    build_f32_plan(sys, std::max(nrhs, 4), s);
  }
  launch_gather_rows_2(sys->perm, sys->N, x, ldx, f.x64, f.x32, sys->N, nrhs, s);
  run_graph(f.graphs.at(nrhs), nrhs, "graph:fmm_matvec_f32far", s, [&](cudaStream_t gs) {
    size_t a = 0, u = 0;
    for (int kind : f.order) {
      if (kind == 0) launch_spmm_f32(f.far[a++], nrhs, gs);
      else launch_uniform<float>(f.far_uni[u++], nrhs, gs);
    }
    for (const SpmmPlan& p : f.near) launch_spmm(p, nrhs, gs);
  });
  launch_scatter_rows_add(sys->perm, sys->N, f.y64, f.y32, sys->N, y, ldy, nrhs, s);
}

// ---------------------------------------------------------------------------
// sigma_0(E): power iteration on E^T E (Sec. 2.4) with the raw operators of
// order cheb_n.  Extended vector: [x | z^(L) y^(L) | ... | z^(2) y^(2)].
// ---------------------------------------------------------------------------
double system_sigma0(ifmm_system* sys, cudaStream_t s, int* iters) {
  const int L = sys->L, dim = sys->dim;
  const ChebOps& ops = sys->ops_f;
  const int nd = ops.nd;
  const long long N = sys->N;
  std::vector<long long> zo(L + 1, 0), yo(L + 1, 0);
  long long n = N;
  for (int l = L; l >= 2; l--) {
    zo[l] = n;
    n += (long long)sys->lv[l].nb * nd;
    yo[l] = n;
    n += (long long)sys->lv[l].nb * nd;
  }
  SpPlan pE, pT;
  double* v = pE.mem.alloc<double>(n);
  double* w = pE.mem.alloc<double>(n);
  double* u = pE.mem.alloc<double>(n);
  double* red = pE.mem.alloc<double>(4096);
  const LevelTopo& leaf = sys->lv[L];
  auto build = [&](bool T, const double* in, double* out, SpPlan& plan) {
    SpBuild b;
    for (int i = 0; i < leaf.nb; i++) {  // rows x_i
      const int m = leaf.p1[i] - leaf.p0[i];
      b.row(out + leaf.p0[i], n, m);
      for (int k = leaf.nbr_ptr[i]; k < leaf.nbr_ptr[i + 1]; k++) {
        const int j = leaf.nbr[k];
        const int mj = leaf.p1[j] - leaf.p0[j];
        if (!T) {
          b.ent(sys->p2p + sys->p2p_off[k], m, mj, 0, in + leaf.p0[j], n);
        } else {  // column x_i of E: S_ji (rows x_j)
          const int kj = leaf.nslot(j, i);
          b.ent(sys->p2p + sys->p2p_off[kj], mj, mj, 1, in + leaf.p0[j], n);
        }
      }
      b.ent(ops.leafU + ops.uoff[i], m, nd, 0, in + zo[L] + (long long)i * nd, n);
    }
    for (int l = L; l >= 2; l--) {
      const LevelTopo& lv = sys->lv[l];
      for (int i = 0; i < lv.nb; i++) {  // rows z_i: V^T xtilde - y   /  U^T (.) - y
        b.row(out + zo[l] + (long long)i * nd, n, nd);
        if (l == L) {
          const int m = leaf.p1[i] - leaf.p0[i];
          b.ent(ops.leafU + ops.uoff[i], m, m, 1, in + leaf.p0[i], n);
        } else {
          const LevelTopo& c = sys->lv[l + 1];
          for (int ch = lv.cb[i]; ch < lv.ce[i]; ch++)
            b.ent(ops.transfer + (size_t)c.child_pos(ch, dim) * nd * nd, nd, nd, 1,
                  in + yo[l + 1] + (long long)ch * nd, n);
        }
        b.ent(nullptr, nd, nd, 0, in + yo[l] + (long long)i * nd, n, -1.0);
      }
      for (int i = 0; i < lv.nb; i++) {  // rows y_i
        b.row(out + yo[l] + (long long)i * nd, n, nd);
        b.ent(nullptr, nd, nd, 0, in + zo[l] + (long long)i * nd, n, -1.0);
        for (int k = lv.far_ptr[i]; k < lv.far_ptr[i + 1]; k++) {
          const int q = lv.far[k];
          // E: K_iq in (y_i, y_q); E^T row y_i: K_qi^T from (y_q, y_i)
          if (!T)
            b.ent(ops.m2l[l] + (size_t)lv.m2l_offset(i, q, dim) * nd * nd, nd, nd, 0,
                  in + yo[l] + (long long)q * nd, n);
          else
            b.ent(ops.m2l[l] + (size_t)lv.m2l_offset(q, i, dim) * nd * nd, nd, nd, 1,
                  in + yo[l] + (long long)q * nd, n);
        }
        if (l > 2) {
          // E: T_i in (y_i, z_p); E^T row y_i: T_i from (z_p, y_i) = T_i^T  -> (T_i^T)^T
          if (!T)
            b.ent(ops.transfer + (size_t)lv.child_pos(i, dim) * nd * nd, nd, nd, 0,
                  in + zo[l - 1] + (long long)lv.parent[i] * nd, n);
          else
            b.ent(ops.transfer + (size_t)lv.child_pos(i, dim) * nd * nd, nd, nd, 0,
                  in + zo[l - 1] + (long long)lv.parent[i] * nd, n);
        }
      }
    }
    b.flush(plan, s);
  };
  // E^T differs from E only where E is not symmetric; with these operators E
  // is block-transposed as follows: rows z_i of E^T carry U_i^T (l == L) or
  // T_c^T (children) -- the same entries as rows z_i of E -- and rows y_i of
  // E^T carry T_i applied to z_p.  The builder above encodes both.
  build(false, v, w, pE);
  build(true, w, u, pT);
  std::vector<double> h1(1, 1.0 / std::sqrt((double)n));
  // v = 1/sqrt(n)
  {
    std::vector<double> ones(n, h1[0]);
    CK(cudaMemcpyAsync(v, ones.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  double prev = 0.0, sig = 0.0;
  int it = 0;
  for (it = 1; it <= 100; it++) {
    pE.run(1, s);
    pT.run(1, s);
    double nrm2 = 0.0;
    launch_dots(u, n, u, n, n, 1, red, red + 1, s);
    CK(cudaMemcpyAsync(&nrm2, red, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double nw = std::sqrt(nrm2);
    sig = std::sqrt(nw);
    launch_axpby(n, 1, nullptr, 1.0 / nw, u, n, 0.0, v, n, s);
    if (it > 1 && std::fabs(sig - prev) <= 1e-6 * sig) break;
    prev = sig;
  }
  if (it > 100) it = 100;
  CK(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  return sig;
}

}  // namespace ifmm
