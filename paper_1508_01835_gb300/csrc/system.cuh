// system.cuh -- the system object: tree topology, raw operators, product plans.
#pragma once
#include <algorithm>
#include <limits>

#include "kernels_ops.cuh"

struct ifmm_ctx {
  int device = 0;
  std::string last_error;
};

namespace ifmm {

void build_lists_device(const std::vector<std::vector<unsigned long long>>& keys, int dim,
                        std::vector<std::vector<int>>& nbr, std::vector<std::vector<int>>& far,
                        cudaStream_t s);
void morton_decode_host(unsigned long long k, int dim, int* c);

// One depth of the tree, boxes in Morton order.
struct LevelTopo {
  int l = 0, nb = 0;
  double h = 0.0;                       // box half-width
  std::vector<int> coords;              // nb x 3
  std::vector<int> parent;              // index at depth l-1
  std::vector<int> cb, ce;              // children range at depth l+1
  std::vector<int> colour;
  std::vector<int> nbr_ptr, nbr;        // N_i, sorted, includes i
  std::vector<int> far_ptr, far;        // I_i, sorted
  std::vector<int> yl_ptr, yl;          // N_i u I_i, sorted
  std::vector<int> p0, p1;              // leaves: point range (tree order)
  int find(const std::vector<int>& ptr, const std::vector<int>& v, int i, int j) const {
    auto b = v.begin() + ptr[i], e = v.begin() + ptr[i + 1];
    auto it = std::lower_bound(b, e, j);
    return (it != e && *it == j) ? (int)(it - v.begin()) : -1;
  }
  int nslot(int i, int j) const { return find(nbr_ptr, nbr, i, j); }
  int yslot(int i, int j) const { return find(yl_ptr, yl, i, j); }
  bool is_nbr(int i, int j) const { return nslot(i, j) >= 0; }
  int child_pos(int i, int dim) const {
    int p = 0;
    for (int d = 0; d < dim; d++) p |= (coords[i * 3 + d] & 1) << d;
    return p;
  }
  int m2l_offset(int i, int q, int dim) const {
    int o = 0, w = 1;
    for (int d = 0; d < dim; d++) {
      o += (coords[q * 3 + d] - coords[i * 3 + d] + 3) * w;
      w *= 7;
    }
    return o;
  }
};

// Chebyshev operators of one order n.
struct ChebOps {
  int n = 0, nd = 0;
  ChebSpec spec{};
  double* leafU = nullptr;          // per leaf m_i x nd (ld m_i)
  std::vector<long long> uoff;
  double* transfer = nullptr;       // 2^D blocks nd x nd
  std::vector<double*> m2l;         // per depth: 7^D blocks nd x nd (depth >= 2)
  // the same tables in the padded column layout of the uniform block-row
  // kernel (nd columns of uniform_ndp(nd) entries), made with the FMM plan
  double* transfer_pad = nullptr;   // L2L
  double* transferT_pad = nullptr;  // M2M (transposed)
  std::vector<double*> m2l_pad;
};

// Device copies of the lists the allocation-free matvec reads (built once when
// the system is created, in the system's own memory).
struct StaticLevelLists {
  const int* child_begin = nullptr;  // nb + 1: children of box p are [child_begin[p], child_begin[p+1])
  const int* cpos = nullptr;         // nb: position of the box inside its parent
  const int* parent = nullptr;       // nb
  const int* far_ptr = nullptr;      // nb + 1
  const int* far_idx = nullptr;      // interaction list entries
  const int* far_off = nullptr;      // M2L table offset of each entry
};
struct StaticLeafLists {
  const int* p0 = nullptr;             // nb + 1 point offsets (tree order)
  const long long* uoff = nullptr;     // nb: offset of U_i
  const int* nbr_ptr = nullptr;        // nb + 1
  const int* nbr_idx = nullptr;
  const long long* p2p_off = nullptr;  // per neighbour entry
};

// A launch sequence of block-row products.
struct SpPlan {
  std::vector<SpmmPlan> phases;
  Arena mem;
  void run(int nrhs, cudaStream_t s) const {
    for (const SpmmPlan& p : phases) launch_spmm(p, nrhs, s);
  }
};
// FMM matvec with the far field in FP32: P2M, M2M, M2L, L2L and L2P read
// FP32 copies of the operators (P2M reads stored transposes of U_i, M2M the
// transposed transfers) and FP32 coefficients; the near field (P2P) stays
// FP64.  Used for the inner iterations of GMRES with iterative refinement,
// whose residuals are FP64.
struct Fmm32 {
  Arena ops;                  // operator copies, kept once made
  Arena ws;                   // plans and workspace, rebuilt when nrhs grows
  float* leafU = nullptr;     // per leaf m_i x nd (offsets as ChebOps::uoff)
  float* leafUT = nullptr;    // per leaf nd x m_i
  float* transfer = nullptr;  // 2^D blocks nd x nd (padded layout when uniform)
  float* transferT = nullptr;
  std::vector<float*> m2l;    // per depth: 7^D blocks
  std::vector<SpmmPlanF> far;           // P2M, L2P (and M2M, M2L/L2L when nd > 64)
  std::vector<UniPlan<float>> far_uni;  // M2M, M2L + L2L (nd <= 64)
  std::vector<int> order;               // phase sequence: 0 next far, 1 next far_uni
  std::vector<SpmmPlan> near;
  double *x64 = nullptr, *y64 = nullptr;  // tree order
  float *x32 = nullptr, *y32 = nullptr;
  int cap = 0;
  GraphSet graphs;  // per right-hand-side count (<= cap)
};

struct SpBuild {
  std::vector<SpRow> rows;
  std::vector<SpEnt> ents;
  void row(double* y, long long ldy, int m, double beta = 0.0) {
    rows.push_back({y, ldy, m, (int)ents.size(), 0, beta});
  }
  void ent(const double* A, int lda, int k, int transA, const double* x, long long ldx,
           double alpha = 1.0) {
    ents.push_back({A, x, ldx, lda, k, transA, alpha});
    rows.back().ne++;
  }
  void flush(SpPlan& plan, cudaStream_t s, int nrhs = 1) {
    if (rows.empty()) return;
    plan.phases.push_back(plan_spmm(plan.mem, rows, ents, nrhs, s));
    rows.clear();
    ents.clear();
  }
};

}  // namespace ifmm

struct ifmm_system {
  ifmm_ctx* ctx = nullptr;
  long long N = 0;
  int dim = 3;
  ifmm::KSpec ks{};
  ifmm_options opt{};
  int L = 0;
  double lo[3] = {0, 0, 0};
  double edge = 1.0;
  int max_leaf = 0;
  ifmm::Arena mem;                           // points, perm, operators, near field
  double* pts_user = nullptr;
  double* pts_tree = nullptr;
  long long* perm = nullptr;
  std::vector<long long> perm_h;
  std::vector<ifmm::LevelTopo> lv;           // depths 0..L
  double* p2p = nullptr;                     // near-field blocks
  std::vector<long long> p2p_off;            // per leaf neighbour slot
  ifmm::ChebOps ops_f, ops_mv;               // factor order / matvec order
  bool same_ops = true;
  // FMM matvec plan and its workspace (grown on demand)
  ifmm::Arena fmm_ws;
  ifmm::SpPlan fmm_plan;
  std::vector<ifmm::UniPlan<double>> fmm_uni;  // M2M, M2L + L2L phases (nd <= 64)
  std::vector<int> fmm_order;                  // 0: next fmm_plan phase, 1: next fmm_uni
  ifmm::GraphSet fmm_graphs;   // the FMM phases as one graph per right-hand-side count
  int fmm_cap = 0;
  double *fmm_x = nullptr, *fmm_y = nullptr;
  ifmm::Fmm32 f32;                           // FP32 far field (made on first use)
  std::vector<ifmm::StaticLevelLists> static_lv;  // per depth 2..L (fmm_matvec_static)
  ifmm::StaticLeafLists static_leaf;
  double sigma0 = std::numeric_limits<double>::quiet_NaN();
  int sigma0_iters = 0;
  const ifmm::ChebOps& mv() const { return same_ops ? ops_f : ops_mv; }
};

namespace ifmm {
ifmm_system* system_create(ifmm_ctx* ctx, const double* pts, bool host, long long N,
                           const ifmm_kernel* k, const ifmm_options* opt, cudaStream_t s);
void system_matvec(ifmm_system* sys, int mode, const double* x, long long ldx, double* y,
                   long long ldy, int nrhs, cudaStream_t s);
// FP64 FMM plan and workspace: bytes for `cap` columns (estimate), bytes held
// by the FMM plans of both precisions, and building the plan for `cap` now
size_t system_fmm_bytes(const ifmm_system* sys, int cap);
size_t system_fmm_held(const ifmm_system* sys);
void system_prepare_fmm(ifmm_system* sys, int cap, cudaStream_t s);
// y = A_n x with the far field in FP32 (see Fmm32); the FP64 product when the
// system has no tree.  Builds the FP32 operators and plan on first use.
void system_matvec_f32far(ifmm_system* sys, const double* x, long long ldx, double* y,
                          long long ldy, int nrhs, cudaStream_t s);
// makes the FP32 far-field operators and a plan for `cap` columns now
void system_prepare_f32far(ifmm_system* sys, int cap, cudaStream_t s);
// device bytes of the FP32 far-field operators and plan for `cap` columns
size_t system_f32far_bytes(const ifmm_system* sys, int cap);
double system_sigma0(ifmm_system* sys, cudaStream_t s, int* iters);
void system_matvec_static(ifmm_system* sys, const double* x, double* y, int nrhs, long long ld,
                          int device, cudaStream_t s);
void build_static_lists(ifmm_system* sys, cudaStream_t s);
}  // namespace ifmm
