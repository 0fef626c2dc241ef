// factor.cuh -- the IFMM factorisation object and its substitution plan.
#pragma once
#include <map>
#include <memory>

#include "system.cuh"

namespace ifmm {

// One eliminated box: what the substitution phase needs (the downward pass of Algorithm 1).
struct BlockRef {
  char kind;  // 'x': xtilde_j of a box not yet eliminated; 'y': ybar_h of an eliminated one
  int box, dim, off;
};
// The substitution phase needs, per box, three blocks derived from the
// pivot block's LU (kept in the factorisation; E(P,P), E(R,P) and G itself
// live only while their colour is eliminated):
//   W  = E(P,P)^-1 [I_a; 0]          (p x a): w = W b_i        (RHS of the pivot set)
//   F  = E(R,P) W                    (nC x a): b_R -= F b_i    (right-hand-side update)
//   Ga = (E(P,P)^-1 E(P,C))[0:a, :]  (a x nC): x_i = w[0:a] - Ga x_C
// (the z rows of the pivot set are never read by another box).
struct FRec {
  int l, i, a, r, p, nC, colour;
  int* info;     // pivot test of the LU (0: passed)
  double* W;     // p x a, ld p
  double* F;     // nC x a, ld nC
  double* Ga;    // a x nC, ld a
  std::vector<BlockRef> blk;
};

// Substitution plan, built for a right-hand-side capacity.
struct SolvePlan {
  int cap = 0;
  Arena mem;
  double* xt = nullptr;                 // tree-order RHS / solution at the leaves, ld N
  std::vector<double*> ybar;            // per depth: ybar^(l), ld nybar[l]
  std::vector<long long> nybar;
  std::vector<double*> w;               // per record: p x cap (ld p)
  struct Step {
    int kind;             // 0 copy, 1 getrs, 2 spmm
    CopyTask* copies = nullptr;
    int ncopies = 0;
    GetrsPlan rs;
    SpmmPlan sp;
  };
  std::vector<Step> steps;
  Arena task_mem;
  GraphCache graph;  // the steps (and the ybar clears) as one graph
};

// FP32 copies of the substitution blocks and the top system's inverse, made
// on first use by the reduced-precision sweeps.
struct F32Data {
  Arena mem;
  std::vector<const float*> W, F, Ga;  // per record
  const float* top_inv = nullptr;      // top_n x top_n (or the dense N x N inverse)
  bool ready = false;
};

// Reduced-precision substitution plan (FP32 vectors and blocks).
struct SolvePlan32 {
  int cap = 0;
  Arena mem;
  float* xt = nullptr;        // tree-order RHS / solution at the leaves, ld N
  float* xt2 = nullptr;       // dense system only: the solution
  float* top_tmp = nullptr;   // copy of the top right-hand side
  std::vector<float*> ybar;
  std::vector<long long> nybar;
  std::vector<float*> w;
  std::vector<SpmmPlanF> steps;
  Arena task_mem;
  GraphSet graphs;  // per right-hand-side count (<= cap)
};

}  // namespace ifmm

struct ifmm_factorization {
  ifmm_system* sys = nullptr;
  ifmm::Arena store;                  // LU, E(R,P), G of every eliminated box; top LU
  std::vector<ifmm::FRec> recs;       // in elimination order
  std::vector<std::vector<int>> rank; // per depth: rank at elimination
  std::vector<std::vector<long long>> yoff;  // per depth: offset of ybar_i
  int top_n = 0;
  double* top_LU = nullptr;
  int* top_piv = nullptr;
  int* top_info = nullptr;
  double* dense_LU = nullptr;         // L == 0 only
  int* dense_piv = nullptr;
  int* dense_info = nullptr;
  int* d_info_all = nullptr;
  ifmm_factor_info info{};
  // substitution plans by right-hand-side count (built on first use; a plan is
  // specific to its column count, so alternating batch widths keep theirs)
  std::map<int, std::unique_ptr<ifmm::SolvePlan>> plans;
  ifmm::F32Data f32;
  // FP32 plans by capacity: one plan of 32 columns serves every block of up
  // to 32 right-hand sides (wider requests get a plan of their own width)
  std::map<int, std::unique_ptr<ifmm::SolvePlan32>> plans32;
  size_t plan_bytes() const {
    size_t b = f32.mem.held;
    for (auto& kv : plans) b += kv.second->mem.held + kv.second->task_mem.held;
    for (auto& kv : plans32) b += kv.second->mem.held + kv.second->task_mem.held;
    return b;
  }
};

namespace ifmm {
ifmm_factorization* factor_create(ifmm_system* sys, cudaStream_t s);
void factor_solve(ifmm_factorization* f, const double* b, long long ldb, double* x,
                  long long ldx, int nrhs, cudaStream_t s);
// The same substitution with FP32 blocks and vectors (b, x still FP64).
void factor_solve_f32(ifmm_factorization* f, const double* b, long long ldb, double* x,
                      long long ldx, int nrhs, cudaStream_t s);
// Builds the FP32 copies (allocating); called by the first FP32 solve.
void factor_prepare_f32(ifmm_factorization* f, cudaStream_t s);
// Builds the FP32 substitution plan that serves up to max_cols columns now.
void factor_prepare_plans_f32(ifmm_factorization* f, int max_cols, cudaStream_t s);
struct GmresOpts {
  int side = IFMM_GMRES_RIGHT;  // ifmm_gmres_side
  int refine = 2;               // restarts from x when the true residual misses tol
  int precond_fp32 = 0;         // substitution sweeps in FP32 (flexible GMRES only)
  int block = 0;                // block GMRES over the columns
  int mv_fp32 = 0;              // iterative refinement: Arnoldi products with the far
                                // field in FP32, true residuals in FP64
};
// Iterative refinement: each cycle's inner GMRES stops once its residual
// estimate has fallen by this factor (or below tol / 2), since the FP32 far
// field bounds what one cycle can gain.
constexpr double IR_INNER_REDUCTION = 1e-4;
ifmm_status gmres_run(ifmm_system* sys, ifmm_factorization* fac, int mode, const double* b,
                      double* x, int nrhs, long long ld, double tol, int maxit,
                      ifmm_gmres_report* rep, cudaStream_t s, Arena* workspace = nullptr,
                      const GmresOpts& opt = GmresOpts());
ifmm_status block_gmres_run(ifmm_system* sys, ifmm_factorization* fac, int mode, const double* b,
                            double* x, int k, long long ld, double tol, int maxit,
                            ifmm_gmres_report* rep, cudaStream_t s, const GmresOpts& opt);
}  // namespace ifmm
