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
struct FRec {
  int l, i, a, r, p, nC, colour;
  double* LU;
  int* piv;
  int* info;
  double* ERP;  // nC x p, ld nC
  double* G;    // p x nC, ld p: E(P,P)^-1 E(P,C)
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
  size_t plan_bytes() const {
    size_t b = 0;
    for (auto& kv : plans) b += kv.second->mem.held + kv.second->task_mem.held;
    return b;
  }
};

namespace ifmm {
ifmm_factorization* factor_create(ifmm_system* sys, cudaStream_t s);
void factor_solve(ifmm_factorization* f, const double* b, long long ldb, double* x,
                  long long ldx, int nrhs, cudaStream_t s);
ifmm_status gmres_run(ifmm_system* sys, ifmm_factorization* fac, int mode, const double* b,
                      double* x, int nrhs, long long ld, double tol, int maxit,
                      ifmm_gmres_report* rep, cudaStream_t s, Arena* workspace = nullptr);
}  // namespace ifmm
