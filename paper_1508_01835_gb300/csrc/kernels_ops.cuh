// kernels_ops.cuh -- launchers for operator construction and sparse products.
#pragma once
#include "internal.cuh"

namespace ifmm {

struct KSpec {
  int kind;
  double param, diag;
};

struct ChebSpec {
  int n, nd;
  double t[8];  // Chebyshev nodes cos((2a - 1) pi / (2n)), a = 1..n
};

struct LeafGeom {
  int p0, p1;         // point range in tree order
  long long uoff;     // offset of the m x n^D interpolation matrix
  double centre[3];
  double h;           // half-width
};

struct P2PTask {
  int i0, i1, j0, j1;  // point ranges of the two leaves
  long long off;       // offset of the (i1-i0) x (j1-j0) block
};

void launch_leaf_interp(ChebSpec c, int dim, const double* pts_tree, const LeafGeom* leaves,
                        int nleaves, double* U, cudaStream_t s);
void launch_transfer(ChebSpec c, int dim, double* T, cudaStream_t s);
void launch_m2l_table(ChebSpec c, int dim, KSpec ks, double h, double* K, cudaStream_t s);
void launch_p2p_blocks(KSpec ks, int dim, const double* pts_tree, const P2PTask* tasks, int n,
                       double* S, cudaStream_t s);
void launch_direct(KSpec ks, int dim, const double* pts, long long N, const double* x,
                   long long ldx, double* y, long long ldy, int nrhs, cudaStream_t s);
void launch_gather_rows(const long long* perm, long long N, const double* in, long long ldi,
                        double* out, long long ldo, int ncols, cudaStream_t s);
void launch_scatter_rows(const long long* perm, long long N, const double* in, long long ldi,
                         double* out, long long ldo, int ncols, cudaStream_t s);

// pts_tree[t, :] = pts_user[perm[t], :] (row-major, dim columns)
void launch_permute_points(const long long* perm, long long N, int dim, const double* in,
                           double* out, cudaStream_t s);

// tree construction (kernels_tree.cu)
struct TreeOut {
  int L = 0;
  double lo[3] = {0, 0, 0};
  double edge = 1.0;
  std::vector<long long> perm;                  // tree order -> user index
  std::vector<std::vector<unsigned long long>> keys;  // per depth 0..L, Morton order
  std::vector<int> leaf_begin;                  // per leaf: first point (tree order)
};
TreeOut build_tree_device(const double* d_pts, long long N, int dim, int leaf_max,
                          long long* d_perm, cudaStream_t s);

// vector helpers (kernels_vec.cu)
// out[c] = sum_i x[i + c ldx] * y[i + c ldy], deterministic fixed-order reduction
void launch_count_nonzero(const int* const* d_flags, int n, int* d_count, cudaStream_t s);
void launch_dots(const double* x, long long ldx, const double* y, long long ldy, long long n,
                 int ncols, double* out, double* partial, cudaStream_t s);
void launch_axpby(long long n, int ncols, const double* alpha, double alpha_scale, const double* x,
                  long long ldx, double beta, double* y, long long ldy, cudaStream_t s);

}  // namespace ifmm
