// kernels_edges.cu -- edge redirection of Algorithm 3 on the device.
//
// When box j's bases are recompressed (U_hat = U r_j^-style transforms r_j,
// t_j of Eqs. K_kj_update, U/V_parent_j_update) every M2L edge of j changes:
//   K(j, q) <- r_j K(j, q) [t_q^T if q was recompressed too],
//   K(q, j) <- K(q, j) t_j^T             (q not recompressed; otherwise q's own
//                                          pass covers the edge as K(q, j) with
//                                          its r_q on the left)
// for every q in the interaction list I_j.  One CTA per recompressed box walks
// j's interaction list in device memory, so the host builds no per-edge work:
// r_j and t_j stay in shared memory, each product runs out of shared memory,
// and every edge block has exactly one writer (j's CTA writes K(j, .) and the
// K(q, j) of boxes q that were not recompressed).
#include "internal.cuh"

namespace ifmm {

// C (m x n, ld ldc, shared or global) = A (m x k, ld lda) * op(B), op(B) = B
// (k x n, ld ldb) or B^T (B: n x k, ld ldb); block-wide, FP64.
__device__ inline void block_gemm(const double* A, int lda, const double* B, int ldb, bool tB,
                                  double* C, int ldc, int m, int n, int k) {
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int r = e % m, c = e / m;
    double s = 0.0;
    if (tB)
      for (int q = 0; q < k; q++) s = fma(A[r + q * lda], B[c + q * ldb], s);
    else
      for (int q = 0; q < k; q++) s = fma(A[r + q * lda], B[q + c * ldb], s);
    C[r + c * ldc] = s;
  }
}

__global__ void __launch_bounds__(256) k_edge_redirect(const EdgeLevel L, const EdgeColour E) {
  const int j = E.boxes[blockIdx.x];
  extern __shared__ double sm[];
  const int R = E.rmax;            // shared tiles are R x R (ld R)
  double* rj = sm;                 // r_j  (r1_j x r0_j)
  double* tj = sm + R * R;         // t_j  (r1_j x r0_j)
  double* T = sm + 2 * R * R;      // product scratch
  double* Yc = sm + 3 * R * R;     // copy of a block read and rewritten in place
  const int a0 = E.r_old[j], a1 = E.r_new[j];
  for (int e = threadIdx.x; e < a1 * a0; e += blockDim.x) {
    const int r = e % a1, c = e / a1;
    rj[r + c * R] = E.rm[j][r + c * a1];
    tj[r + c * R] = E.tm[j][r + c * a1];
  }
  __syncthreads();
  for (int k = L.far_ptr[j]; k < L.far_ptr[j + 1]; k++) {
    const int q = L.far[k];
    const int q0 = E.r_old[q], q1 = E.r_new[q];
    const bool qr = E.rm[q] != nullptr;
    // K(j, q) <- r_j K(j, q) [t_q^T]
    double* Yjq = L.y_out[k];
    const int ldj = L.rcap[j];
    block_gemm(rj, R, Yjq, ldj, false, T, R, a1, q0, a0);
    __syncthreads();
    if (qr) {
      block_gemm(T, R, E.tm[q], q1, true, Yjq, ldj, a1, q1, q0);
    } else {
      for (int e = threadIdx.x; e < a1 * q0; e += blockDim.x) {
        const int r = e % a1, c = e / a1;
        Yjq[r + c * ldj] = T[r + c * R];
      }
    }
    __syncthreads();
    if (!qr) {
      // K(q, j) <- K(q, j) t_j^T
      double* Yqj = L.y_in[k];
      const int ldq = L.rcap[q];
      for (int e = threadIdx.x; e < q0 * a0; e += blockDim.x) {
        const int r = e % q0, c = e / q0;
        Yc[r + c * R] = Yqj[r + c * ldq];
      }
      __syncthreads();
      block_gemm(Yc, R, tj, R, true, Yqj, ldq, q0, a1, a0);
      __syncthreads();
    }
  }
}

void launch_edge_redirect(const EdgeLevel& L, const EdgeColour& E, int nboxes, cudaStream_t s,
                          double flops) {
  if (nboxes <= 0) return;
  const int bytes = 4 * E.rmax * E.rmax * (int)sizeof(double);
  set_max_dynamic_smem((const void*)k_edge_redirect, 4 * 64 * 64 * (int)sizeof(double) + 1024);
  if (E.rmax > 64) throw Error(IFMM_ERR_CUDA, "internal: edge redirection needs ranks <= 64");
  Prof p("k_edge_redirect", flops, 0.0, s);
  k_edge_redirect<<<nboxes, 256, bytes, s>>>(L, E);
  CK_LAUNCH("k_edge_redirect");
}

}  // namespace ifmm
