// kernels_vec.cu -- deterministic vector reductions and updates (GMRES of
// Sec. 3.2, power iteration of Sec. 2.4).  Reductions use a fixed block count
// and a fixed summation order, so results do not depend on launch timing.
#include "kernels_ops.cuh"

namespace ifmm {

constexpr int DOT_BLOCKS = 256;

__global__ void k_dot_partial(const double* __restrict__ x, long long ldx,
                              const double* __restrict__ y, long long ldy, long long n,
                              double* __restrict__ part) {
  const int col = blockIdx.y;
  const double* xc = x + col * ldx;
  const double* yc = y + col * ldy;
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s += xc[i] * yc[i];
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[col * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void k_dot_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  const int col = blockIdx.x;
  __shared__ double sh[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[col * nparts + b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[col] = sh[0];
}

// partial must hold ncols * DOT_BLOCKS doubles
void launch_dots(const double* x, long long ldx, const double* y, long long ldy, long long n,
                 int ncols, double* out, double* partial, cudaStream_t s) {
  if (ncols <= 0) return;
  k_dot_partial<<<dim3(DOT_BLOCKS, ncols), 256, 0, s>>>(x, ldx, y, ldy, n, partial);
  CK_LAUNCH("k_dot_partial");
  k_dot_final<<<ncols, 256, 0, s>>>(partial, DOT_BLOCKS, out);
  CK_LAUNCH("k_dot_final");
}

// y = a_c x + beta y per column, a_c = alpha_scale * (alpha ? alpha[c] : 1)
__global__ void k_axpby(long long n, const double* __restrict__ alpha, double alpha_scale,
                        const double* __restrict__ x, long long ldx, double beta,
                        double* __restrict__ y, long long ldy) {
  const int col = blockIdx.y;
  const double a = alpha_scale * (alpha ? alpha[col] : 1.0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = a * x[i + col * ldx];
    y[i + col * ldy] = (beta == 0.0) ? v : beta * y[i + col * ldy] + v;
  }
}

void launch_axpby(long long n, int ncols, const double* alpha, double alpha_scale, const double* x,
                  long long ldx, double beta, double* y, long long ldy, cudaStream_t s) {
  if (ncols <= 0 || n <= 0) return;
  const int bx = (int)std::min<long long>(1024, (n + 255) / 256);
  k_axpby<<<dim3(bx, ncols), 256, 0, s>>>(n, alpha, alpha_scale, x, ldx, beta, y, ldy);
  CK_LAUNCH("k_axpby");
}

// *count = number of nonzero *flags[k] (pivot-test results of many blocks)
__global__ void k_count_nonzero(const int* const* __restrict__ flags, int n, int* __restrict__ count) {
  int c = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) c += *flags[k] != 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ int sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
    *count = t;
  }
}

void launch_count_nonzero(const int* const* d_flags, int n, int* d_count, cudaStream_t s) {
  k_count_nonzero<<<1, 1024, 0, s>>>(d_flags, n, d_count);
  CK_LAUNCH("k_count_nonzero");
}

}  // namespace ifmm
