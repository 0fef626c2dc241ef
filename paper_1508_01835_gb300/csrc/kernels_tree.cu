// kernels_tree.cu -- uniform 2^D-tree of the points (the first step of Algorithm 1;
// Sec. 2.3 lists; Sec. 3 uniform tree with a bounded number of points per leaf).
//
// Root: the cube of edge max_d(max_d - min_d) (1 + 1e-12) at the per-dimension
// minimum.  A point's box at depth l is floor(((x - lo) / edge) 2^l); the leaf
// depth is the smallest L >= 2 with every leaf holding <= leaf_max points.
// Points are ordered by leaf Morton key (x bit lowest), stably, so points of
// a leaf keep their input order.
#include <cub/cub.cuh>
#include <thrust/iterator/counting_iterator.h>

#include "kernels_ops.cuh"

namespace ifmm {

constexpr int KEY_BITS = 20;  // coordinate bits per dimension (depth <= 20)

__host__ __device__ inline unsigned long long morton_encode(const int* c, int dim) {
  unsigned long long k = 0;
  for (int b = 0; b < KEY_BITS; b++)
    for (int d = 0; d < dim; d++)
      k |= (unsigned long long)((c[d] >> b) & 1) << (dim * b + d);
  return k;
}
__host__ __device__ inline void morton_decode(unsigned long long k, int dim, int* c) {
  for (int d = 0; d < dim; d++) c[d] = 0;
  for (int b = 0; b < KEY_BITS; b++)
    for (int d = 0; d < dim; d++) c[d] |= (int)((k >> (dim * b + d)) & 1ull) << b;
}

__global__ void k_bbox_partial(const double* __restrict__ p, long long N, int dim,
                               double* __restrict__ part) {
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    for (int d = 0; d < dim; d++) {
      mn[d] = fmin(mn[d], p[i * dim + d]);
      mx[d] = fmax(mx[d], p[i * dim + d]);
    }
  __shared__ double s[256][6];
  for (int d = 0; d < 3; d++) { s[threadIdx.x][d] = mn[d]; s[threadIdx.x][3 + d] = mx[d]; }
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int d = 0; d < 3; d++) {
        s[threadIdx.x][d] = fmin(s[threadIdx.x][d], s[threadIdx.x + h][d]);
        s[threadIdx.x][3 + d] = fmax(s[threadIdx.x][3 + d], s[threadIdx.x + h][3 + d]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int d = 0; d < 6; d++) part[blockIdx.x * 6 + d] = s[0][d];
}

__global__ void k_bbox_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double r[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  for (int b = 0; b < nparts; b++)
    for (int d = 0; d < 3; d++) {
      r[d] = fmin(r[d], part[b * 6 + d]);
      r[3 + d] = fmax(r[3 + d], part[b * 6 + 3 + d]);
    }
  for (int d = 0; d < 6; d++) out[d] = r[d];
}

struct Frame {
  double lo[3];
  double edge;
};

// Morton key of the depth-20 box of each point; the depth-l key is key >> dim (20 - l)
__global__ void k_keys20(const double* __restrict__ p, long long N, int dim, Frame f,
                         unsigned long long* __restrict__ key, int* __restrict__ idx) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int c[3] = {0, 0, 0};
  const double scale = (double)(1 << KEY_BITS);
  for (int d = 0; d < dim; d++) {
    const double t = __ddiv_rn(__dsub_rn(p[i * dim + d], f.lo[d]), f.edge);
    long long k = (long long)floor(__dmul_rn(t, scale));
    if (k < 0) k = 0;
    if (k > (1 << KEY_BITS) - 1) k = (1 << KEY_BITS) - 1;
    c[d] = (int)k;
  }
  key[i] = morton_encode(c, dim);
  idx[i] = (int)i;
}

// any run of equal depth-L prefixes longer than leaf_max?
__global__ void k_check_runs(const unsigned long long* __restrict__ sk, long long N, int shift,
                             int leaf_max, int* __restrict__ bad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i + leaf_max >= N) return;
  if ((sk[i] >> shift) == (sk[i + leaf_max] >> shift)) *bad = 1;
}

__global__ void k_shift_keys(const unsigned long long* __restrict__ in, long long N, int shift,
                             unsigned long long* __restrict__ out, int* __restrict__ idx) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  out[i] = in[i] >> shift;
  if (idx) idx[i] = (int)i;
}

__global__ void k_run_flags(const unsigned long long* __restrict__ sk, long long N,
                            char* __restrict__ flag) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  flag[i] = (i == 0) || (sk[i] != sk[i - 1]);
}

__global__ void k_widen(const int* __restrict__ in, long long N, long long* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = in[i];
}

static inline int nblk(long long n) { return (int)((n + 255) / 256); }

TreeOut build_tree_device(const double* d_pts, long long N, int dim, int leaf_max,
                          long long* d_perm, cudaStream_t s) {
  TreeOut T;
  Arena ar;
  ar.chunk_bytes = std::max<size_t>(size_t(64) << 20, (size_t)N * 64 + (size_t(16) << 20));
  // bounding box
  double* part = ar.alloc<double>(256 * 6);
  double* bb = ar.alloc<double>(6);
  k_bbox_partial<<<256, 256, 0, s>>>(d_pts, N, dim, part);
  CK_LAUNCH("k_bbox_partial");
  k_bbox_final<<<1, 32, 0, s>>>(part, 256, bb);
  CK_LAUNCH("k_bbox_final");
  double hb[6];
  CK(cudaMemcpyAsync(hb, bb, sizeof(hb), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double ext = 0.0;
  for (int d = 0; d < dim; d++) {
    T.lo[d] = hb[d];
    ext = std::max(ext, hb[3 + d] - hb[d]);
  }
  T.edge = ext * (1.0 + 1e-12);
  if (T.edge == 0.0) T.edge = 1.0;
  if (N <= leaf_max) {
    T.L = 0;
    T.perm.resize(N);
    for (long long i = 0; i < N; i++) T.perm[i] = i;
    T.keys.assign(1, std::vector<unsigned long long>{0ull});
    T.leaf_begin = {0};
    CK(cudaMemcpyAsync(d_perm, T.perm.data(), N * sizeof(long long), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return T;
  }
  Frame f;
  for (int d = 0; d < 3; d++) f.lo[d] = T.lo[d];
  f.edge = T.edge;
  auto* key20 = ar.alloc<unsigned long long>(N);
  auto* keyA = ar.alloc<unsigned long long>(N);
  auto* keyB = ar.alloc<unsigned long long>(N);
  int* idxA = ar.alloc<int>(N);
  int* idxB = ar.alloc<int>(N);
  int* bad = ar.alloc<int>(1);
  k_keys20<<<nblk(N), 256, 0, s>>>(d_pts, N, dim, f, key20, idxA);
  CK_LAUNCH("k_keys20");
  size_t tmp_bytes = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, key20, keyA, idxA, idxB, (int)N, 0,
                                  dim * KEY_BITS, s);
  size_t tmp2 = 0;
  cub::DeviceSelect::Unique(nullptr, tmp2, keyA, keyB, bad, (int)N, s);
  tmp_bytes = std::max(tmp_bytes, tmp2);
  void* tmp = ar.alloc_bytes(tmp_bytes + 256);
  CK(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, key20, keyA, idxA, idxB, (int)N, 0,
                                     dim * KEY_BITS, s));
  // depth: smallest L >= 2 whose runs are all <= leaf_max
  int L = 0;
  for (int l = 2; l <= KEY_BITS; l++) {
    CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_check_runs<<<nblk(N), 256, 0, s>>>(keyA, N, dim * (KEY_BITS - l), leaf_max, bad);
    CK_LAUNCH("k_check_runs");
    int hbad = 0;
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!hbad) { L = l; break; }
  }
  if (L == 0) throw Error(IFMM_ERR_INVALID_ARG, "points too clustered: no depth <= 20 fits leaf_max");
  T.L = L;
  // stable sort of the depth-L keys in input order -> tree order
  k_shift_keys<<<nblk(N), 256, 0, s>>>(key20, N, dim * (KEY_BITS - L), keyB, idxA);
  CK_LAUNCH("k_shift_keys");
  CK(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keyB, keyA, idxA, idxB, (int)N, 0,
                                     dim * L, s));
  k_widen<<<nblk(N), 256, 0, s>>>(idxB, N, d_perm);
  CK_LAUNCH("k_widen");
  T.perm.resize(N);
  CK(cudaMemcpyAsync(T.perm.data(), d_perm, N * sizeof(long long), cudaMemcpyDeviceToHost, s));
  // leaf boxes: run starts of the sorted keys
  char* flag = ar.alloc<char>(N);
  int* starts = idxA;
  int* nsel = bad;
  k_run_flags<<<nblk(N), 256, 0, s>>>(keyA, N, flag);
  CK_LAUNCH("k_run_flags");
  size_t tmp3 = 0;
  thrust::counting_iterator<int> it(0);
  cub::DeviceSelect::Flagged(nullptr, tmp3, it, flag, starts, nsel, (int)N, s);
  void* tmpf = ar.alloc_bytes(tmp3 + 256);
  CK(cub::DeviceSelect::Flagged(tmpf, tmp3, it, flag, starts, nsel, (int)N, s));
  int nleaf = 0;
  CK(cudaMemcpyAsync(&nleaf, nsel, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  T.leaf_begin.resize(nleaf);
  CK(cudaMemcpyAsync(T.leaf_begin.data(), starts, nleaf * sizeof(int), cudaMemcpyDeviceToHost, s));
  // unique keys per depth L..0
  T.keys.assign(L + 1, {});
  CK(cub::DeviceSelect::Unique(tmp, tmp_bytes, keyA, keyB, nsel, (int)N, s));
  long long cnt = nleaf;
  for (int l = L; l >= 0; l--) {
    T.keys[l].resize(cnt);
    CK(cudaMemcpyAsync(T.keys[l].data(), keyB, cnt * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s));
    if (l == 0) break;
    k_shift_keys<<<nblk(cnt), 256, 0, s>>>(keyB, cnt, dim, keyA, nullptr);
    CK_LAUNCH("k_shift_keys");
    CK(cub::DeviceSelect::Unique(tmp, tmp_bytes, keyA, keyB, nsel, (int)cnt, s));
    int c2 = 0;
    CK(cudaMemcpyAsync(&c2, nsel, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    cnt = c2;
  }
  CK(cudaStreamSynchronize(s));
  return T;
}

// ---------------------------------------------------------------------------
// neighbour (N_i) and interaction (I_i) lists of one depth, padded tables
// ---------------------------------------------------------------------------
__device__ int bsearch_key(const unsigned long long* keys, int n, unsigned long long k) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (keys[mid] < k) lo = mid + 1; else hi = mid;
  }
  return (lo < n && keys[lo] == k) ? lo : -1;
}
__device__ int lower_bound_key(const unsigned long long* keys, int n, unsigned long long k) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (keys[mid] < k) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_child_range(const unsigned long long* __restrict__ pkeys, int np,
                              const unsigned long long* __restrict__ ckeys, int nc, int dim,
                              int* __restrict__ cb, int* __restrict__ ce) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  cb[p] = lower_bound_key(ckeys, nc, pkeys[p] << dim);
  ce[p] = lower_bound_key(ckeys, nc, (pkeys[p] + 1) << dim);
}

__global__ void k_lists(const unsigned long long* __restrict__ keys, int nb, int l, int dim,
                        const unsigned long long* __restrict__ pkeys, int npb,
                        const int* __restrict__ pnbr, const int* __restrict__ cb,
                        const int* __restrict__ ce, int* __restrict__ nbr, int* __restrict__ far) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int c[3], q[3];
  morton_decode(keys[i], dim, c);
  const int nstencil = (dim == 3) ? 27 : 9;
  const int side = 1 << l;
  for (int s = nstencil; s < 27; s++) nbr[i * 27 + s] = -1;
  for (int s = 0; s < nstencil; s++) {
    int ss = s, ok = 1;
    for (int d = 0; d < dim; d++) {
      q[d] = c[d] + (ss % 3) - 1;
      ss /= 3;
      if (q[d] < 0 || q[d] >= side) ok = 0;
    }
    nbr[i * 27 + s] = ok ? bsearch_key(keys, nb, morton_encode(q, dim)) : -1;
  }
  const int maxfar = (dim == 3) ? 189 : 27;
  for (int s = 0; s < 189; s++) far[i * 189 + s] = -1;
  if (l < 2) return;
  const int p = bsearch_key(pkeys, npb, keys[i] >> dim);
  if (p < 0) return;
  int cnt = 0;
  for (int s = 0; s < nstencil; s++) {
    const int pn = pnbr[p * 27 + s];
    if (pn < 0) continue;
    for (int ch = cb[pn]; ch < ce[pn]; ch++) {
      morton_decode(keys[ch], dim, q);
      int dmax = 0;
      for (int d = 0; d < dim; d++) dmax = max(dmax, abs(q[d] - c[d]));
      if (dmax >= 2 && cnt < maxfar) far[i * 189 + cnt++] = ch;
    }
  }
}

void build_lists_device(const std::vector<std::vector<unsigned long long>>& keys, int dim,
                        std::vector<std::vector<int>>& nbr, std::vector<std::vector<int>>& far,
                        cudaStream_t s) {
  const int L = (int)keys.size() - 1;
  Arena ar;
  nbr.assign(L + 1, {});
  far.assign(L + 1, {});
  std::vector<unsigned long long*> dk(L + 1);
  std::vector<int*> dn(L + 1);
  for (int l = 0; l <= L; l++) {
    const int nb = (int)keys[l].size();
    dk[l] = ar.alloc<unsigned long long>(nb);
    CK(cudaMemcpyAsync(dk[l], keys[l].data(), nb * sizeof(unsigned long long),
                       cudaMemcpyHostToDevice, s));
  }
  for (int l = 0; l <= L; l++) {
    const int nb = (int)keys[l].size();
    dn[l] = ar.alloc<int>((size_t)nb * 27);
    int* df = ar.alloc<int>((size_t)nb * 189);
    int *cb = nullptr, *ce = nullptr;
    const int np = l > 0 ? (int)keys[l - 1].size() : 0;
    if (l > 0) {
      cb = ar.alloc<int>(np);
      ce = ar.alloc<int>(np);
      k_child_range<<<(np + 127) / 128, 128, 0, s>>>(dk[l - 1], np, dk[l], nb, dim, cb, ce);
      CK_LAUNCH("k_child_range");
    }
    k_lists<<<(nb + 127) / 128, 128, 0, s>>>(dk[l], nb, l, dim, l > 0 ? dk[l - 1] : nullptr, np,
                                             l > 0 ? dn[l - 1] : nullptr, cb, ce, dn[l], df);
    CK_LAUNCH("k_lists");
    nbr[l].resize((size_t)nb * 27);
    far[l].resize((size_t)nb * 189);
    CK(cudaMemcpyAsync(nbr[l].data(), dn[l], nbr[l].size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(far[l].data(), df, far[l].size() * sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
}

void morton_decode_host(unsigned long long k, int dim, int* c) { morton_decode(k, dim, c); }

}  // namespace ifmm
