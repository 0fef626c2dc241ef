// kernels_m2l.cu -- block rows whose blocks are all nd x nd: the FMM's M2M,
// M2L and L2L translations (Sec. 2.1: multipole-to-multipole, multipole-to-
// local and local-to-local operators of the Chebyshev interpolant).
//
// A row is one target box: y_i = sum_e A_e x_e over its entries (the boxes of
// its interaction list with the M2L table of their offset, plus the L2L term
// from the parent; or its children with the transposed transfers for M2M).
// One warp computes one row for up to 32 right-hand sides:
//   * each entry's table (nd columns of ndp entries, zero padded) and its
//     source coefficients (32 columns of ndp entries) are copied with cp.async
//     into a double-buffered per-warp shared-memory stage while the previous
//     entry is multiplied;
//   * ndp = 8 RG with RG the smallest power of two with 8 RG >= nd (nd <= 64);
//     a pass of 32 columns gives lane (rg, cg) the 8 rows rg*8 .. rg*8+7 of RG
//     columns in registers (RG row groups, 32 / RG column groups); passes of
//     at most 8 columns or of one column use narrower tiles (UniTile), so a
//     single right-hand side does not pay for 32; a lane reads its table
//     values as 16-byte broadcasts and its source values from a column stride
//     of ndp + 16 / sizeof(T) elements (no bank conflicts);
//   * the sums over entries are taken in entry order, so results do not depend
//     on scheduling.
// Coefficient vectors are stored with ndp entries per box (16-byte aligned).
#include "internal.cuh"

namespace ifmm {

namespace {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;  // 0 source bytes: the 16 bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int N>
__device__ __forceinline__ void load8_any(const float* p, float (&a)[N]) {
#pragma unroll
  for (int q = 0; q < N / 4; q++) {
    const float4 u = reinterpret_cast<const float4*>(p)[q];
    a[4 * q] = u.x; a[4 * q + 1] = u.y; a[4 * q + 2] = u.z; a[4 * q + 3] = u.w;
  }
}
template <int N>
__device__ __forceinline__ void load8_any(const double* p, double (&a)[N]) {
#pragma unroll
  for (int q = 0; q < N / 2; q++) {
    const double2 v = reinterpret_cast<const double2*>(p)[q];
    a[2 * q] = v.x;
    a[2 * q + 1] = v.y;
  }
}

}  // namespace

constexpr int UNI_MAX_WARPS = 4;
constexpr int UNI_NB = 32;

// Lane tiling of an NDP x NBT output tile (NBT columns per pass): RGN row
// groups of RPL rows times CGN column groups of CPL columns (columns j * CGN +
// cg of lane cg); lanes beyond RGN * CGN idle (single-column passes of small
// tables only).
template <int NDP, int NBT>
struct UniTile {
  static constexpr int RPL = NBT == 32 ? 8 : NBT == 8 ? NDP / 8 : (NDP >= 32 ? NDP / 32 : 1);
  static constexpr int RGN = NDP / RPL;
  static constexpr int CGN = NBT == 32 ? 32 / RGN : NBT == 8 ? 4 : 1;
  static constexpr int CPL = NBT / CGN;
  static_assert(RGN * CGN <= 32 && CGN * CPL == NBT && RGN * RPL == NDP, "tile");
};

template <class T>
__host__ __device__ constexpr int uni_xs(int ndp) {
  return ndp + 16 / (int)sizeof(T);  // column stride of the staged source block
}
template <class T>
__host__ __device__ constexpr int uni_stage(int nd, int ndp, int nbt) {
  return nd * ndp + nbt * uni_xs<T>(ndp);  // elements per stage
}

template <class T, int N>
__device__ __forceinline__ void loadn(const T* p, T (&a)[N]) {
  if constexpr (N * sizeof(T) % 16 == 0) {
    load8_any(p, a);
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) a[i] = p[i];
  }
}

template <class T, int NDP, int NBT>
__global__ void __launch_bounds__(32 * UNI_MAX_WARPS)
    k_uniform(const UniRow<T>* __restrict__ rows, const UniEnt<T>* __restrict__ ents, int nrows,
              int nd, int c0, int nb) {
  using Tl = UniTile<NDP, NBT>;
  constexpr int RPL = Tl::RPL, RGN = Tl::RGN, CGN = Tl::CGN, CPL = Tl::CPL;
  constexpr int VN = 16 / (int)sizeof(T);
  constexpr int XS = uni_xs<T>(NDP);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * (int)(blockDim.x >> 5) + warp;
  if (row >= nrows) return;  // warp-uniform; no block-wide barrier below
  const int stage = uni_stage<T>(nd, NDP, NBT);
  T* buf = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 2 * stage;
  const UniRow<T> R = rows[row];
  const int rg = lane / CGN, cg = lane % CGN;
  const bool active = rg < RGN;

  auto prefetch = [&](int e, T* st) {
    const UniEnt<T> E = ents[R.e0 + e];
    T* As = st;
    T* Xs = st + nd * NDP;
    const int achunks = nd * (NDP / VN);
    for (int q = lane; q < achunks; q += 32) cp_async16(As + q * VN, E.A + (size_t)q * VN, true);
    const int xchunks = NBT * (NDP / VN);
    for (int q = lane; q < xchunks; q += 32) {
      const int c = q / (NDP / VN), k4 = q % (NDP / VN);
      const bool ok = c < nb;
      const T* src = E.x + (ok ? (long long)(c0 + c) * E.ldx : 0) + k4 * VN;
      cp_async16(Xs + c * XS + k4 * VN, src, ok);
    }
    cp_async_commit();
  };

  T acc[RPL][CPL];
#pragma unroll
  for (int i = 0; i < RPL; i++)
#pragma unroll
    for (int j = 0; j < CPL; j++) acc[i][j] = T(0);

  if (R.ne > 0) prefetch(0, buf);
  for (int e = 0; e < R.ne; e++) {
    T* cur = buf + (e & 1) * stage;
    if (e + 1 < R.ne) {
      prefetch(e + 1, buf + ((e + 1) & 1) * stage);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    if (active) {
      const T* As = cur + rg * RPL;
      const T* Xs = cur + nd * NDP + cg * XS;
#pragma unroll 3
      for (int k = 0; k < nd; k++) {
        T a[RPL];
        loadn<T, RPL>(As + k * NDP, a);
        T xv[CPL];
#pragma unroll
        for (int j = 0; j < CPL; j++) xv[j] = Xs[(j * CGN) * XS + k];
#pragma unroll
        for (int i = 0; i < RPL; i++)
#pragma unroll
          for (int j = 0; j < CPL; j++) acc[i][j] = fma(a[i], xv[j], acc[i][j]);
      }
    }
    __syncwarp();  // the stage is refilled by the next prefetch
  }
  if (!active) return;
#pragma unroll
  for (int j = 0; j < CPL; j++) {
    const int c = j * CGN + cg;
    if (c >= nb) continue;
    T* y = R.y + (long long)(c0 + c) * R.ldy;
#pragma unroll
    for (int i = 0; i < RPL; i++) {
      const int r = rg * RPL + i;
      if (r < nd) y[r] = acc[i][j];
    }
  }
}

int uniform_ndp(int nd) {
  int rg = 1;
  while (8 * rg < nd) rg *= 2;
  return 8 * rg;
}
bool uniform_supported(int nd) { return nd >= 1 && nd <= 64; }

template <class T>
UniPlan<T> plan_uniform(Arena& ar, const std::vector<UniRow<T>>& rows,
                        const std::vector<UniEnt<T>>& ents, int nd, int cap, cudaStream_t s) {
  UniPlan<T> P;
  if (rows.empty()) return P;
  if (!uniform_supported(nd)) throw Error(IFMM_ERR_INVALID_ARG, "uniform block rows: nd > 64");
  const int ndp = uniform_ndp(nd);
  const size_t es = sizeof(T);
  for (const UniRow<T>& R : rows) {
    Ranges::check(R.y, es * ((size_t)(cap - 1) * R.ldy + nd), "uniform y");
    if ((reinterpret_cast<uintptr_t>(R.y) % 16) || ((R.ldy * es) % 16))
      throw Error(IFMM_ERR_CUDA, "uniform block rows: y not 16-byte aligned");
    for (int e = R.e0; e < R.e0 + R.ne; e++) {
      const UniEnt<T>& E = ents[e];
      Ranges::check(E.A, es * (size_t)nd * ndp, "uniform A");
      Ranges::check(E.x, es * ((size_t)(cap - 1) * E.ldx + ndp), "uniform x");
      if ((reinterpret_cast<uintptr_t>(E.A) % 16) || (reinterpret_cast<uintptr_t>(E.x) % 16) ||
          ((E.ldx * es) % 16))
        throw Error(IFMM_ERR_CUDA, "uniform block rows: operands not 16-byte aligned");
    }
    P.flops += 2.0 * nd * nd * R.ne;
    P.bytes += es * ((double)nd * nd * R.ne + (double)nd * R.ne + nd);
  }
  P.rows = upload(ar, rows, s);
  P.ents = upload(ar, ents, s);
  P.nrows = (int)rows.size();
  P.nd = nd;
  P.ndp = ndp;
  return P;
}

// warps per CTA: as many (<= 4) as fit 200 KB of double-buffered stages
template <class T>
static int uni_warps(int nd, int ndp, int nbt) {
  const int per = 2 * uni_stage<T>(nd, ndp, nbt) * (int)sizeof(T);
  return std::max(1, std::min(UNI_MAX_WARPS, (200 << 10) / per));
}

template <class T, int NDP, int NBT>
static void launch_tile(const UniPlan<T>& p, int c0, int nb, cudaStream_t s) {
  const int warps = uni_warps<T>(p.nd, NDP, NBT);
  const int smem = warps * 2 * uni_stage<T>(p.nd, NDP, NBT) * (int)sizeof(T);
  set_max_dynamic_smem((const void*)k_uniform<T, NDP, NBT>, smem);
  const int grid = (p.nrows + warps - 1) / warps;
  k_uniform<T, NDP, NBT><<<grid, 32 * warps, smem, s>>>(p.rows, p.ents, p.nrows, p.nd, c0, nb);
  CK_LAUNCH("k_uniform");
}

template <class T, int NDP>
static void launch_ndp(const UniPlan<T>& p, int c0, int nb, cudaStream_t s) {
  if (nb <= 1) launch_tile<T, NDP, 1>(p, c0, nb, s);
  else if (nb <= 8) launch_tile<T, NDP, 8>(p, c0, nb, s);
  else launch_tile<T, NDP, 32>(p, c0, nb, s);
}

// passes of up to 32 columns; each pass with the narrowest tile (1, 8, 32)
template <class T>
void launch_uniform(const UniPlan<T>& p, int nrhs, cudaStream_t s) {
  if (p.nrows <= 0 || nrhs <= 0) return;
  const char* name = sizeof(T) == 4 ? "k_uniform_f32" : "k_uniform_f64";
  for (int c0 = 0; c0 < nrhs; c0 += UNI_NB) {
    const int nb = std::min(UNI_NB, nrhs - c0);
    Prof pr(name, p.flops * nb, p.bytes, s);
    switch (p.ndp) {
      case 8: launch_ndp<T, 8>(p, c0, nb, s); break;
      case 16: launch_ndp<T, 16>(p, c0, nb, s); break;
      case 32: launch_ndp<T, 32>(p, c0, nb, s); break;
      default: launch_ndp<T, 64>(p, c0, nb, s); break;
    }
  }
}

template UniPlan<float> plan_uniform(Arena&, const std::vector<UniRow<float>>&,
                                     const std::vector<UniEnt<float>>&, int, int, cudaStream_t);
template UniPlan<double> plan_uniform(Arena&, const std::vector<UniRow<double>>&,
                                      const std::vector<UniEnt<double>>&, int, int, cudaStream_t);
template void launch_uniform(const UniPlan<float>&, int, cudaStream_t);
template void launch_uniform(const UniPlan<double>&, int, cudaStream_t);

// dst[b][k][r] (r < ndp, zero for r >= nd) = src[b][r + k * nd] (or its
// transpose): count tables nd x nd (column-major) to the padded column layout
// the kernel stages
template <class T>
__global__ void k_pad_tables(const double* __restrict__ src, T* __restrict__ dst, int count,
                             int nd, int ndp, int transpose) {
  const long long n = (long long)count * nd * ndp;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % ndp);
    const long long t = e / ndp;
    const int k = (int)(t % nd);
    const long long b = t / nd;
    const double* A = src + b * nd * nd;
    dst[e] = r < nd ? (T)(transpose ? A[k + (long long)r * nd] : A[r + (long long)k * nd]) : T(0);
  }
}

template <class T>
void launch_pad_tables(const double* src, T* dst, int count, int nd, bool transpose,
                       cudaStream_t s) {
  const int ndp = uniform_ndp(nd);
  const long long n = (long long)count * nd * ndp;
  if (n <= 0) return;
  Ranges::check(src, sizeof(double) * (size_t)count * nd * nd, "pad src");
  Ranges::check(dst, sizeof(T) * (size_t)n, "pad dst");
  k_pad_tables<T><<<(int)std::min<long long>(4096, (n + 255) / 256), 256, 0, s>>>(
      src, dst, count, nd, ndp, transpose ? 1 : 0);
  CK_LAUNCH("k_pad_tables");
}
template void launch_pad_tables(const double*, float*, int, int, bool, cudaStream_t);
template void launch_pad_tables(const double*, double*, int, int, bool, cudaStream_t);

}  // namespace ifmm
