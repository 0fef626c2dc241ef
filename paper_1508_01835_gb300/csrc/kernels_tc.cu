// kernels_tc.cu -- Schur products of the IFMM elimination on the tcgen05 tensor
// cores (mixed-precision mode).
//
// The trailing update of an eliminated box, E(R,C) -= E(R,P) E(P,P)^-1 E(P,C)
// (Sec. 2.2, Algorithm 2), is the one dense contraction of the factorisation.
// In the mixed-precision mode its product S = E(R,P) G runs here:
//   * operands are FP64 in global memory; each CTA rounds a 128 x 32 slice of
//     A and of B to TF32 (round to nearest, with integer arithmetic: the FP64
//     unit is the scarce one) and stores them in shared memory in the tensor
//     core's K-major, unswizzled core-matrix layout;
//   * IFMM_P_FP32 splits every operand into a TF32 head and a TF32 tail
//     (x = hi + lo) and accumulates hi*hi + hi*lo + lo*hi -- the three-term
//     error-compensated TF32 product of Ootomo and Yokota (2022), close to
//     FP32 accuracy; IFMM_P_TF32 accumulates hi*hi only;
//   * one elected thread issues tcgen05.mma (kind::tf32, M = 128, N = 128,
//     K = 8 per instruction) into an FP32 accumulator in tensor memory and
//     commits each stage to an mbarrier; two stages let the next slice load
//     while the tensor core works on the previous one;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w owns lanes
//     32w .. 32w + 31, i.e. output rows) and writes C = beta C + alpha S in FP64.
// The pivot LU, the solve for G and every rank decision stay in FP64.
//
// Every wait on an mbarrier is bounded; a wait that runs out records an error
// code in *err and the CTA still drains its own tensor-core work (again with a
// bound) and frees its tensor memory before it returns.  A pipeline wait that
// takes more than `soft_polls` polls is also recorded in *err (the caller
// reports IFMM_ERR_TIMEOUT) but keeps waiting up to the hard bound; the soft
// limit equals the hard one unless IFMM_TC_SOFT_WAIT_POLLS lowers it (then the
// first polls are non-blocking test_wait), which is how a test makes a wait run
// out without leaving any work in flight.
#include "internal.cuh"

namespace ifmm {

namespace tc {

constexpr int BM = 128, BN = 128, BK = 32;  // output tile and K slice per stage
constexpr int NTHREADS = 128;
constexpr int TMEM_COLS = 128;              // FP32 accumulator: 128 lanes x 128 columns
// one operand slice: 128 rows x 32 TF32 values = 16 KB
constexpr int SLICE_BYTES = BM * BK * 4;
constexpr long long SPIN_LIMIT = 1ll << 22;  // bounded waits (far above any legal wait)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, no swizzle.  Core matrices are
// 8 rows x 16 bytes stored as 128 contiguous bytes; `lbo` is the byte distance
// between core matrices adjacent in K, `sbo` between core matrices adjacent in
// the row (M or N) direction.  Bits 46-47 carry the descriptor version (1).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;  // base offset 0, absolute LBO mode off, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false when the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < SPIN_LIMIT; it++)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Pipeline wait with a reporting limit.  With a limit below the hard bound the
// wait first makes `soft` non-blocking polls (test_wait); if the phase is not
// complete by then the wait counts as late (*late = true, reported as
// IFMM_ERR_TIMEOUT) and continues with the blocking polls up to the hard
// bound, so the pipeline's phase accounting stays exact and no tensor memory
// is freed while its MMAs run.  Returns false only when the hard bound ran out.
__device__ __forceinline__ bool mbar_wait_soft(uint64_t* bar, uint32_t parity, long long soft,
                                               bool* late) {
  if (soft < SPIN_LIMIT) {
    for (long long it = 0; it < soft; it++)
      if (mbar_test(bar, parity)) return true;
    *late = true;
  }
  return mbar_wait(bar, parity);
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 lanes x 32 columns of 32-bit accumulator into r[0..31] (this warp's lanes)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* r) {
  uint32_t v[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) r[i] = __uint_as_float(v[i]);
}

// FP64 <-> FP32 conversions with integer arithmetic only.  On this part the
// FP64 unit executes a few operations per clock per SM, and double/float
// conversions and subtractions would run there; integer and FP32 units are
// tens of times wider.
//
// split_tf32: v = hi + lo + (rounding), with hi = v rounded to 11 significant
// bits (TF32 precision, nearest, halves rounded away from zero) and lo = the
// exact remainder v - hi rounded to 11 significant bits; both returned as FP32
// bit patterns.  |v| < 2^-100 flushes to zero (far below what an FP32
// accumulation resolves next to the operands this kernel sees); |v| >= 2^128
// becomes infinity.
__device__ __forceinline__ void split_tf32(double v, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned int sgn = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF);  // biased exponent
  if (e < 1023 - 100) {
    hi = __uint_as_float(sgn);
    lo = __uint_as_float(sgn);
    return;
  }
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // 53-bit significand
  const unsigned long long mr = ((m + (1ull << 41)) >> 42) << 42;       // m rounded to 11 bits
  unsigned long long mh = mr >> 42;                                     // 11 bits, or 2^11
  int eh = e;
  if (mh >> 11) { mh >>= 1; eh += 1; }
  const int fe = eh - 1023 + 127;
  hi = __uint_as_float(fe >= 255 ? (sgn | 0x7F800000u)
                                 : (sgn | ((unsigned int)fe << 23) |
                                    ((unsigned int)(mh & 0x3FF) << 13)));
  const long long r = (long long)m - (long long)mr;  // |r| <= 2^41, value r 2^(e-1075)
  if (r == 0) {
    lo = __uint_as_float(0u);
    return;
  }
  unsigned long long ar = (unsigned long long)(r < 0 ? -r : r);
  int p = 63 - __clzll((long long)ar);  // leading bit of |r|
  unsigned long long ml;
  if (p > 10) {
    ml = (ar + (1ull << (p - 11))) >> (p - 10);
    if (ml >> 11) { ml >>= 1; p += 1; }
  } else {
    ml = ar << (10 - p);
  }
  const int le = p + e - 1075 + 127;  // biased FP32 exponent of |r| 2^(e-1075)
  const unsigned int ls = (r < 0) ? (sgn ^ 0x80000000u) : sgn;
  lo = __uint_as_float(le <= 0 ? ls : (ls | ((unsigned int)le << 23) |
                                       ((unsigned int)(ml & 0x3FF) << 13)));
}

// Exact FP32 -> FP64 widening (FP32 subnormals flush to zero).
__device__ __forceinline__ double widen(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
  const unsigned int ex = (u >> 23) & 0xFF;
  const unsigned long long mant = (unsigned long long)(u & 0x7FFFFF) << 29;
  if (ex == 0) return __longlong_as_double((long long)sgn);
  const unsigned long long de = (ex == 255) ? 0x7FFull : (unsigned long long)(ex + 896);
  return __longlong_as_double((long long)(sgn | (de << 52) | mant));
}

// Byte offset of element (row, k) of a 128 x 32 K-major slice: core matrix
// (row / 8, k / 4) at ((k / 4) * 16 + row / 8) * 128, inside it row % 8 at
// 16-byte stride and k % 4 at 4-byte stride.  Hence sbo = 128 (next 8 rows)
// and lbo = 2048 (next 4 values of k).
constexpr uint32_t SBO = 128, LBO = (BM / 8) * 128;
__device__ __forceinline__ uint32_t slice_off(int row, int kq) {  // kq = k / 4
  return (uint32_t)((kq * (BM / 8) + (row >> 3)) * 128 + (row & 7) * 16);
}

// Load op(X)[row0 + r, k0 + k] for r < 128, k < 32 (zero outside rows x K),
// rounded to TF32 (head; tail = TF32 of the remainder when `split`).
// op(X)[m, k] = X[m + k ld] (trans == 0) or X[k + m ld] (trans == 1).
__device__ __forceinline__ void load_slice(const double* __restrict__ X, int ld, int trans,
                                           int rows, int K, int row0, int k0, char* hi, char* lo,
                                           bool split) {
  // 128 rows x 8 groups of 4 values; thread t takes row t % 128 for trans == 0
  // (consecutive threads read consecutive rows: coalesced) and the 4 values of
  // one k-group (contiguous for trans == 1).
  for (int e = threadIdx.x; e < BM * (BK / 4); e += NTHREADS) {
    const int r = e % BM, kq = e / BM;
    const int gr = row0 + r;
    float4 h, l;
    float hv[4], lv[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int gk = k0 + kq * 4 + j;
      double v = 0.0;
      if (gr < rows && gk < K) v = trans ? X[gk + (long long)gr * ld] : X[gr + (long long)gk * ld];
      split_tf32(v, hv[j], lv[j]);
      if (!split) lv[j] = 0.0f;
    }
    h = make_float4(hv[0], hv[1], hv[2], hv[3]);
    l = make_float4(lv[0], lv[1], lv[2], lv[3]);
    const uint32_t off = slice_off(r, kq);
    *reinterpret_cast<float4*>(hi + off) = h;
    if (split) *reinterpret_cast<float4*>(lo + off) = l;
  }
}

}  // namespace tc

// One 128 x 128 output tile per CTA.  Shared memory: 2 stages x {A hi, B hi,
// A lo, B lo} slices (the lo slices only in split mode) + barriers.
__global__ void __launch_bounds__(tc::NTHREADS) k_gemm_tc(const GemmTask* __restrict__ tasks,
                                                          const GemmTile* __restrict__ tiles,
                                                          int split, int* __restrict__ err,
                                                          long long soft_polls) {
  using namespace tc;
  extern __shared__ __align__(1024) char smem_raw[];
  // 1024-byte alignment of the operand area
  char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nsl = split ? 4 : 2;  // slices per stage
  char* stage[2] = {smem, smem + nsl * SLICE_BYTES};
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_base_s;
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask t = tasks[tl.task];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_s;

  const int nk = (t.K + BK - 1) / BK;
  bool ok = true, late = false;
  for (int kt = 0; kt < nk; kt++) {
    const int s = kt & 1;
    if (kt >= 2) {
      // the MMAs that read this stage two slices ago must be done
      if (!mbar_wait_soft(&bar[s], (uint32_t)(((kt - 2) >> 1) & 1), soft_polls, &late)) ok = false;
    }
    char* st = stage[s];
    load_slice(t.A, t.lda, t.transA, t.M, t.K, tl.m0, kt * BK, st, split ? st + 2 * SLICE_BYTES : nullptr,
               split != 0);
    load_slice(t.B, t.ldb, !t.transB, t.N, t.K, tl.n0, kt * BK, st + SLICE_BYTES,
               split ? st + 3 * SLICE_BYTES : nullptr, split != 0);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_after();
      const uint32_t a_hi = smem_u32(st), b_hi = smem_u32(st + SLICE_BYTES);
      const uint32_t a_lo = smem_u32(st + 2 * SLICE_BYTES), b_lo = smem_u32(st + 3 * SLICE_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 8; kk++) {
        const uint32_t o = kk * 2 * LBO;  // 8 values of k = two core matrices
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        if (split) {
          mma_tf32(tmem, smem_desc(a_lo + o, LBO, SBO), smem_desc(b_hi + o, LBO, SBO), acc);
          mma_tf32(tmem, smem_desc(a_hi + o, LBO, SBO), smem_desc(b_lo + o, LBO, SBO), 1u);
          mma_tf32(tmem, smem_desc(a_hi + o, LBO, SBO), smem_desc(b_hi + o, LBO, SBO), 1u);
        } else {
          mma_tf32(tmem, smem_desc(a_hi + o, LBO, SBO), smem_desc(b_hi + o, LBO, SBO), acc);
        }
      }
      mma_commit(&bar[s]);
    }
  }
  // wait for the last commit of each stage (every thread, so all see the result)
  for (int s = 0; s < 2; s++) {
    const int n_s = (nk - s + 1) / 2;  // commits on stage s
    if (n_s > 0 && !mbar_wait_soft(&bar[s], (uint32_t)((n_s - 1) & 1), soft_polls, &late)) ok = false;
  }
  if (late) atomicExch(err, 1);  // results are complete; the lateness is reported
  // one verdict for the whole CTA: the epilogue's tcgen05.ld is warp-collective
  ok = __syncthreads_and(ok) != 0;
  fence_after();
  if (ok && nk > 0) {
    const int row = tl.m0 + warp * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < BN; c0 += 32) {
      if (tl.n0 + c0 >= t.N) break;  // warp-uniform
      float v[32];
      tc::tmem_ld32(lane_addr + c0, v);
      if (row < t.M) {
        const bool plain = (t.alpha == 1.0 && t.beta == 0.0);  // the Schur product: C = S
#pragma unroll
        for (int j = 0; j < 32; j++) {
          const int col = tl.n0 + c0 + j;
          if (col < t.N) {
            double* c = t.C + row + (long long)col * t.ldc;
            const double s = widen(v[j]);
            *c = plain ? s : ((t.beta == 0.0) ? t.alpha * s : t.beta * (*c) + t.alpha * s);
          }
        }
      }
    }
  } else if (nk == 0) {
    // K == 0: C = beta C
    for (int e = threadIdx.x; e < BM * BN; e += NTHREADS) {
      const int r = tl.m0 + e % BM, c = tl.n0 + e / BM;
      if (r < t.M && c < t.N) {
        double* p = t.C + r + (long long)c * t.ldc;
        *p = (t.beta == 0.0) ? 0.0 : t.beta * (*p);
      }
    }
  }
  if (!ok) {
    // a wait ran out: record it, then give the committed work one more bounded
    // chance to finish before the accumulator's tensor memory is freed
    if (threadIdx.x == 0) atomicExch(err, 1);
    for (int s = 0; s < 2; s++) {
      const int n_s = (nk - s + 1) / 2;
      if (n_s > 0) mbar_wait(&bar[s], (uint32_t)((n_s - 1) & 1));
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// Two stages of slices, 1 KB for alignment, and 48 KB of slack past the last
// slice so that no descriptor walk can leave the CTA's allocation.
size_t gemm_tc_smem(bool split) {
  return (size_t)2 * (split ? 4 : 2) * tc::SLICE_BYTES + 1024 + 48 * 1024;
}

void gemm_tc_tiles(const GemmTask& t, int ti, std::vector<GemmTile>& tiles) {
  if (t.M <= 0 || t.N <= 0) return;
  for (int n0 = 0; n0 < t.N; n0 += tc::BN)
    for (int m0 = 0; m0 < t.M; m0 += tc::BM) tiles.push_back({ti, m0, n0});
}

void launch_gemm_tc(const GemmTask* d_tasks, const GemmTile* d_tiles, int ntiles, bool split,
                    int* d_err, cudaStream_t s, double flops) {
  if (ntiles <= 0) return;
  set_max_dynamic_smem((const void*)k_gemm_tc, (int)gemm_tc_smem(true));
  Prof p(split ? "k_gemm_tc_3xtf32" : "k_gemm_tc_tf32", flops, 0.0, s);
  // test hook: a lower reporting limit for the pipeline waits (see k_gemm_tc)
  long long soft = tc::SPIN_LIMIT;
  if (const char* e = std::getenv("IFMM_TC_SOFT_WAIT_POLLS")) {
    const long long v = std::atoll(e);
    if (v >= 1) soft = std::min(v, tc::SPIN_LIMIT);
  }
  k_gemm_tc<<<ntiles, tc::NTHREADS, gemm_tc_smem(split), s>>>(d_tasks, d_tiles, split ? 1 : 0,
                                                             d_err, soft);
  CK_LAUNCH("k_gemm_tc");
}

void run_gemms_tc(Arena& ar, const std::vector<GemmTask>& tasks, bool split, int* d_err,
                  cudaStream_t s) {
  std::vector<GemmTask> kept;
  std::vector<GemmTile> tiles;
  double flops = 0.0;
  for (const GemmTask& t : tasks) {
    if (t.M <= 0 || t.N <= 0) continue;
    validate(t);
    flops += 2.0 * t.M * (double)t.N * std::max(t.K, 0);
    gemm_tc_tiles(t, (int)kept.size(), tiles);
    kept.push_back(t);
  }
  if (tiles.empty()) return;
  launch_gemm_tc(upload(ar, kept, s), upload(ar, tiles, s), (int)tiles.size(), split, d_err, s,
                 flops);
}

}  // namespace ifmm
