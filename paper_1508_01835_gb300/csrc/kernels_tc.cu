// kernels_tc.cu -- Schur products of the IFMM elimination on the tcgen05 tensor
// cores (mixed-precision mode).
//
// The trailing update of an eliminated box, E(R,C) -= E(R,P) E(P,P)^-1 E(P,C)
// (Sec. 2.2, Algorithm 2), is the one dense contraction of the factorisation.
// In the mixed-precision modes its product S = E(R,P) G runs here, in two
// passes:
//   1. packing: every operand (FP64 in global memory) is rounded once --
//      TF32 head and tail (x = hi + lo, IFMM_P_FP32: the three-term
//      error-compensated product of Ootomo and Yokota, 2022), TF32 head only
//      (IFMM_P_TF32), or BF16 (IFMM_P_BF16) -- with integer arithmetic (the
//      FP64 unit is the scarce one) and written in the tensor core's K-major,
//      unswizzled core-matrix layout: one 16 KB block per 128 rows and K slice
//      (32 TF32 or 64 BF16 values), zero-padded, ready to be copied verbatim;
//   2. the product: a persistent kernel, one CTA per SM looping over 128 x 128
//      output tiles, with warp roles: warp 0 streams each K slice's blocks into
//      a ring of shared-memory stages with bulk asynchronous copies (the TMA
//      engine's cp.async.bulk, completion counted in bytes on an mbarrier);
//      warp 1's elected thread issues tcgen05.mma (K = 8 per instruction for
//      TF32, 16 for BF16) into one of two FP32 accumulators in tensor memory
//      and commits each stage back to the producer; warps 2-5 read a finished
//      accumulator with tcgen05.ld (each warp its quarter of the 128 lanes =
//      output rows), write C = beta C + alpha S in FP64 and hand the
//      accumulator back, so the epilogue of one tile overlaps the MMAs of the
//      next.
// The pivot LU, the solve for G and every rank decision stay in FP64.
//
// Every wait on an mbarrier is bounded.  A wait that runs out records an
// error code in *err and its role stops; the MMA thread's last commit is
// waited for (again bounded) before the tensor memory is freed, so no MMA is
// in flight when it is.  A pipeline wait that takes more than `soft_polls`
// non-blocking polls is also recorded in *err (the caller reports
// IFMM_ERR_TIMEOUT) but keeps waiting up to the hard bound; the soft limit
// equals the hard one unless IFMM_TC_SOFT_WAIT_POLLS lowers it, which is how a
// test makes a wait run out without leaving any work in flight.
#include "internal.cuh"

namespace ifmm {

namespace tc {

constexpr int BM = 128, BN = 128;            // output tile
constexpr int BLOCK_BYTES = 16384;           // one packed operand block: 128 rows x 128 bytes of K
constexpr int NTHREADS = 192;                // warp 0 producer, warp 1 MMA, warps 2-5 epilogue
constexpr int TMEM_COLS = 256;               // two FP32 accumulators of 128 columns
constexpr int STAGE_BUDGET = 3 * 65536;      // shared-memory ring
constexpr long long SPIN_LIMIT = 1ll << 22;  // bounded waits (far above any legal wait)
constexpr int MODE_TF32 = 0, MODE_SPLIT = 1, MODE_BF16 = 2;

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


// Instruction descriptors: D = F32, A and B K-major, N >> 3 in bits 17-22,
// M >> 4 in bits 24-28; kind::tf32 with A = B = TF32 (format 2), kind::f16
// with A = B = BF16 (format 1).
constexpr uint32_t IDESC_TF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t IDESC_BF16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC_TF32), "r"(acc));
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC_BF16), "r"(acc));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// bulk asynchronous copy global -> shared (TMA engine, non-tensor form);
// completion is counted in bytes on `bar`
__device__ __forceinline__ void bulk_copy(void* dst_smem, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// v rounded to BF16 (8 significant bits, nearest, halves away from zero) as
// a 16-bit pattern, with integer arithmetic; |v| < 2^-100 flushes to zero,
// overflow becomes infinity.
__device__ __forceinline__ unsigned short round_bf16(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned int sgn = (unsigned int)(b >> 63) << 15;
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 1023 - 100) return (unsigned short)sgn;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned long long mh = (m + (1ull << 44)) >> 45;  // 8 significant bits, or 2^8
  int eh = e;
  if (mh >> 8) { mh >>= 1; eh += 1; }
  const int fe = eh - 1023 + 127;
  if (fe >= 255) return (unsigned short)(sgn | 0x7F80u);
  return (unsigned short)(sgn | ((unsigned int)fe << 7) | (unsigned int)(mh & 0x7F));
}

// Byte offset of element (row, k) inside a packed 16 KB block: core matrix
// (row / 8, k-group) at (kgroup * 16 + row / 8) * 128 and row % 8 at 16-byte
// stride inside it, where a k-group is 16 bytes of K (4 TF32 or 8 BF16
// values).  Hence the descriptors' sbo = 128 (next 8 rows) and lbo = 2048
// (next 16 bytes of K); one MMA (32 bytes of K) spans two k-groups.
constexpr uint32_t SBO = 128, LBO = (BM / 8) * 128;
__device__ __forceinline__ uint32_t block_off(int row, int kgroup) {
  return (uint32_t)((kgroup * (BM / 8) + (row >> 3)) * 128 + (row & 7) * 16);
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Pass 1: packing.  One CTA per (operand, row block, K slice) writes the
// block(s) of 128 rows x one K slice of op(X) (rows / K beyond the matrix are
// zero).  op(X)[r, k] = X[r + k ld] (trans == 0) or X[k + r ld] (trans == 1).
// ---------------------------------------------------------------------------
struct TcPack {
  const double* X;
  long long ld;
  int trans, rows, K;
  int rb, ks;          // row block and K slice of this CTA
  char* hi;            // destination block (16 KB)
  char* lo;            // tail block (split mode) or nullptr
};

__global__ void __launch_bounds__(128) k_tc_pack(const TcPack* __restrict__ packs, int mode) {
  using namespace tc;
  const TcPack P = packs[blockIdx.x];
  const int kslice = mode == MODE_BF16 ? 64 : 32;
  const int per = mode == MODE_BF16 ? 8 : 4;  // values per 16-byte k-group
  const int ngroups = kslice / per;           // 8
  for (int e = threadIdx.x; e < BM * ngroups; e += blockDim.x) {
    const int r = e % BM, g = e / BM;  // consecutive threads: consecutive rows
    const int gr = P.rb * BM + r;
    const uint32_t off = block_off(r, g);
    if (mode == MODE_BF16) {
      unsigned int w[4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        unsigned short h2[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
          const int gk = P.ks * kslice + g * per + j + q;
          double v = 0.0;
          if (gr < P.rows && gk < P.K) v = P.trans ? P.X[gk + (long long)gr * P.ld] : P.X[gr + (long long)gk * P.ld];
          h2[q] = round_bf16(v);
        }
        w[j / 2] = (unsigned int)h2[0] | ((unsigned int)h2[1] << 16);
      }
      *reinterpret_cast<uint4*>(P.hi + off) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
      float hv[4], lv[4];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int gk = P.ks * kslice + g * per + j;
        double v = 0.0;
        if (gr < P.rows && gk < P.K) v = P.trans ? P.X[gk + (long long)gr * P.ld] : P.X[gr + (long long)gk * P.ld];
        split_tf32(v, hv[j], lv[j]);
      }
      *reinterpret_cast<float4*>(P.hi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
      if (P.lo) *reinterpret_cast<float4*>(P.lo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
    }
  }
}

// ---------------------------------------------------------------------------
// Pass 2: the persistent product kernel.
// ---------------------------------------------------------------------------
struct TcTask {
  const char* A;   // packed A: block (rb, ks) at ((rb * nks + ks) * planes + plane) * 16 KB
  const char* B;   // packed op(B) (N rows), same arrangement
  double* C;
  int ldc, M, N, nks;
  double alpha, beta;
};
struct TcTile {
  int task, rb, nb;
};

__global__ void __launch_bounds__(tc::NTHREADS, 1)
    k_gemm_tc(const TcTask* __restrict__ tasks, const TcTile* __restrict__ tiles, int ntiles,
              int mode, int* __restrict__ err, long long soft_polls) {
  using namespace tc;
  extern __shared__ __align__(1024) char smem_raw[];
  char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int planes = mode == MODE_SPLIT ? 2 : 1;
  const int stage_bytes = 2 * planes * BLOCK_BYTES;  // A and B blocks of one K slice
  const int nst = STAGE_BUDGET / stage_bytes;         // 3 (split) or 6 stages
  __shared__ uint64_t full[6], empty[6], accf[2], acce[2], done;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_sh;
  volatile int& abort_s = abort_sh;  // read in loops: never cached in a register
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; a++) {
      mbar_init(&accf[a], 1);
      mbar_init(&acce[a], 128);
    }
    mbar_init(&done, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_s;
  bool late = false;

  if (warp == 0) {
    // ---- producer: stream the K slices of every tile into the ring ----
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0;
      for (int t = blockIdx.x; t < ntiles && !abort_s; t += gridDim.x) {
        const TcTile tl = tiles[t];
        const TcTask T = tasks[tl.task];
        for (int ks = 0; ks < T.nks; ks++) {
          if (!mbar_wait_soft(&empty[st], ph ^ 1u, soft_polls, &late)) { abort_s = 1; break; }
          char* sa = smem + st * stage_bytes;
          char* sb = sa + planes * BLOCK_BYTES;
          const char* ga = T.A + ((size_t)tl.rb * T.nks + ks) * planes * BLOCK_BYTES;
          const char* gb = T.B + ((size_t)tl.nb * T.nks + ks) * planes * BLOCK_BYTES;
          mbar_expect_tx(&full[st], (uint32_t)stage_bytes);
          bulk_copy(sa, ga, planes * BLOCK_BYTES, &full[st]);
          bulk_copy(sb, gb, planes * BLOCK_BYTES, &full[st]);
          if (++st == nst) { st = 0; ph ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      int st = 0, acc = 0;
      uint32_t ph = 0, aph = 0;
      for (int t = blockIdx.x; t < ntiles && !abort_s; t += gridDim.x) {
        const TcTask T = tasks[tiles[t].task];
        if (!mbar_wait_soft(&acce[acc], aph ^ 1u, soft_polls, &late)) { abort_s = 1; break; }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * BN);
        for (int ks = 0; ks < T.nks; ks++) {
          if (!mbar_wait_soft(&full[st], ph, soft_polls, &late)) { abort_s = 1; break; }
          fence_after();
          const uint32_t a_hi = smem_u32(smem + st * stage_bytes);
          const uint32_t a_lo = a_hi + BLOCK_BYTES;
          const uint32_t b_hi = a_hi + planes * BLOCK_BYTES;
          const uint32_t b_lo = b_hi + BLOCK_BYTES;
#pragma unroll
          for (int kk = 0; kk < 4; kk++) {
            const uint32_t o = kk * 2 * LBO;  // 32 bytes of K = two k-groups
            const uint32_t first = (ks > 0 || kk > 0) ? 1u : 0u;
            if (mode == MODE_SPLIT) {
              mma_tf32(d, smem_desc(a_lo + o, LBO, SBO), smem_desc(b_hi + o, LBO, SBO), first);
              mma_tf32(d, smem_desc(a_hi + o, LBO, SBO), smem_desc(b_lo + o, LBO, SBO), 1u);
              mma_tf32(d, smem_desc(a_hi + o, LBO, SBO), smem_desc(b_hi + o, LBO, SBO), 1u);
            } else if (mode == MODE_TF32) {
              mma_tf32(d, smem_desc(a_hi + o, LBO, SBO), smem_desc(b_hi + o, LBO, SBO), first);
            } else {
              mma_bf16(d, smem_desc(a_hi + o, LBO, SBO), smem_desc(b_hi + o, LBO, SBO), first);
            }
          }
          mma_commit(&empty[st]);  // the stage is free once these MMAs have read it
          if (++st == nst) { st = 0; ph ^= 1u; }
        }
        mma_commit(&accf[acc]);  // the accumulator is complete
        if (++acc == 2) { acc = 0; aph ^= 1u; }
      }
      mma_commit(&done);  // completes when every MMA issued above has
    }
  } else {
    // ---- epilogue: warps 2..5, TMEM lane quarter = warp % 4 ----
    const int q = warp & 3;
    const int rl = q * 32 + lane;  // row inside the tile
    int acc = 0;
    uint32_t aph = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const TcTile tl = tiles[t];
      const TcTask T = tasks[tl.task];
      bool ok = mbar_wait_soft(&accf[acc], aph, soft_polls, &late);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok || abort_s) { abort_s = 1; break; }
      fence_after();
      const int row = tl.rb * BM + rl;
      const uint32_t lane_addr = tmem + (uint32_t)(acc * BN) + ((uint32_t)(q * 32) << 16);
      const bool plain = (T.alpha == 1.0 && T.beta == 0.0);  // the Schur product: C = S
      for (int c0 = 0; c0 < BN; c0 += 32) {
        if (tl.nb * BN + c0 >= T.N) break;  // warp-uniform
        float v[32];
        tmem_ld32(lane_addr + c0, v);
        if (row < T.M) {
#pragma unroll
          for (int j = 0; j < 32; j++) {
            const int col = tl.nb * BN + c0 + j;
            if (col < T.N) {
              double* c = T.C + row + (long long)col * T.ldc;
              const double s = widen(v[j]);
              *c = plain ? s : ((T.beta == 0.0) ? T.alpha * s : T.beta * (*c) + T.alpha * s);
            }
          }
        }
      }
      fence_before();
      mbar_arrive(&acce[acc]);  // hand the accumulator back
      if (++acc == 2) { acc = 0; aph ^= 1u; }
    }
  }
  // every thread waits for the MMA thread's last commit (so no MMA is in
  // flight), then warp 1 frees the tensor memory
  __syncthreads();
  if (!mbar_wait(&done, 0u)) abort_s = 1;
  __syncthreads();
  if (threadIdx.x == 0 && (late || abort_s)) atomicExch(err, 1);
  if (late && threadIdx.x != 0) atomicExch(err, 1);
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// Ring of stages (3 x 64 KB), 1 KB for alignment and 16 KB of slack past the
// last stage so that no descriptor walk can leave the CTA's allocation.
static size_t gemm_tc_smem() { return (size_t)tc::STAGE_BUDGET + 1024 + 16 * 1024; }

void run_gemms_tc(Arena& ar, const std::vector<GemmTask>& tasks, int prec, int* d_err,
                  cudaStream_t s) {
  using namespace tc;
  const int mode = prec == IFMM_P_FP32 ? MODE_SPLIT : (prec == IFMM_P_BF16 ? MODE_BF16 : MODE_TF32);
  const int planes = mode == MODE_SPLIT ? 2 : 1;
  const int kslice = mode == MODE_BF16 ? 64 : 32;
  std::vector<TcPack> packs;
  std::vector<TcTask> tt;
  std::vector<TcTile> tiles;
  std::vector<GemmTask> zero_k;
  double flops = 0.0;
  for (const GemmTask& t : tasks) {
    if (t.M <= 0 || t.N <= 0) continue;
    validate(t);
    if (t.K <= 0) { zero_k.push_back(t); continue; }
    flops += 2.0 * t.M * (double)t.N * t.K;
    const int nmb = (t.M + BM - 1) / BM, nnb = (t.N + BN - 1) / BN, nks = (t.K + kslice - 1) / kslice;
    char* pa = ar.alloc<char>((size_t)nmb * nks * planes * BLOCK_BYTES);
    char* pb = ar.alloc<char>((size_t)nnb * nks * planes * BLOCK_BYTES);
    for (int rb = 0; rb < nmb; rb++)
      for (int ks = 0; ks < nks; ks++) {
        char* h = pa + ((size_t)rb * nks + ks) * planes * BLOCK_BYTES;
        packs.push_back({t.A, t.lda, t.transA, t.M, t.K, rb, ks, h,
                         planes == 2 ? h + BLOCK_BYTES : nullptr});
      }
    for (int nb = 0; nb < nnb; nb++)
      for (int ks = 0; ks < nks; ks++) {
        char* h = pb + ((size_t)nb * nks + ks) * planes * BLOCK_BYTES;
        packs.push_back({t.B, t.ldb, !t.transB, t.N, t.K, nb, ks, h,
                         planes == 2 ? h + BLOCK_BYTES : nullptr});
      }
    const int ti = (int)tt.size();
    tt.push_back({pa, pb, t.C, t.ldc, t.M, t.N, nks, t.alpha, t.beta});
    for (int nb = 0; nb < nnb; nb++)
      for (int rb = 0; rb < nmb; rb++) tiles.push_back({ti, rb, nb});
  }
  if (!zero_k.empty()) run_gemms(ar, zero_k, s);  // C = beta C
  if (tiles.empty()) return;
  {
    Prof p("k_tc_pack", 0.0, (double)packs.size() * (2.0 * BLOCK_BYTES * planes), s);
    k_tc_pack<<<(int)packs.size(), 128, 0, s>>>(upload(ar, packs, s), mode);
    CK_LAUNCH("k_tc_pack");
  }
  int dev = 0, nsm = 1;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  set_max_dynamic_smem((const void*)k_gemm_tc, (int)gemm_tc_smem());
  // test hook: a lower reporting limit for the pipeline waits (see above)
  long long soft = SPIN_LIMIT;
  if (const char* e = std::getenv("IFMM_TC_SOFT_WAIT_POLLS")) {
    const long long v = std::atoll(e);
    if (v >= 1) soft = std::min(v, SPIN_LIMIT);
  }
  const int grid = std::min((int)tiles.size(), nsm);
  const char* name = mode == MODE_SPLIT ? "k_gemm_tc_3xtf32" : (mode == MODE_BF16 ? "k_gemm_tc_bf16"
                                                                                 : "k_gemm_tc_tf32");
  Prof p(name, flops, 0.0, s);
  k_gemm_tc<<<grid, NTHREADS, gemm_tc_smem(), s>>>(upload(ar, tt, s), upload(ar, tiles, s),
                                                   (int)tiles.size(), mode, d_err, soft);
  CK_LAUNCH("k_gemm_tc");
}

}  // namespace ifmm
