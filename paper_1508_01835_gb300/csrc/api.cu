// api.cu -- the extern "C" boundary of the IFMM library (include/ifmm.h).
// Every entry point converts exceptions into an ifmm_status and records the
// message in the context.
#include <cstdio>

#include "factor.cuh"

using namespace ifmm;

namespace {
template <class F>
ifmm_status guard(ifmm_ctx* ctx, F&& fn) {
  try {
    fn();
    return IFMM_OK;
  } catch (const Error& e) {
    if (ctx) ctx->last_error = e.what();
    return e.st;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->last_error = "host out of memory";
    return IFMM_ERR_OOM;
  } catch (const std::exception& e) {
    if (ctx) ctx->last_error = e.what();
    return IFMM_ERR_CUDA;
  }
}
inline cudaStream_t st(ifmm_stream s) { return reinterpret_cast<cudaStream_t>(s); }
}  // namespace

extern "C" {

const char* ifmm_status_string(ifmm_status s) {
  switch (s) {
    case IFMM_OK: return "ok";
    case IFMM_ERR_INVALID_ARG: return "invalid argument";
    case IFMM_ERR_OOM: return "out of memory";
    case IFMM_ERR_CUDA: return "CUDA error";
    case IFMM_ERR_SINGULAR_PIVOT: return "singular pivot block";
    case IFMM_ERR_NOT_CONVERGED: return "GMRES did not converge";
    case IFMM_ERR_TIMEOUT: return "timeout";
    case IFMM_ERR_BUDGET: return "memory budget exceeded";
    case IFMM_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

ifmm_status ifmm_ctx_create(int device, ifmm_ctx** out) {
  if (!out) return IFMM_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return device < 0 ? IFMM_ERR_INVALID_ARG : IFMM_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return IFMM_ERR_CUDA;
  auto* c = new ifmm_ctx();
  c->device = device;
  *out = c;
  return IFMM_OK;
}

void ifmm_ctx_destroy(ifmm_ctx* ctx) { delete ctx; }

const char* ifmm_last_error(const ifmm_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

static ifmm_status system_create_common(ifmm_ctx* ctx, const double* pts, bool host, long long N,
                                        const ifmm_kernel* k, const ifmm_options* opt,
                                        ifmm_stream stream, ifmm_system** out) {
  if (!ctx || !out || !pts) return IFMM_ERR_INVALID_ARG;
  *out = nullptr;
  return guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    *out = system_create(ctx, pts, host, N, k, opt, st(stream));
  });
}

ifmm_status ifmm_system_create(ifmm_ctx* ctx, const double* pts, long long N,
                               const ifmm_kernel* kernel, const ifmm_options* opt,
                               ifmm_stream stream, ifmm_system** out) {
  return system_create_common(ctx, pts, false, N, kernel, opt, stream, out);
}

ifmm_status ifmm_system_create_host(ifmm_ctx* ctx, const double* pts_host, long long N,
                                    const ifmm_kernel* kernel, const ifmm_options* opt,
                                    ifmm_stream stream, ifmm_system** out) {
  return system_create_common(ctx, pts_host, true, N, kernel, opt, stream, out);
}

void ifmm_system_destroy(ifmm_system* sys) { delete sys; }

ifmm_status ifmm_system_get_info(const ifmm_system* sys, ifmm_system_info* info) {
  if (!sys || !info) return IFMM_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  info->N = sys->N;
  info->dim = sys->dim;
  info->levels = sys->L;
  info->max_leaf = sys->max_leaf;
  info->edge = sys->edge;
  for (int d = 0; d < 3; d++) info->lo[d] = sys->lo[d];
  if (sys->L == 0) info->boxes[0] = 1;
  for (int l = 0; l < (int)sys->lv.size() && l < 32; l++) info->boxes[l] = sys->lv[l].nb;
  return IFMM_OK;
}

ifmm_status ifmm_system_get_perm(const ifmm_system* sys, long long* perm_host) {
  if (!sys || !perm_host) return IFMM_ERR_INVALID_ARG;
  std::memcpy(perm_host, sys->perm_h.data(), sizeof(long long) * sys->N);
  return IFMM_OK;
}

ifmm_status ifmm_sigma0(ifmm_ctx* ctx, ifmm_system* sys, ifmm_stream stream, double* sigma0,
                        int* iters) {
  if (!ctx || !sys || !sigma0) return IFMM_ERR_INVALID_ARG;
  if (sys->L == 0) return IFMM_ERR_UNSUPPORTED;
  return guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    if (std::isnan(sys->sigma0)) sys->sigma0 = system_sigma0(sys, st(stream), &sys->sigma0_iters);
    *sigma0 = sys->sigma0;
    if (iters) *iters = sys->sigma0_iters;
  });
}

ifmm_status ifmm_factor(ifmm_ctx* ctx, ifmm_system* sys, ifmm_stream stream,
                        ifmm_factorization** out) {
  if (!ctx || !sys || !out) return IFMM_ERR_INVALID_ARG;
  *out = nullptr;
  ifmm_status r = guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    *out = factor_create(sys, st(stream));
  });
  if (r == IFMM_OK && (*out)->info.singular_pivots > 0) {
    ctx->last_error = "a pivot block failed the singular-pivot test";
    return IFMM_ERR_SINGULAR_PIVOT;
  }
  return r;
}

void ifmm_factor_destroy(ifmm_factorization* fac) { delete fac; }

ifmm_status ifmm_factor_get_info(const ifmm_factorization* fac, ifmm_factor_info* info) {
  if (!fac || !info) return IFMM_ERR_INVALID_ARG;
  *info = fac->info;
  info->factor_bytes = (long long)fac->store.held;
  return IFMM_OK;
}

ifmm_status ifmm_factor_get_ranks(const ifmm_factorization* fac, int level, int* ranks_host,
                                  int capacity, int* count) {
  if (!fac || !count) return IFMM_ERR_INVALID_ARG;
  if (level < 0 || level >= (int)fac->rank.size()) return IFMM_ERR_INVALID_ARG;
  const auto& r = fac->rank[level];
  *count = (int)r.size();
  if (ranks_host) {
    if (capacity < (int)r.size()) return IFMM_ERR_INVALID_ARG;
    std::memcpy(ranks_host, r.data(), sizeof(int) * r.size());
  }
  return IFMM_OK;
}

ifmm_status ifmm_factor_footprint(const ifmm_factorization* fac, unsigned long long* bytes) {
  if (!fac || !bytes) return IFMM_ERR_INVALID_ARG;
  *bytes = fac->store.held + fac->plan_bytes();
  return IFMM_OK;
}

ifmm_status ifmm_solve(ifmm_ctx* ctx, const ifmm_factorization* fac, const double* b, double* x,
                       int nrhs, long long ld, ifmm_stream stream) {
  if (!ctx || !fac || !b || !x || nrhs < 0) return IFMM_ERR_INVALID_ARG;
  if (ld < fac->sys->N) return IFMM_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    factor_solve(const_cast<ifmm_factorization*>(fac), b, ld, x, ld, nrhs, st(stream));
  });
}

ifmm_status ifmm_solve_prec(ifmm_ctx* ctx, const ifmm_factorization* fac, int prec,
                            const double* b, double* x, int nrhs, long long ld,
                            ifmm_stream stream) {
  if (!ctx || !fac || !b || !x || nrhs < 0) return IFMM_ERR_INVALID_ARG;
  if (ld < fac->sys->N || (prec != IFMM_P_FP64 && prec != IFMM_P_FP32)) return IFMM_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    auto* f = const_cast<ifmm_factorization*>(fac);
    if (prec == IFMM_P_FP32) factor_solve_f32(f, b, ld, x, ld, nrhs, st(stream));
    else factor_solve(f, b, ld, x, ld, nrhs, st(stream));
  });
}

ifmm_status fmm_matvec(ifmm_ctx* ctx, const ifmm_system* sys, int mode, const double* x,
                       double* y, int nrhs, long long ld, ifmm_stream stream) {
  if (!ctx || !sys || !x || !y || nrhs < 0) return IFMM_ERR_INVALID_ARG;
  if (ld < sys->N || (mode != IFMM_MV_FMM && mode != IFMM_MV_DIRECT)) return IFMM_ERR_INVALID_ARG;
  if (x == y) return IFMM_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    system_matvec(const_cast<ifmm_system*>(sys), mode, x, ld, y, ld, nrhs, st(stream));
  });
}

ifmm_status fmm_matvec_prec(ifmm_ctx* ctx, const ifmm_system* sys, int prec, const double* x,
                            double* y, int nrhs, long long ld, ifmm_stream stream) {
  if (!ctx || !sys || !x || !y || nrhs < 0) return IFMM_ERR_INVALID_ARG;
  if (ld < sys->N || x == y) return IFMM_ERR_INVALID_ARG;
  if (prec != IFMM_P_FP64 && prec != IFMM_P_FP32) return IFMM_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    ifmm_system* sy = const_cast<ifmm_system*>(sys);
    if (prec == IFMM_P_FP32) system_matvec_f32far(sy, x, ld, y, ld, nrhs, st(stream));
    else system_matvec(sy, IFMM_MV_FMM, x, ld, y, ld, nrhs, st(stream));
  });
}

ifmm_status fmm_matvec_static(ifmm_ctx* ctx, const ifmm_system* sys, const double* x, double* y,
                              int nrhs, long long ld, ifmm_stream stream) {
  if (!ctx || !sys || !x || !y || nrhs < 0) return IFMM_ERR_INVALID_ARG;
  if (ld < sys->N || x == y) return IFMM_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    system_matvec_static(const_cast<ifmm_system*>(sys), x, y, nrhs, ld, ctx->device, st(stream));
  });
}

ifmm_status gmres_solve(ifmm_ctx* ctx, const ifmm_system* sys, const ifmm_factorization* fac,
                        int mode, const double* b, double* x, int nrhs, long long ld, double tol,
                        int maxit, ifmm_gmres_report* rep, ifmm_stream stream) {
  if (!ctx || !sys || !b || !x || !rep || nrhs < 1) return IFMM_ERR_INVALID_ARG;
  if (ld < sys->N || maxit < 1 || !(tol > 0.0)) return IFMM_ERR_INVALID_ARG;
  if (mode != IFMM_MV_FMM && mode != IFMM_MV_DIRECT) return IFMM_ERR_INVALID_ARG;
  if (fac && fac->sys != sys) return IFMM_ERR_INVALID_ARG;
  ifmm_status res = IFMM_OK;
  ifmm_status g = guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    // the caller's vectors join the bounds validation (IFMM_VALIDATE=1)
    ScopedRange rb(b, mat_bytes(sys->N, nrhs, ld)), rx(x, mat_bytes(sys->N, nrhs, ld));
    res = gmres_run(const_cast<ifmm_system*>(sys), const_cast<ifmm_factorization*>(fac), mode, b,
                    x, nrhs, ld, tol, maxit, rep, st(stream));
  });
  return g != IFMM_OK ? g : res;
}

ifmm_status gmres_solve_ex(ifmm_ctx* ctx, const ifmm_system* sys, const ifmm_factorization* fac,
                           int mode, const double* b, double* x, int nrhs, long long ld, double tol,
                           int maxit, const ifmm_gmres_options* opt, ifmm_gmres_report* rep,
                           ifmm_stream stream) {
  if (!ctx || !sys || !b || !x || !rep || nrhs < 1) return IFMM_ERR_INVALID_ARG;
  if (ld < sys->N || maxit < 1 || !(tol > 0.0)) return IFMM_ERR_INVALID_ARG;
  if (mode != IFMM_MV_FMM && mode != IFMM_MV_DIRECT) return IFMM_ERR_INVALID_ARG;
  if (fac && fac->sys != sys) return IFMM_ERR_INVALID_ARG;
  GmresOpts go;
  if (opt) {
    if (opt->side < IFMM_GMRES_RIGHT || opt->side > IFMM_GMRES_FLEXIBLE || opt->refine < 0)
      return IFMM_ERR_INVALID_ARG;
    if (opt->precond_precision != IFMM_P_FP64 && opt->precond_precision != IFMM_P_FP32)
      return IFMM_ERR_INVALID_ARG;
    if (opt->precond_precision == IFMM_P_FP32 && fac && opt->side != IFMM_GMRES_FLEXIBLE)
      return IFMM_ERR_INVALID_ARG;
    go.side = opt->side;
    go.refine = opt->refine;
    go.precond_fp32 = opt->precond_precision == IFMM_P_FP32;
    if (opt->block != 0 && opt->block != 1) return IFMM_ERR_INVALID_ARG;
    if (opt->block && fac && opt->side == IFMM_GMRES_LEFT) return IFMM_ERR_INVALID_ARG;
    go.block = opt->block;
    if (opt->matvec_precision != IFMM_P_FP64 && opt->matvec_precision != IFMM_P_FP32)
      return IFMM_ERR_INVALID_ARG;
    if (opt->matvec_precision == IFMM_P_FP32 &&
        (mode != IFMM_MV_FMM || opt->block || (fac && opt->side == IFMM_GMRES_LEFT)))
      return IFMM_ERR_INVALID_ARG;
    go.mv_fp32 = opt->matvec_precision == IFMM_P_FP32;
  }
  ifmm_status res = IFMM_OK;
  ifmm_status g = guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    ScopedRange rb(b, mat_bytes(sys->N, nrhs, ld)), rx(x, mat_bytes(sys->N, nrhs, ld));
    res = gmres_run(const_cast<ifmm_system*>(sys), const_cast<ifmm_factorization*>(fac), mode, b,
                    x, nrhs, ld, tol, maxit, rep, st(stream), nullptr, go);
  });
  return g != IFMM_OK ? g : res;
}

ifmm_status gmres_solve_host(ifmm_ctx* ctx, const ifmm_system* sys, const ifmm_factorization* fac,
                             int mode, const double* b_host, double* x_host, int nrhs, long long ld,
                             double tol, int maxit, ifmm_gmres_report* rep, ifmm_stream stream) {
  if (!ctx || !sys || !b_host || !x_host || !rep || nrhs < 1) return IFMM_ERR_INVALID_ARG;
  if (ld < sys->N) return IFMM_ERR_INVALID_ARG;
  ifmm_status res = IFMM_OK;
  ifmm_status g = guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = st(stream);
    Arena ar;
    const size_t bytes = sizeof(double) * (size_t)ld * nrhs;
    double* db = ar.alloc<double>((size_t)ld * nrhs);
    double* dx = ar.alloc<double>((size_t)ld * nrhs);
    CK(cudaMemcpyAsync(db, b_host, bytes, cudaMemcpyHostToDevice, s));
    res = gmres_solve(ctx, sys, fac, mode, db, dx, nrhs, ld, tol, maxit, rep, stream);
    if (res == IFMM_OK || res == IFMM_ERR_NOT_CONVERGED) {
      CK(cudaMemcpyAsync(x_host, dx, bytes, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
  });
  return g != IFMM_OK ? g : res;
}

ifmm_status ifmm_schur_product(ifmm_ctx* ctx, int prec, int M, int N, int K, const double* A,
                               int lda, int transA, const double* B, int ldb, int transB,
                               double* C, int ldc, double alpha, double beta, ifmm_stream stream) {
  if (!ctx || M < 0 || N < 0 || K < 0 || !C) return IFMM_ERR_INVALID_ARG;
  if (prec != IFMM_P_FP64 && prec != IFMM_P_TF32 && prec != IFMM_P_FP32 && prec != IFMM_P_BF16)
    return IFMM_ERR_INVALID_ARG;
  if (K > 0 && (!A || !B)) return IFMM_ERR_INVALID_ARG;
  if (ldc < std::max(M, 1) || lda < std::max(transA ? K : M, 1) ||
      ldb < std::max(transB ? N : K, 1))
    return IFMM_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return IFMM_OK;
  return guard(ctx, [&] {
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = st(stream);
    // the caller's matrices join the bounds validation (IFMM_VALIDATE=1)
    ScopedRange ra(A, K > 0 ? mat_bytes(transA ? K : M, transA ? M : K, lda) : 0);
    ScopedRange rb(B, K > 0 ? mat_bytes(transB ? N : K, transB ? K : N, ldb) : 0);
    ScopedRange rc(C, mat_bytes(M, N, ldc));
    Arena ar;
    int* err = ar.alloc<int>(1);
    CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    const GemmTask t{A, B, C, lda, ldb, ldc, M, N, K, transA ? 1 : 0, transB ? 1 : 0, alpha, beta};
    if (prec == IFMM_P_FP64) run_gemms(ar, {t}, s);
    else run_gemms_tc(ar, {t}, prec, err, s);
    int h = 0;
    CK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h) throw Error(IFMM_ERR_TIMEOUT, "tensor-core product: a bounded wait ran out");
  });
}

ifmm_status ifmm_profile_start(ifmm_ctx* ctx) {
  if (!ctx) return IFMM_ERR_INVALID_ARG;
  return guard(ctx, [&] { prof::start(); });
}

ifmm_status ifmm_profile_stop(ifmm_ctx* ctx, ifmm_kernel_stat* stats, int capacity, int* count) {
  if (!ctx || !count || capacity < 0) return IFMM_ERR_INVALID_ARG;
  return guard(ctx, [&] { *count = prof::stop(stats, capacity); });
}

}  // extern "C"
