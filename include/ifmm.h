/*
 * ifmm.h -- C ABI of the GB300 inverse fast multipole method (IFMM) library.
 *
 * The library factorises the H^2 (Chebyshev black-box FMM) representation
 * A_n of a dense kernel matrix a_ij = K(|r_i - r_j|) (Coulier, Pouransari,
 * Darve, "The inverse fast multipole method", Sec. 2) and uses the
 * factorisation as a right preconditioner for FP64 GMRES whose products are
 * FMM (or direct) matvecs (Sec. 3.2).
 *
 * Conventions that hold for every call:
 *  - every function returns ifmm_status; no C++ exception crosses the ABI;
 *    ifmm_last_error(ctx) gives a one-line description of the last failure;
 *  - vectors are FP64, column-major (N rows, nrhs columns, leading dimension
 *    ld >= N) in USER point order; the library permutes internally;
 *  - "device" pointers are CUDA device memory of the context's device;
 *    "host" pointers are ordinary host memory;
 *  - calls run on the caller's CUDA stream (ifmm_stream is a cudaStream_t;
 *    NULL = the legacy default stream); a call returns after its work is
 *    queued unless the description says it synchronises;
 *  - handles are opaque, owned by the caller, freed by their *_destroy;
 *    a factorisation keeps a pointer to its system: destroy it first;
 *  - invalid arguments return IFMM_ERR_INVALID_ARG and change nothing.
 */
#ifndef IFMM_H
#define IFMM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ifmm_stream; /* same type as cudaStream_t */

typedef struct ifmm_ctx ifmm_ctx;
typedef struct ifmm_system ifmm_system;
typedef struct ifmm_factorization ifmm_factorization;
typedef struct ifmm_server ifmm_server;

typedef enum {
  IFMM_OK = 0,
  IFMM_ERR_INVALID_ARG = 1,
  IFMM_ERR_OOM = 2,
  IFMM_ERR_CUDA = 3,
  IFMM_ERR_SINGULAR_PIVOT = 4, /* a pivot block E(P,P) had a pivot <= 1e-14 max|E(P,P)| */
  IFMM_ERR_NOT_CONVERGED = 5,  /* GMRES reached maxit above tol (report still filled) */
  IFMM_ERR_TIMEOUT = 6,        /* a bounded device wait ran out, or ifmm_server_wait's limit */
  IFMM_ERR_BUDGET = 7,         /* server admission refused, or a request shed              */
  IFMM_ERR_UNSUPPORTED = 8     /* e.g. a rank query on a system without a tree             */
} ifmm_status;

/* Kernel of the matrix (Sec. 3.1). */
typedef enum {
  IFMM_K_INV_R = 0,    /* 1/r                                  */
  IFMM_K_GAUSSIAN = 1, /* exp(-r^2 / (2 param^2))              */
  IFMM_K_PAPER_D = 2   /* Eq. (K_ij): r/d for r < d, d/r else  */
} ifmm_kernel_kind;

typedef struct {
  int kind;     /* ifmm_kernel_kind                                           */
  double param; /* Gaussian sigma, or d of the paper kernel; unused for 1/r    */
  double diag;  /* A_ii (also used for coincident points); NaN = K(0), which
                   the 1/r kernel does not have (then NaN is invalid)          */
} ifmm_kernel;

/* Precision of the Schur-update products S = E(R,P) E(P,P)^-1 E(P,C) of the
 * elimination (Sec. 2.2, Algorithm 2).  FP64: FP64 FMA.  TF32: operands rounded
 * to TF32 on the tcgen05 tensor cores, FP32 accumulation.  FP32: each operand
 * split into two TF32 parts, three tensor-core products (hi*hi + hi*lo + lo*hi),
 * FP32 accumulation -- close to FP32 accuracy.  BF16: operands rounded to BF16
 * (8 significant bits), FP32 accumulation; allowed only with eps >= 1e-4
 * (IFMM_ERR_INVALID_ARG otherwise).  The pivot LU, the solve for
 * E(P,P)^-1 E(P,C), every SVD and rank decision and GMRES stay in FP64. */
typedef enum { IFMM_P_FP64 = 0, IFMM_P_TF32 = 1, IFMM_P_BF16 = 2, IFMM_P_FP32 = 3 } ifmm_precision;

typedef struct {
  int dim;             /* 2 or 3                                                    */
  int cheb_n;          /* Chebyshev nodes per dimension, 1..8 (Sec. 3)             */
  int leaf_max;        /* leaf boxes hold at most this many points, >= 1           */
  double eps;          /* rank rule tolerance of Eq. (methods_SVD_rank_spectralnorm);
                          0 disables compression (exact block LU of E)             */
  int schur;           /* ifmm_precision of the Schur products                      */
  double tau_override; /* > 0: use this absolute threshold instead of eps*sigma_0   */
  int rank_cap;        /* >= 1: cap on every box rank; 0 = automatic (n^D, or no
                          cap when eps == 0)                                        */
  int fmm_n;           /* Chebyshev order of fmm_matvec; 0 = cheb_n                 */
  int rsvd_rows;       /* blocks with more rows than this (and a rank cap below
                          their height) are recompressed with the randomised SVD
                          of Sec. 2.4; 0 = 160, otherwise 1..65536                 */
  int symmetric;       /* 1: symmetric variant -- the V side of every basis SVD
                          reuses the U side's singular vectors and values (one SVD
                          per box instead of two).  Valid when A is symmetric,
                          which holds for every kernel of this library (radial,
                          U = V at the leaves); the paper's general algorithm is 0 */
} ifmm_options;

typedef enum { IFMM_MV_FMM = 0, IFMM_MV_DIRECT = 1 } ifmm_matvec_mode;

/* Side of the IFMM preconditioner in GMRES (Sec. 3.2 right, Appendix B left). */
typedef enum {
  IFMM_GMRES_RIGHT = 0,    /* A M^-1 u = b, x = M^-1 u; tol on ||b - A x|| / ||b||       */
  IFMM_GMRES_LEFT = 1,     /* M^-1 A x = M^-1 b; tol on ||M^-1 (b - A x)|| / ||M^-1 b||  */
  IFMM_GMRES_FLEXIBLE = 2  /* right, keeping z_k = M^-1 v_k and forming x = Z y: exact
                              for a preconditioner that is not one fixed linear map
                              (applied in reduced precision); twice the basis memory  */
} ifmm_gmres_side;

typedef struct {
  int side;   /* ifmm_gmres_side                                                   */
  int refine; /* right / flexible: when the recomputed true residual is above tol
                 although the Arnoldi estimate met it, restart from x at most this
                 many times (iterations count against the same maxit); >= 0     */
  int precond_precision; /* IFMM_P_FP64 (0): substitution sweeps in FP64;
                 IFMM_P_FP32: FP32 sweeps (FP32 copies of the factors, made on
                 first use), valid only with IFMM_GMRES_FLEXIBLE; products,
                 orthogonalisation and residuals stay FP64                      */
  int block;  /* 1: block GMRES -- one Krylov space shared by the nrhs columns
                 (block Arnoldi, block CGS2, Cholesky QR twice); right or
                 flexible side; maxit counts block steps; columns still above
                 tol when a block loses rank finish with per-column GMRES     */
  int matvec_precision; /* IFMM_P_FP64 (0): every product in FP64.  IFMM_P_FP32:
                 mixed-precision iterative refinement (GMRES-IR; not in the
                 paper): each cycle runs GMRES on A d = r, with the FMM's far
                 field (P2M, M2M, M2L, L2L, L2P) in FP32 and its near field in
                 FP64, until its residual estimate has fallen 1e4-fold (or
                 below tol / 2), then x += d and r = b - A x with the FP64 FMM;
                 a column converges when that true residual is <= tol.  At
                 most `refine` further cycles (one that halves no column's
                 residual ends it); IFMM_MV_FMM, right or flexible side, not
                 with block; rel_residual is the last cycle's estimate
                 relative to ||b||                                           */
} ifmm_gmres_options;

typedef struct {
  int iters;                /* Arnoldi steps taken                                   */
  double rel_residual;      /* GMRES estimate |g_{k+1}| / ||b|| (left: of the
                               preconditioned residual, / ||M^-1 b||)                */
  double true_rel_residual; /* ||b - A x|| / ||b|| recomputed with the same matvec    */
  int status;               /* IFMM_OK or IFMM_ERR_NOT_CONVERGED                      */
} ifmm_gmres_report;

typedef struct {
  long long N;
  int dim;
  int levels;         /* leaf depth L (0 = no tree: N <= leaf_max, one dense block) */
  int boxes[32];      /* non-empty boxes per depth 0..L                              */
  int max_leaf;       /* fullest leaf                                                */
  double lo[3];       /* root box corner                                             */
  double edge;        /* root box edge                                               */
} ifmm_system_info;

typedef struct {
  double sigma0;        /* sigma_0(E) (NaN when tau_override was used)               */
  int sigma0_iters;     /* power iterations                                          */
  double tau;           /* absolute truncation threshold used                        */
  int levels;           /* leaf depth L                                              */
  int top_size;         /* order of the top dense system (sum of level-2 ranks)      */
  int max_rank[32];     /* per depth 2..L: largest rank at elimination               */
  double avg_rank[32];  /* per depth: mean rank at elimination                       */
  int rank_capped;      /* number of rank decisions the cap truncated                */
  int singular_pivots;  /* pivot blocks that triggered the singular-pivot test        */
  double flops_lu, flops_trsm, flops_schur, flops_lowrank, flops_top;
  double seconds_init, seconds_sigma0, seconds_elim, seconds_top;
  long long factor_bytes; /* device bytes held by the factorisation                  */
} ifmm_factor_info;

/* One row of the launch profile: the library's own launches of one kernel. */
typedef struct {
  char name[48];
  long long launches;
  double seconds;   /* summed CUDA-event intervals around the launches        */
  double flops;     /* algorithmic flops of those launches                    */
  double bytes;     /* algorithmic bytes moved (0 where not counted)          */
} ifmm_kernel_stat;

/* ---- context ------------------------------------------------------------ */
/* Select CUDA device `device` and create a context (owns no GPU memory yet). */
ifmm_status ifmm_ctx_create(int device, ifmm_ctx** out);
void ifmm_ctx_destroy(ifmm_ctx* ctx);
const char* ifmm_last_error(const ifmm_ctx* ctx);
const char* ifmm_status_string(ifmm_status st);

/* ---- system: tree, lists, colours, raw operators (Sec. 2.1, 2.3) ------------ */
/* pts: device, N x dim row-major, user order; copied.  Builds the uniform tree
 * (first step of Algorithm 1), the neighbour / interaction lists and colour classes,
 * the Chebyshev operators and the near-field blocks.  Synchronises `stream`. */
ifmm_status ifmm_system_create(ifmm_ctx* ctx, const double* pts, long long N,
                               const ifmm_kernel* kernel, const ifmm_options* opt,
                               ifmm_stream stream, ifmm_system** out);
/* Same, with pts in host memory. */
ifmm_status ifmm_system_create_host(ifmm_ctx* ctx, const double* pts_host, long long N,
                                    const ifmm_kernel* kernel, const ifmm_options* opt,
                                    ifmm_stream stream, ifmm_system** out);
void ifmm_system_destroy(ifmm_system* sys);
ifmm_status ifmm_system_get_info(const ifmm_system* sys, ifmm_system_info* info);
/* perm_host[t] = user index of the t-th point in tree order (N entries). */
ifmm_status ifmm_system_get_perm(const ifmm_system* sys, long long* perm_host);

/* sigma_0(E), the largest singular value of the extended sparse matrix E
 * (Sec. 2.4), by power iteration on E^T E with the raw operators: start
 * vector all ones, stop at relative change <= 1e-6 or 100 iterations.
 * Synchronises `stream`; the value is cached in the system. */
ifmm_status ifmm_sigma0(ifmm_ctx* ctx, ifmm_system* sys, ifmm_stream stream, double* sigma0,
                        int* iters);

/* ---- factorisation (Algorithms 1-3) ---------------------------------------- */
/* Eliminates levels L..2 colour by colour with fill-in compression and
 * redirection, then factorises the top dense system.  Synchronises `stream`
 * (it reads back ranks between colours).  Returns IFMM_ERR_SINGULAR_PIVOT
 * (with *out still valid) if a pivot block failed the pivot test. */
ifmm_status ifmm_factor(ifmm_ctx* ctx, ifmm_system* sys, ifmm_stream stream,
                        ifmm_factorization** out);
void ifmm_factor_destroy(ifmm_factorization* fac);
ifmm_status ifmm_factor_get_info(const ifmm_factorization* fac, ifmm_factor_info* info);
/* Ranks at elimination of the boxes of depth `level` (Morton order), host array
 * of `capacity` ints; *count receives the number of boxes. */
ifmm_status ifmm_factor_get_ranks(const ifmm_factorization* fac, int level, int* ranks_host,
                                  int capacity, int* count);
/* Device bytes held by the factorisation. */
ifmm_status ifmm_factor_footprint(const ifmm_factorization* fac, unsigned long long* bytes);

/* ---- solve (substitution phase, the downward pass of Algorithm 1) ------------- */
/* x = (IFMM factorisation)^-1 b ~= A_n^-1 b.  b, x: device, N x nrhs, ld >= N;
 * b and x may alias. */
ifmm_status ifmm_solve(ifmm_ctx* ctx, const ifmm_factorization* fac, const double* b, double* x,
                       int nrhs, long long ld, ifmm_stream stream);

/* Same as ifmm_solve with the substitution sweeps in precision `prec`:
 * IFMM_P_FP64 (= ifmm_solve) or IFMM_P_FP32 (FP32 copies of the factors and
 * of the top system's inverse, built on the first FP32 call -- that call
 * allocates and synchronises `stream`; b and x stay FP64).  Other precisions
 * are IFMM_ERR_INVALID_ARG. */
ifmm_status ifmm_solve_prec(ifmm_ctx* ctx, const ifmm_factorization* fac, int prec,
                            const double* b, double* x, int nrhs, long long ld,
                            ifmm_stream stream);

/* ---- matvec (Sec. 3.2) ------------------------------------------------------- */
/* y = A_n x (IFMM_MV_FMM, Chebyshev order opt->fmm_n) or y = A x
 * (IFMM_MV_DIRECT, O(N^2)).  x, y: device, N x nrhs, ld >= N, must not alias. */
ifmm_status fmm_matvec(ifmm_ctx* ctx, const ifmm_system* sys, int mode, const double* x,
                       double* y, int nrhs, long long ld, ifmm_stream stream);

/* y = A_n x (IFMM_MV_FMM products) with prec IFMM_P_FP64 (the same as
 * fmm_matvec) or IFMM_P_FP32: the far field (P2M, M2M, M2L, L2L, L2P) from
 * FP32 copies of the operators in FP32 arithmetic, the near field in FP64,
 * y = near + far added in FP64 (the inner products of GMRES-IR).  The FP32
 * copies and plan are made on first use (allocating).  x, y as fmm_matvec. */
ifmm_status fmm_matvec_prec(ifmm_ctx* ctx, const ifmm_system* sys, int prec, const double* x,
                            double* y, int nrhs, long long ld, ifmm_stream stream);

/* ---- allocation-free matvec --------------------------------------------------- */
/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory while they run (a host application that owns
 * a fixed device pool and forbids cudaMalloc, or a real-time loop that must not
 * stall on the allocator).
 * Computes the same y = A_n x as fmm_matvec(IFMM_MV_FMM) (the direct product
 * when the system has no tree) but calls no cudaMalloc, cudaFree or other
 * allocating routine: its scratch -- the multipole / local coefficients and
 * x, y in tree order -- lives in one file-scope device array of 64 MiB that
 * every GPU loading the library holds until the process exits (the tree lists
 * it walks were copied to the device when the system was created).
 * A system and nrhs whose scratch exceeds 64 MiB are rejected with
 * IFMM_ERR_INVALID_ARG and a message naming the bytes needed.
 * The first call on a device looks up the array's address (device current);
 * make that first call before any stream capture.  Every call shares the
 * array and leaves its contents behind: calls that overlap on the GPU race.
 * x, y: device, N x nrhs, ld >= N, must not alias. */
ifmm_status fmm_matvec_static(ifmm_ctx* ctx, const ifmm_system* sys, const double* x, double* y,
                              int nrhs, long long ld, ifmm_stream stream);

/* ---- GMRES (Sec. 3.2) -------------------------------------------------------- */
/* GMRES, x_0 = 0, CGS2 Arnoldi, Givens rotations, the factorisation as right
 * preconditioner (fac may be NULL: unpreconditioned).  Each of the nrhs
 * columns is an independent solve.  A column stops when the Arnoldi residual
 * estimate is <= tol ||b||; the true residual ||b - A x|| is then recomputed
 * with the same matvec, and if rounding left it above tol ||b|| GMRES
 * restarts from x (at most twice, within the same maxit).  rep: host array of
 * nrhs reports.  Synchronises `stream` (reads the residual estimate every
 * step).  Returns IFMM_ERR_NOT_CONVERGED if any column ends above tol. */
ifmm_status gmres_solve(ifmm_ctx* ctx, const ifmm_system* sys, const ifmm_factorization* fac,
                        int mode, const double* b, double* x, int nrhs, long long ld, double tol,
                        int maxit, ifmm_gmres_report* rep, ifmm_stream stream);
/* GMRES with the preconditioner on either side (Sec. 3.2, Appendix B) or in
 * flexible form; opt NULL = right preconditioning with refine = 2, which is
 * what gmres_solve does.  Right / flexible: a column converges when its
 * recomputed true residual is <= tol.  Left: when the preconditioned residual
 * estimate is <= tol (the paper's left-preconditioned criterion);
 * true_rel_residual still reports ||b - A x|| / ||b||.  fac == NULL ignores
 * the side (plain GMRES).  Synchronises `stream`. */
ifmm_status gmres_solve_ex(ifmm_ctx* ctx, const ifmm_system* sys, const ifmm_factorization* fac,
                           int mode, const double* b, double* x, int nrhs, long long ld, double tol,
                           int maxit, const ifmm_gmres_options* opt, ifmm_gmres_report* rep,
                           ifmm_stream stream);
/* Same with b, x in host memory (copied to and from the device inside). */
ifmm_status gmres_solve_host(ifmm_ctx* ctx, const ifmm_system* sys,
                             const ifmm_factorization* fac, int mode, const double* b_host,
                             double* x_host, int nrhs, long long ld, double tol, int maxit,
                             ifmm_gmres_report* rep, ifmm_stream stream);

/* ---- many systems: batched factorisation (the paper factorises one system at a
 * time, Algorithm 1; independent systems share nothing) ------------------------ */
/* Factorises sys[0..count-1] (distinct systems; a repeated handle is
 * IFMM_ERR_INVALID_ARG) concurrently: up to 8 worker
 * threads, each on its own CUDA stream that first waits for the work queued on
 * `stream`, take the systems largest first.  out: host array of count
 * handles, filled in (each freed by ifmm_factor_destroy).  On any error other
 * than IFMM_ERR_SINGULAR_PIVOT every out[k] is NULL; with a singular pivot the
 * handles stay valid, as for ifmm_factor.  Returns after all factorisations
 * are complete. */
ifmm_status ifmm_factor_batch(ifmm_ctx* ctx, ifmm_system* const* sys, int count,
                              ifmm_stream stream, ifmm_factorization** out);

/* ---- serving: continuous batching of GMRES solves (Sec. 3.2 per request) ---- */
/* A server owns `workers` threads (0 = 4), each with its own stream.  A worker
 * takes the registered system whose oldest queued request has waited longest
 * and that no other worker is serving, gathers all of that system's queued
 * requests (at most 32 columns) into one block of right-hand sides, runs GMRES
 * (FMM matvec, the factorisation as preconditioner, true residual <= tol in
 * FP64) on the block -- every column converges on its own -- and returns each
 * request's columns.  Requests that arrive while their system is busy join its
 * next block; other systems are served at the same time by the other workers.
 * Device memory is admitted against hbm_budget twice: a system's resident
 * data at ifmm_server_register, and each block's GMRES memory when the block
 * starts (a block that does not fit waits for running blocks to finish; one
 * that can never fit completes with IFMM_ERR_BUDGET).  ifmm_server_create
 * sweeps the preconditioner in FP32 (flexible GMRES); ifmm_server_create_ex
 * takes precond_precision IFMM_P_FP64 (right-preconditioned GMRES, FP64
 * sweeps) or IFMM_P_FP32.  Destroy a server only after every ifmm_server_wait
 * has returned. */
ifmm_status ifmm_server_create(ifmm_ctx* ctx, unsigned long long hbm_budget, int workers,
                               ifmm_server** out);
ifmm_status ifmm_server_create_ex(ifmm_ctx* ctx, unsigned long long hbm_budget, int workers,
                                  int precond_precision, ifmm_server** out);
void ifmm_server_destroy(ifmm_server* srv);
/* Keeps `bytes` of the budget out of later registrations, for the GMRES
 * memory of blocks (default 0; at most the budget). */
ifmm_status ifmm_server_set_reserve(ifmm_server* srv, unsigned long long bytes);
/* Products of the served GMRES: IFMM_P_FP64 (every product in FP64, the
 * default) or IFMM_P_FP32 (iterative refinement, see
 * ifmm_gmres_options.matvec_precision; at most 10 refinement cycles).  With
 * IFMM_P_FP32 each registration also makes and admits the system's FP32
 * far-field operators and a 32-column plan.  Call before the first
 * ifmm_server_register (IFMM_ERR_INVALID_ARG afterwards). */
ifmm_status ifmm_server_set_matvec_precision(ifmm_server* srv, int prec);
/* Admits (sys, fac) if its resident device memory -- operators,
 * factorisation, solve plans and (FP32 server) the FP32 copies of the
 * factors, which this call builds -- fits what is left of hbm_budget less
 * the reserve; IFMM_ERR_BUDGET otherwise (nothing is registered).  maxit: the largest
 * maxit its requests will use.  A system or factorisation registered twice is
 * IFMM_ERR_INVALID_ARG.  The server does not own sys or fac; they must outlive it.
 * *id: the handle for ifmm_server_submit. */
ifmm_status ifmm_server_register(ifmm_server* srv, ifmm_system* sys, ifmm_factorization* fac,
                                 int maxit, int* id);
/* Queues a solve of A_n x = b for system `id`: b_host, x_host in host memory,
 * N x nrhs column-major (ld N), 1 <= nrhs <= 32; both must stay valid until
 * the ticket is waited for.  Residual target tol (a block uses the smallest
 * tol and the largest maxit of its requests).  Load shedding: if the system
 * already has a full block (32 columns) queued behind the one in flight, the
 * request is refused with IFMM_ERR_BUDGET (and counted as shed); this bounds
 * the queueing delay to about one block's solve time. */
ifmm_status ifmm_server_submit(ifmm_server* srv, int id, const double* b_host, double* x_host,
                               int nrhs, double tol, int maxit, long long* ticket);
/* Same as ifmm_server_submit with b and x in device memory of the context's
 * device (N x nrhs, ld N); both must stay valid until the ticket is waited for. */
ifmm_status ifmm_server_submit_device(ifmm_server* srv, int id, const double* b, double* x,
                                      int nrhs, double tol, int maxit, long long* ticket);
/* Waits up to timeout_ms (< 0: no limit) for a ticket; IFMM_ERR_TIMEOUT if it
 * is not done yet (the ticket stays valid).  On completion fills rep (nrhs
 * entries, host), *latency_s (submit to completion, seconds; may be NULL),
 * releases the ticket and returns the request's status. */
ifmm_status ifmm_server_wait(ifmm_server* srv, long long ticket, int timeout_ms,
                             ifmm_gmres_report* rep, double* latency_s);
/* Device bytes admitted, GMRES blocks run, columns solved and requests shed
 * so far (any pointer may be NULL). */
ifmm_status ifmm_server_stats(ifmm_server* srv, unsigned long long* used_bytes,
                              long long* batches, long long* columns, long long* shed);
const char* ifmm_server_last_error(ifmm_server* srv);

/* ---- Schur product kernel ----------------------------------------------------- */
/* C = alpha op(A) op(B) + beta C with the kernel the elimination uses for its
 * Schur products at precision `prec` (ifmm_precision) --
 * the trailing update of Sec. 2.2, exposed so that a caller can check or time
 * it on its own matrices (prec: FP64, TF32, FP32 or BF16).  A, B, C: device,
 * FP64, column-major; op(A) is M x K
 * (A is M x K with lda >= M, or K x M with lda >= K when transA), op(B) is
 * K x N likewise, C is M x N with ldc >= M and must not overlap A or B.
 * beta == 0 does not read C.  IFMM_ERR_TIMEOUT if a tensor-core wait ran out
 * (the result is then undefined); synchronises `stream`. */
ifmm_status ifmm_schur_product(ifmm_ctx* ctx, int prec, int M, int N, int K, const double* A,
                               int lda, int transA, const double* B, int ldb, int transB,
                               double* C, int ldc, double alpha, double beta, ifmm_stream stream);

/* ---- launch profile ------------------------------------------------------ */
/* Start recording an event pair around each of the library's launches (on
 * the launching stream); resets the totals.  Process-wide. */
ifmm_status ifmm_profile_start(ifmm_ctx* ctx);
/* Synchronise the device, stop recording and return per-kernel totals in
 * stats (host array of `capacity`); *count receives the number of kernels. */
ifmm_status ifmm_profile_stop(ifmm_ctx* ctx, ifmm_kernel_stat* stats, int capacity, int* count);

/* Kernel launches the library has made in this process so far (graph replays
 * count every kernel node of the graph). */
ifmm_status ifmm_launch_count(unsigned long long* launches);

/* Measured peak arithmetic rates of the context's device (TFLOP/s): FP64 and
 * FP32 FMA chains over every SM, timed with CUDA events (~0.1 s).  The
 * roofline denominators of the library's FP64- and FP32-bound kernels. */
ifmm_status ifmm_measure_peaks(ifmm_ctx* ctx, double* fp64_tflops, double* fp32_tflops);

#ifdef __cplusplus
}
#endif
#endif /* IFMM_H */
