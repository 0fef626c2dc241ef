// batch.cu -- many independent systems on one GPU: batched factorisation and
// a continuous-batching GMRES server.
//
// The paper factorises and solves one system at a time (Algorithm 1, Sec. 3.2);
// independent systems share nothing, so on one GPU their work can overlap.
//
// ifmm_factor_batch: worker threads, each with its own CUDA stream, take the
// systems largest first and factorise them (the colour-batched elimination of
// factor.cu); the launches of different systems run concurrently on the GPU,
// filling the SMs that one system's small colour classes leave idle.
//
// Server: requests (one system, nrhs right-hand sides in host or device
// memory, a tolerance) are queued per registered system.  Worker threads,
// each with its own stream, repeatedly take the system whose oldest request
// has waited longest and that no other worker is serving, gather ALL of that
// system's queued requests (up to a column cap) into one block of right-hand
// sides and run GMRES on the block (each column converges independently,
// Sec. 3.2) -- by default flexible GMRES with the substitution sweeps in FP32
// and products, orthogonalisation and residuals in FP64 -- then return every
// request's columns.  Requests that arrive while their system is busy join
// its next block; other systems proceed in parallel on the other workers.
// Device memory is admitted twice against the budget: a system's resident
// data (operators, factorisation, FP32 copies, plans) at registration, and
// each block's GMRES memory when the block starts; a block that does not fit
// waits until running blocks finish (idle workers hand back their memory).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "factor.cuh"

namespace ifmm {

using SteadyClock = std::chrono::steady_clock;

// ---------------------------------------------------------------------------
// batched factorisation
// ---------------------------------------------------------------------------
ifmm_status factor_batch(int device, ifmm_system* const* sys, int count, cudaStream_t s,
                         ifmm_factorization** out, std::string& err) {
  for (int k = 0; k < count; k++) out[k] = nullptr;
  if (count == 0) return IFMM_OK;
  // inputs produced on the caller's stream must be complete before the workers start
  cudaEvent_t ready;
  CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  CK(cudaEventRecord(ready, s));
  std::vector<int> order(count);
  for (int k = 0; k < count; k++) order[k] = k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return sys[a]->N > sys[b]->N; });
  const int nw = std::min(count, 8);
  std::atomic<int> next{0};
  std::mutex mu;
  ifmm_status first = IFMM_OK;
  auto worker = [&]() {
    cudaStream_t ws = nullptr;
    try {
      CK(cudaSetDevice(device));
      CK(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
      CK(cudaStreamWaitEvent(ws, ready, 0));
      for (;;) {
        const int q = next.fetch_add(1);
        if (q >= count) break;
        const int k = order[q];
        out[k] = factor_create(sys[k], ws);
      }
    } catch (const Error& e) {
      std::lock_guard<std::mutex> g(mu);
      if (first == IFMM_OK) { first = e.st; err = e.what(); }
    } catch (const std::exception& e) {
      std::lock_guard<std::mutex> g(mu);
      if (first == IFMM_OK) { first = IFMM_ERR_CUDA; err = e.what(); }
    }
    if (ws) cudaStreamDestroy(ws);
  };
  std::vector<std::thread> th;
  for (int w = 0; w < nw; w++) th.emplace_back(worker);
  for (auto& t : th) t.join();
  cudaEventDestroy(ready);
  if (first != IFMM_OK) return first;
  for (int k = 0; k < count; k++)
    if (out[k] && out[k]->info.singular_pivots > 0) {
      err = "a pivot block failed the singular-pivot test";
      return IFMM_ERR_SINGULAR_PIVOT;
    }
  return IFMM_OK;
}

}  // namespace ifmm

// ---------------------------------------------------------------------------
// server
// ---------------------------------------------------------------------------
struct ifmm_server {
  struct Request {
    int id = 0, nrhs = 0;
    const double* b = nullptr;  // N x nrhs, ld N: host, or device when `device`
    double* x = nullptr;
    bool device = false;
    double tol = 1e-10;
    int maxit = 500;
    ifmm::SteadyClock::time_point t_submit, t_done;
    bool done = false;
    ifmm_status status = IFMM_OK;
    std::vector<ifmm_gmres_report> rep;
  };
  struct Entry {
    ifmm_system* sys = nullptr;
    ifmm_factorization* fac = nullptr;
    size_t bytes = 0;
    bool busy = false;
    std::deque<long long> queue;  // tickets in arrival order
  };
  ifmm_ctx* ctx = nullptr;
  int device = 0;
  int precond_fp32 = 1;  // flexible GMRES with FP32 substitution sweeps
  int mv_fp32 = 0;       // iterative refinement with the FMM far field in FP32
  bool any_registered = false;
  size_t budget = 0, used = 0;  // used: resident systems (operators, factors, plans)
  size_t reserve = 0;           // kept from registrations for the GMRES blocks
  int col_cap = 32;
  int queue_cap = 32;  // queued columns per system (one block) beyond which requests are shed
  long long shed = 0, refused = 0;
  std::deque<Entry> systems;  // stable references while workers hold one
  std::map<long long, std::unique_ptr<Request>> reqs;
  long long next_ticket = 1;
  long long batches = 0, batched_columns = 0;
  // GMRES working memory of the blocks: reserved per worker (what its arena
  // holds, or what its running block may grow it to), admitted block by block
  std::vector<size_t> ws_res;
  size_t ws_total = 0;
  int running = 0, mem_waiters = 0;
  bool release_req = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::vector<std::thread> workers;
  std::string last_error;

  // device bytes a block of `width` columns is admitted with: the Krylov basis
  // (and the preconditioned basis of flexible GMRES) in chunks of 16 vectors
  // up to the first 64 vectors, four work vectors, the block's b and x.  A
  // block that iterates further grows its workspace by a chunk at a time.
  size_t block_bytes(long long N, int width, int maxit) const {
    const long long vecs = std::min<long long>(((maxit + 16) / 16) * 16, 64);
    const long long nb = precond_fp32 ? 2 : 1;
    return sizeof(double) * (size_t)N * width * (size_t)(nb * vecs + 6);
  }

  void finish(std::vector<Request*>& batch, ifmm_status st, const std::string& msg,
              const std::vector<ifmm_gmres_report>& reps, int cols) {
    // caller holds the lock
    const auto now = ifmm::SteadyClock::now();
    long long off = 0;
    for (Request* r : batch) {
      r->rep.assign(reps.begin() + off, reps.begin() + off + r->nrhs);
      off += r->nrhs;
      r->status = st;
      if (st == IFMM_OK)
        for (auto& q : r->rep)
          if (q.status != IFMM_OK) r->status = (ifmm_status)q.status;
      r->t_done = now;
      r->done = true;
    }
    if (!msg.empty()) last_error = msg;
    batches++;
    batched_columns += cols;
  }

  void work(int w) {
    using namespace ifmm;
    cudaStream_t ws = nullptr;
    Arena buf;
    Arena gws;  // GMRES workspace, reused block after block
    gws.chunk_bytes = size_t(256) << 20;
    size_t buf_cols = 0;
    long long buf_n = 0;
    double *db = nullptr, *dx = nullptr;
    try {
      CK(cudaSetDevice(device));
      CK(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
    } catch (const std::exception& e) {
      std::lock_guard<std::mutex> g(mu);
      last_error = e.what();
      return;
    }
    auto held = [&] { return gws.held + buf.held; };
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
      if (release_req && held() > 0) {  // another block waits for memory this idle worker holds
        lk.unlock();
        gws.release();
        buf.release();
        buf_cols = 0;
        buf_n = 0;
        lk.lock();
        ws_total -= ws_res[w];
        ws_res[w] = 0;
        cv_done.notify_all();
      }
      // the idle system whose oldest request has waited longest
      int pick = -1;
      SteadyClock::time_point best{};
      for (int i = 0; i < (int)systems.size(); i++) {
        Entry& E = systems[i];
        if (E.busy || E.queue.empty()) continue;
        const auto t = reqs[E.queue.front()]->t_submit;
        if (pick < 0 || t < best) { pick = i; best = t; }
      }
      if (pick < 0) {
        cv_work.wait(lk);
        continue;
      }
      Entry& E = systems[pick];
      E.busy = true;
      std::vector<Request*> batch;
      int cols = 0, maxit = 1;
      double tol = 1.0;
      while (!E.queue.empty()) {
        Request* r = reqs[E.queue.front()].get();
        if (!batch.empty() && cols + r->nrhs > col_cap) break;
        batch.push_back(r);
        cols += r->nrhs;
        tol = std::min(tol, r->tol);
        maxit = std::max(maxit, r->maxit);
        E.queue.pop_front();
      }
      // pad to a power of two so that the solve and matvec plans of a few
      // widths are reused; padding columns are zero and never iterate
      int width = 1;
      while (width < cols) width <<= 1;
      const long long N = E.sys->N;
      // admission of the block's working memory: wait while running blocks
      // (or idle workers' arenas) hold what it needs
      const size_t need = std::max(block_bytes(N, width, maxit), held());
      bool fits = false;
      for (;;) {
        if (used + ws_total - ws_res[w] + need <= budget) { fits = true; break; }
        bool idle_memory = false;
        for (int v = 0; v < (int)ws_res.size(); v++) idle_memory |= v != w && ws_res[v] > 0;
        if (running == 0 && !idle_memory) break;  // can never fit
        release_req = idle_memory;
        mem_waiters++;
        cv_work.notify_all();
        cv_done.wait(lk);
        mem_waiters--;
        if (mem_waiters == 0) release_req = false;
        if (stop) break;
      }
      if (!fits) {
        refused += (long long)batch.size();
        std::vector<ifmm_gmres_report> none(cols);
        for (auto& q : none) q = {0, 0.0, 0.0, IFMM_ERR_BUDGET};
        finish(batch, IFMM_ERR_BUDGET,
               "a block of " + std::to_string(width) + " columns needs " + std::to_string(need) +
                   " bytes of GMRES memory beyond what the budget leaves",
               none, cols);
        E.busy = false;
        cv_done.notify_all();
        cv_work.notify_all();
        continue;
      }
      ws_total += need - ws_res[w];
      ws_res[w] = need;
      running++;
      lk.unlock();
      ifmm_status st = IFMM_OK;
      std::string msg;
      std::vector<ifmm_gmres_report> reps(width);
      try {
        if ((size_t)width > buf_cols || N > buf_n) {
          buf.release();
          buf_cols = std::max<size_t>(buf_cols, width);
          buf_n = std::max(buf_n, N);
          db = buf.alloc<double>((size_t)buf_n * buf_cols);
          dx = buf.alloc<double>((size_t)buf_n * buf_cols);
        }
        CK(cudaMemsetAsync(db, 0, sizeof(double) * N * width, ws));
        long long off = 0;
        for (Request* r : batch) {
          CK(cudaMemcpyAsync(db + off * N, r->b, sizeof(double) * N * r->nrhs,
                             r->device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ws));
          off += r->nrhs;
        }
        GmresOpts go;
        if (precond_fp32) {
          go.side = IFMM_GMRES_FLEXIBLE;
          go.precond_fp32 = 1;
        }
        if (mv_fp32) {
          go.mv_fp32 = 1;
          go.refine = 10;
        }
        gmres_run(E.sys, E.fac, IFMM_MV_FMM, db, dx, width, N, tol, maxit, reps.data(), ws, &gws,
                  go);
        off = 0;
        for (Request* r : batch) {
          CK(cudaMemcpyAsync(r->x, dx + off * N, sizeof(double) * N * r->nrhs,
                             r->device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ws));
          off += r->nrhs;
        }
        CK(cudaStreamSynchronize(ws));
      } catch (const Error& e) {
        st = e.st;
        msg = e.what();
      } catch (const std::exception& e) {
        st = IFMM_ERR_CUDA;
        msg = e.what();
      }
      lk.lock();
      running--;
      const size_t h = held();  // what the arena keeps after the block
      ws_total -= ws_res[w];
      ws_res[w] = h;
      ws_total += h;
      finish(batch, st, msg, reps, cols);
      E.busy = false;
      cv_done.notify_all();
      cv_work.notify_all();
    }
    lk.unlock();
    buf.release();
    gws.release();
    if (ws) cudaStreamDestroy(ws);
  }
};

extern "C" {

ifmm_status ifmm_factor_batch(ifmm_ctx* ctx, ifmm_system* const* sys, int count,
                              ifmm_stream stream, ifmm_factorization** out) {
  if (!ctx || count < 0 || (count > 0 && (!sys || !out))) return IFMM_ERR_INVALID_ARG;
  for (int k = 0; k < count; k++) {
    if (!sys[k]) return IFMM_ERR_INVALID_ARG;
    for (int q = 0; q < k; q++)  // one worker per system: a system may appear once
      if (sys[q] == sys[k]) return IFMM_ERR_INVALID_ARG;
  }
  std::string err;
  ifmm_status st = IFMM_OK;
  try {
    CK(cudaSetDevice(ctx->device));
    st = ifmm::factor_batch(ctx->device, sys, count, reinterpret_cast<cudaStream_t>(stream), out,
                            err);
  } catch (const std::exception& e) {
    st = IFMM_ERR_CUDA;
    err = e.what();
  }
  if (st != IFMM_OK) {
    ctx->last_error = err;
    if (st != IFMM_ERR_SINGULAR_PIVOT)
      for (int k = 0; k < count; k++) {
        delete out[k];
        out[k] = nullptr;
      }
  }
  return st;
}

ifmm_status ifmm_server_create_ex(ifmm_ctx* ctx, unsigned long long hbm_budget, int workers,
                                  int precond_precision, ifmm_server** out) {
  if (!ctx || !out || workers < 0 || workers > 64) return IFMM_ERR_INVALID_ARG;
  if (precond_precision != IFMM_P_FP64 && precond_precision != IFMM_P_FP32)
    return IFMM_ERR_INVALID_ARG;
  auto* s = new ifmm_server();
  s->ctx = ctx;
  s->device = ctx->device;
  s->budget = hbm_budget;
  s->precond_fp32 = precond_precision == IFMM_P_FP32;
  const int nw = workers > 0 ? workers : 4;
  s->ws_res.assign(nw, 0);
  for (int w = 0; w < nw; w++) s->workers.emplace_back([s, w] { s->work(w); });
  *out = s;
  return IFMM_OK;
}

ifmm_status ifmm_server_set_matvec_precision(ifmm_server* s, int prec) {
  if (!s || (prec != IFMM_P_FP64 && prec != IFMM_P_FP32)) return IFMM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  if (s->any_registered) {
    s->last_error = "the matvec precision is set before the first registration";
    return IFMM_ERR_INVALID_ARG;
  }
  s->mv_fp32 = prec == IFMM_P_FP32;
  return IFMM_OK;
}

ifmm_status ifmm_server_create(ifmm_ctx* ctx, unsigned long long hbm_budget, int workers,
                               ifmm_server** out) {
  return ifmm_server_create_ex(ctx, hbm_budget, workers, IFMM_P_FP32, out);
}

void ifmm_server_destroy(ifmm_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
}

ifmm_status ifmm_server_register(ifmm_server* s, ifmm_system* sys, ifmm_factorization* fac,
                                 int maxit, int* id) {
  if (!s || !sys || !fac || !id || fac->sys != sys || maxit < 1) return IFMM_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> g(s->mu);
    for (const auto& e : s->systems)
      if (e.sys == sys || e.fac == fac) {  // a system is served by one worker at a time
        s->last_error = "this system or factorisation is already registered";
        return IFMM_ERR_INVALID_ARG;
      }
  }
  // resident device memory: operators, factorisation, its FP32 copies (built
  // here when the server sweeps in FP32), solve plans, and the FMM plans and
  // workspace for a full block (FP64, and the FP32 far field with iterative
  // refinement), built here; the GMRES memory of a block is admitted when the
  // block starts
  size_t bytes = sys->mem.held + fac->store.held + fac->plan_bytes();
  if (s->precond_fp32 && !fac->f32.ready) {
    size_t est = 0;
    for (const auto& R : fac->recs)
      est += sizeof(float) * ((size_t)R.p * R.a + 2 * (size_t)R.nC * R.a);
    const long long n = sys->L == 0 ? sys->N : fac->top_n;
    est += sizeof(float) * (size_t)n * n;
    bytes += est;
  }
  if (s->precond_fp32) {  // the FP32 sweep plan for col_cap columns, if not built yet
    size_t per_col = (size_t)sys->N;
    for (int l = 2; l < (int)fac->yoff.size(); l++)
      if (!fac->yoff[l].empty()) per_col += (size_t)fac->yoff[l].back();
    for (const auto& R : fac->recs) per_col += (size_t)std::max(R.p, 1);
    if (!fac->plans32.count(s->col_cap))  // one plan serves every width up to col_cap
      bytes += sizeof(float) * per_col * s->col_cap + (size_t(8) << 20);
  }
  {
    size_t fmm = ifmm::system_fmm_bytes(sys, s->col_cap);
    if (s->mv_fp32) fmm += ifmm::system_f32far_bytes(sys, s->col_cap);
    bytes += std::max(fmm, ifmm::system_fmm_held(sys));
  }
  std::lock_guard<std::mutex> g(s->mu);
  const size_t avail = s->budget > s->reserve ? s->budget - s->reserve : 0;
  if (s->used + bytes > avail) {
    s->last_error = "admission refused: the system needs " + std::to_string(bytes) +
                    " bytes of device memory, " +
                    std::to_string(avail > s->used ? avail - s->used : 0) +
                    " remain for resident systems";
    return IFMM_ERR_BUDGET;
  }
  {
    cudaStream_t st = nullptr;
    try {
      CK(cudaSetDevice(s->device));
      CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      if (s->precond_fp32) {
        // the FP32 copies, and the sweep plan that serves every block width
        ifmm::factor_prepare_f32(fac, st);
        ifmm::factor_prepare_plans_f32(fac, s->col_cap, st);
      }
      ifmm::system_prepare_fmm(sys, s->col_cap, st);
      if (s->mv_fp32) ifmm::system_prepare_f32far(sys, s->col_cap, st);
      CK(cudaStreamSynchronize(st));
      cudaStreamDestroy(st);
    } catch (const std::exception& e) {
      if (st) cudaStreamDestroy(st);
      s->last_error = e.what();
      return IFMM_ERR_CUDA;
    }
  }
  // what the system now holds (the estimate above bounded the admission)
  bytes = std::max(bytes, sys->mem.held + fac->store.held + fac->plan_bytes() +
                              ifmm::system_fmm_held(sys));
  s->any_registered = true;
  s->used += bytes;
  ifmm_server::Entry e;
  e.sys = sys;
  e.fac = fac;
  e.bytes = bytes;
  s->systems.push_back(std::move(e));
  *id = (int)s->systems.size() - 1;
  return IFMM_OK;
}

static ifmm_status server_submit(ifmm_server* s, int id, const double* b, double* x, bool device,
                                 int nrhs, double tol, int maxit, long long* ticket) {
  if (!s || !b || !x || !ticket || nrhs < 1 || !(tol > 0.0) || maxit < 1)
    return IFMM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  if (id < 0 || id >= (int)s->systems.size()) return IFMM_ERR_INVALID_ARG;
  if (nrhs > s->col_cap) {
    s->last_error = "a request may carry at most " + std::to_string(s->col_cap) + " columns";
    return IFMM_ERR_INVALID_ARG;
  }
  ifmm_server::Entry& E = s->systems[id];
  int queued = 0;
  for (long long q : E.queue) queued += s->reqs[q]->nrhs;
  if (queued + nrhs > s->queue_cap) {
    s->shed++;
    s->last_error = "request shed: its system already has " + std::to_string(queued) +
                    " columns queued (limit " + std::to_string(s->queue_cap) + ")";
    return IFMM_ERR_BUDGET;
  }
  auto r = std::make_unique<ifmm_server::Request>();
  r->id = id;
  r->nrhs = nrhs;
  r->b = b;
  r->x = x;
  r->device = device;
  r->tol = tol;
  r->maxit = maxit;
  r->t_submit = ifmm::SteadyClock::now();
  const long long t = s->next_ticket++;
  s->reqs[t] = std::move(r);
  s->systems[id].queue.push_back(t);
  *ticket = t;
  s->cv_work.notify_one();
  return IFMM_OK;
}

ifmm_status ifmm_server_submit(ifmm_server* s, int id, const double* b_host, double* x_host,
                               int nrhs, double tol, int maxit, long long* ticket) {
  return server_submit(s, id, b_host, x_host, false, nrhs, tol, maxit, ticket);
}

ifmm_status ifmm_server_submit_device(ifmm_server* s, int id, const double* b, double* x,
                                      int nrhs, double tol, int maxit, long long* ticket) {
  return server_submit(s, id, b, x, true, nrhs, tol, maxit, ticket);
}

ifmm_status ifmm_server_wait(ifmm_server* s, long long ticket, int timeout_ms,
                             ifmm_gmres_report* rep, double* latency_s) {
  if (!s) return IFMM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return IFMM_ERR_INVALID_ARG;
  ifmm_server::Request* r = it->second.get();
  auto ready = [&] { return r->done; };
  if (timeout_ms < 0) s->cv_done.wait(lk, ready);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return IFMM_ERR_TIMEOUT;
  if (rep) std::copy(r->rep.begin(), r->rep.end(), rep);
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  const ifmm_status st = r->status;
  s->reqs.erase(it);
  return st;
}

ifmm_status ifmm_server_set_reserve(ifmm_server* s, unsigned long long bytes) {
  if (!s) return IFMM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  if (bytes > s->budget) return IFMM_ERR_INVALID_ARG;
  s->reserve = bytes;
  return IFMM_OK;
}

ifmm_status ifmm_server_stats(ifmm_server* s, unsigned long long* used_bytes, long long* batches,
                              long long* columns, long long* shed) {
  if (!s) return IFMM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  if (shed) *shed = s->shed;
  if (used_bytes) *used_bytes = s->used;
  if (batches) *batches = s->batches;
  if (columns) *columns = s->batched_columns;
  return IFMM_OK;
}

const char* ifmm_server_last_error(ifmm_server* s) {
  if (!s) return "";
  std::lock_guard<std::mutex> g(s->mu);
  thread_local std::string copy;
  copy = s->last_error;
  return copy.c_str();
}

}  // extern "C"
