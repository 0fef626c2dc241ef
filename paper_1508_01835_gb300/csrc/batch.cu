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
// Server: requests (one system, nrhs right-hand sides in host memory, a
// tolerance) are queued per registered system.  Worker threads, each with its
// own stream, repeatedly take the system whose oldest request has waited
// longest and that no other worker is serving, gather ALL of that system's
// queued requests (up to a column cap) into one block of right-hand sides and
// run FP64 GMRES on the block (each column converges independently, Sec. 3.2),
// then return every request's columns.  Requests that arrive while their
// system is busy join its next block; other systems proceed in parallel on
// the other workers.  Registration admits a system only if the device memory
// of its factorisation, operators and GMRES workspace fits the budget.
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
    const double* b = nullptr;  // host, N x nrhs, ld N
    double* x = nullptr;        // host, N x nrhs, ld N
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
  size_t budget = 0, used = 0;
  int col_cap = 32;
  int queue_cap = 32;  // queued columns per system (one block) beyond which requests are shed
  long long shed = 0;
  std::deque<Entry> systems;  // stable references while workers hold one
  std::map<long long, std::unique_ptr<Request>> reqs;
  long long next_ticket = 1;
  long long batches = 0, batched_columns = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::vector<std::thread> workers;
  std::string last_error;

  void work() {
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
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
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
      int cols = 0;
      while (!E.queue.empty()) {
        Request* r = reqs[E.queue.front()].get();
        if (!batch.empty() && cols + r->nrhs > col_cap) break;
        batch.push_back(r);
        cols += r->nrhs;
        E.queue.pop_front();
      }
      lk.unlock();
      // pad to a power of two so that the solve and matvec plans of a few
      // widths are reused; padding columns are zero and never iterate
      int width = 1;
      while (width < cols) width <<= 1;
      const long long N = E.sys->N;
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
        double tol = 1.0;
        int maxit = 1;
        long long off = 0;
        for (Request* r : batch) {
          CK(cudaMemcpyAsync(db + off * N, r->b, sizeof(double) * N * r->nrhs,
                             cudaMemcpyHostToDevice, ws));
          off += r->nrhs;
          tol = std::min(tol, r->tol);
          maxit = std::max(maxit, r->maxit);
        }
        gmres_run(E.sys, E.fac, IFMM_MV_FMM, db, dx, width, N, tol, maxit, reps.data(), ws, &gws);
        off = 0;
        for (Request* r : batch) {
          CK(cudaMemcpyAsync(r->x, dx + off * N, sizeof(double) * N * r->nrhs,
                             cudaMemcpyDeviceToHost, ws));
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
      const auto now = SteadyClock::now();
      lk.lock();
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

ifmm_status ifmm_server_create(ifmm_ctx* ctx, unsigned long long hbm_budget, int workers,
                               ifmm_server** out) {
  if (!ctx || !out || workers < 0 || workers > 64) return IFMM_ERR_INVALID_ARG;
  auto* s = new ifmm_server();
  s->ctx = ctx;
  s->device = ctx->device;
  s->budget = hbm_budget;
  const int nw = workers > 0 ? workers : 4;
  for (int w = 0; w < nw; w++) s->workers.emplace_back([s] { s->work(); });
  *out = s;
  return IFMM_OK;
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
  // device memory: operators + factorisation + GMRES workspace of one block of
  // col_cap columns (Krylov basis of maxit + 1 vectors, solve and matvec plans)
  const size_t cols = (size_t)s->col_cap;
  const size_t gm = sizeof(double) * (size_t)sys->N * cols * ((size_t)maxit + 8);
  const size_t bytes = sys->mem.held + fac->store.held + fac->plan_bytes() + gm;
  std::lock_guard<std::mutex> g(s->mu);
  for (const auto& e : s->systems)
    if (e.sys == sys || e.fac == fac) {  // a system is served by one worker at a time
      s->last_error = "this system or factorisation is already registered";
      return IFMM_ERR_INVALID_ARG;
    }
  if (s->used + bytes > s->budget) {
    s->last_error = "admission refused: the system needs " + std::to_string(bytes) +
                    " bytes of device memory, " + std::to_string(s->budget - s->used) +
                    " remain in the budget";
    return IFMM_ERR_BUDGET;
  }
  s->used += bytes;
  ifmm_server::Entry e;
  e.sys = sys;
  e.fac = fac;
  e.bytes = bytes;
  s->systems.push_back(std::move(e));
  *id = (int)s->systems.size() - 1;
  return IFMM_OK;
}

ifmm_status ifmm_server_submit(ifmm_server* s, int id, const double* b_host, double* x_host,
                               int nrhs, double tol, int maxit, long long* ticket) {
  if (!s || !b_host || !x_host || !ticket || nrhs < 1 || !(tol > 0.0) || maxit < 1)
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
  r->b = b_host;
  r->x = x_host;
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
