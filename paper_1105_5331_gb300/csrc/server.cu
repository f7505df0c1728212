// Continuous batching of CP decompositions on one GPU.
//
// A server owns `max_active` slots; each slot has its own streams, event,
// status word and pinned buffers (SolverRes).  Requests wait in arrival order
// and are admitted while a slot is free and the sum of the device footprints
// of running requests plus the new one stays within the HBM budget.  An
// admitted request uploads its tensor (per-mode copies, bf16 planes) and
// launches its own device-resident solve (one CUDA graph per precision phase,
// see solve.cu) on its slot's stream, so the iterations of all running
// requests overlap on the device.  A worker thread polls the slots without
// blocking, retires finished requests (result copied to the caller's host
// buffer, latency stamped) and admits waiting ones as slots and memory free
// up.  Every allocation on this path is stream-ordered, so admitting or
// retiring one request never waits for the others.
//
// Each request's result depends only on its own data (no cross-request
// reduction, fixed launch shapes), so it is the same alone and in a mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cp_internal.cuh"
#include "solver.cuh"

namespace cpg {

cp_status solve_impl(cp_ctx* ctx, const cp_tensor* t, const cp_solve_opts* o, double* u_user, bool user_on_device,
                     cp_solve_report* rep);

// The cluster engine (many.cu).
struct ManyEngine;
ManyEngine* many_engine_create(cp_ctx* ctx, int capacity, cp_status* st);
void many_engine_destroy(ManyEngine* e);
cp_status many_engine_add(ManyEngine* e, const cp_tensor* t, const cp_solve_opts& o, const double* u0, int* slot);
int many_engine_running(ManyEngine* e);
void many_engine_set_cta_cap(ManyEngine* e, int max_ctas);
bool many_engine_in_flight(ManyEngine* e);
cp_status many_engine_launch(ManyEngine* e, double budget_s);
cp_status many_engine_poll(ManyEngine* e, bool block, bool* idle, std::vector<int>* finished);
cp_status many_engine_result(ManyEngine* e, int slot, double* u_out, cp_solve_report* rep, cp_status* st);
void many_engine_release(ManyEngine* e, int slot);
const char* many_unsupported_dims(int kind, int N, const int64_t* dims, const cp_solve_opts& o);
size_t many_state_bytes(const int64_t* dims, const cp_solve_opts& o);

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

enum ReqState { REQ_PENDING = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_CANCELLED = 3 };

struct Request {
  uint64_t id = 0;
  int N = 0;
  int64_t dims[CP_MAX_N] = {0};
  cp_dtype dtype = CP_DTYPE_F32;
  std::vector<char> data;          // host copy of the tensor
  std::vector<double> u0;          // host copy of the initial guess
  double* u_out = nullptr;         // caller's host buffer for the result
  cp_solve_opts opts{};
  size_t footprint = 0;
  bool engine_ok = false;          // fits the cluster engine
  long long work = 0;              // entries x R
  Clock::time_point t_submit, t_admit, t_done;
  int state = REQ_PENDING;
  cp_status status = CP_OK;
  cp_solve_report rep{};
};

struct Slot {
  SolverRes res;
  std::unique_ptr<Solver> solver;
  cp_tensor* t = nullptr;
  Request* req = nullptr;
};

}  // namespace

// Device bytes a request needs while it runs (tensor copies, bf16 planes,
// solver state, graph workspace): an estimate used for admission.
size_t request_footprint(int N, const int64_t* dims, cp_dtype dtype, const cp_solve_opts& o) {
  size_t K = 1, sumI = 0, Imax = 1;
  for (int n = 0; n < N; ++n) {
    K *= (size_t)dims[n];
    sumI += (size_t)dims[n];
    Imax = std::max(Imax, (size_t)dims[n]);
  }
  const size_t esz = dtype == CP_DTYPE_F64 ? 8 : 4;
  const size_t P = sumI * (size_t)o.R;
  size_t bytes = (size_t)N * K * esz + K * esz;                 // per-mode copies + upload
  if (o.prec != CP_FP64) bytes += (size_t)N * (K + 8 * Imax) * 4;  // bf16 hi/lo planes
  // solver state: iterate-sized vectors and the window, M^(1) / M^(N) copies,
  // the line-search variants of every mode, Grams, inverses, FP32 copies
  const size_t RR = (size_t)o.R * o.R;
  const size_t rs = ((size_t)o.R + 3) / 4 * 4;
  const size_t n32 = (sumI * rs + 31) / 32 * 16;
  bytes += sizeof(double) * ((9 + 2 * (size_t)o.w) * P + Imax * o.R + (size_t)N * RR + 5 * Imax * o.R +
                             ((size_t)1 << (N - 1)) * P + 6 * (size_t)N * RR + 3 * (RR + 2) + 3 * n32 + 128);
  bytes += sizeof(double) * 12 * P + (size_t)4 * 152 * Imax * o.R * 6 + ((size_t)8 << 20);   // workspace
  return bytes;
}

}  // namespace cpg

using namespace cpg;

struct cp_server {
  // requests on the cluster engine, by engine slot
  struct EngReq {
    Request* r = nullptr;
    cp_tensor* t = nullptr;
  };
  cp_ctx* ctx = nullptr;        // caller's context (device)
  ManyEngine* eng = nullptr;    // the cluster engine (3-way dense requests within its limits)
  bool engine_on = true;
  long long engine_max_work = 1ll << 26;   // entries x R of the largest request routed to the engine
  std::vector<EngReq> ereq;
  int eng_used = 0;
  double round_s = 0.010;       // engine round length
  cp_ctx* wctx = nullptr;       // worker's own context (stream for uploads)
  size_t budget = 0, used = 0, peak = 0;
  int max_active = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<double> latencies;
  bool any_submit = false;
  Clock::time_point t_first, t_last;
  uint64_t next_id = 1;
  int running = 0, completed = 0;
  std::atomic<bool> stop{false};
  std::thread worker;
  cp_status worker_error = CP_OK;

  void admit(Slot& sl, Request* r) {
    sl.req = r;
    r->t_admit = Clock::now();
    cp_tensor* t = nullptr;
    cp_status st = cp_tensor_dense(wctx, r->N, r->dims, r->dtype, r->data.data(), &t);
    if (st == CP_OK) {
      sl.t = t;
      // the slot's stream must see the finished upload
      cudaEvent_t ev;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(ev, wctx->stream);
        cudaStreamWaitEvent(sl.res.stream, ev, 0);
        cudaEventDestroy(ev);
      }
      sl.solver.reset(new Solver());
      st = sl.solver->start(ctx, t, r->opts, r->u0.data(), false, &sl.res);
    }
    if (st != CP_OK) {
      if (sl.solver) {
        sl.solver->finished = true;
        sl.solver->result = st;
      }
      finish(sl, st);
      return;
    }
  }

  void finish(Slot& sl, cp_status st) {
    Request* r = sl.req;
    if (sl.solver) {
      if (st == CP_OK) st = sl.solver->result;
      if (st == CP_OK || st == CP_ERR_MAXIT) {
        const cp_status c = sl.solver->copy_out(r->u_out, false);
        if (c != CP_OK) st = c;
      }
      sl.solver->rep_fill();
      r->rep = sl.solver->rep;
      if (st == CP_OK && !sl.solver->converged) st = CP_ERR_MAXIT;
      sl.solver.reset();   // stream-ordered frees on the slot stream
    }
    if (sl.t) {
      tensor_release(sl.t, sl.res.stream);
      sl.t = nullptr;
    }
    sl.req = nullptr;
    done(r, st);
  }

  void done(Request* r, cp_status st) {
    r->t_done = Clock::now();
    std::lock_guard<std::mutex> lock(mu);
    r->status = st;
    r->state = REQ_DONE;
    used -= r->footprint;
    --running;
    ++completed;
    latencies.push_back(seconds_since(r->t_submit, r->t_done));
    t_last = r->t_done;
    cv.notify_all();
  }

  // Admit r to the cluster engine: its tensor (complete on return), then
  // its state; it joins the next engine round.
  void admit_engine(Request* r) {
    r->t_admit = Clock::now();
    cp_tensor* t = nullptr;
    cp_status st = cp_tensor_dense(wctx, r->N, r->dims, r->dtype, r->data.data(), &t);
    int k = -1;
    if (st == CP_OK) st = many_engine_add(eng, t, r->opts, r->u0.data(), &k);
    if (st != CP_OK) {
      if (t) tensor_release(t, wctx->stream);
      done(r, st);
      return;
    }
    ereq[(size_t)k].r = r;
    ereq[(size_t)k].t = t;
    ++eng_used;
  }

  void finish_engine(int k) {
    EngReq& e = ereq[(size_t)k];
    Request* r = e.r;
    cp_status rs = CP_OK;
    cp_status st = many_engine_result(eng, k, r->u_out, &r->rep, &rs);
    if (st == CP_OK) st = rs;
    r->rep.t_total_s = seconds_since(r->t_admit, Clock::now());
    many_engine_release(eng, k);
    tensor_release(e.t, wctx->stream);
    e = EngReq();
    --eng_used;
    done(r, st);
  }

  void loop() {
    cudaSetDevice(ctx->device);
    while (!stop.load()) {
      bool progress = false;
      for (auto& sl : slots) {
        if (sl.req && sl.solver && sl.solver->poll(false)) {
          finish(sl, CP_OK);
          progress = true;
        }
      }
      if (eng && many_engine_in_flight(eng)) {
        bool idle = false;
        std::vector<int> fin;
        const cp_status st = many_engine_poll(eng, false, &idle, &fin);
        if (st != CP_OK) {
          worker_error = st;
          for (size_t k = 0; k < ereq.size(); ++k)
            if (ereq[k].r) fin.push_back((int)k);
        }
        for (int k : fin) finish_engine(k);
        if (idle || st != CP_OK) progress = true;
      }
      // admission in arrival order: the head request goes to the engine when
      // it fits it, else to a graph slot; it waits while its kind is full
      for (;;) {
        Request* r = nullptr;
        bool to_engine = false;
        Slot* free_slot = nullptr;
        for (auto& sl : slots)
          if (!sl.req) {
            free_slot = &sl;
            break;
          }
        {
          std::lock_guard<std::mutex> lock(mu);
          while (!pending.empty() && pending.front()->state == REQ_CANCELLED) pending.pop_front();
          if (!pending.empty()) {
            Request* h = pending.front();
            // FP64 requests compute their passes in FP64 on the engine's
            // few SMs (2 FP64 FMA per clock per SM): a 64th of the limit
            const long long mw = h->opts.prec == CP_FP64 ? engine_max_work / 64 : engine_max_work;
            to_engine = eng && engine_on && h->engine_ok && (engine_max_work <= 0 || h->work <= mw);
            const bool room = to_engine ? eng_used < (int)ereq.size() : free_slot != nullptr;
            if (room && used + h->footprint <= budget) {
              r = h;
              pending.pop_front();
              r->state = REQ_RUNNING;   // under the lock: a cancel from now on is refused
              used += r->footprint;
              peak = std::max(peak, used);
              ++running;
            }
          }
        }
        if (!r) break;
        if (to_engine)
          admit_engine(r);
        else
          admit(*free_slot, r);
        progress = true;
      }
      if (eng && !many_engine_in_flight(eng) && many_engine_running(eng) > 0) {
        const cp_status st = many_engine_launch(eng, round_s);
        if (st != CP_OK) worker_error = st;
        progress = true;
      }
      if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
};

extern "C" {

cp_status cp_server_create(cp_ctx* ctx, size_t hbm_budget_bytes, int max_active, cp_server** out) {
  if (!ctx || !out || max_active < 1 || max_active > 1024 || hbm_budget_bytes == 0) {
    set_error("cp_server_create: bad arguments");
    return CP_ERR_ARG;
  }
  *out = nullptr;
  CP_CUDA(cudaSetDevice(ctx->device));
  std::unique_ptr<cp_server> s(new cp_server());
  s->ctx = ctx;
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  CP_TRY(cp_ctx_create(ctx->device, nullptr, &s->wctx));
  s->slots.resize((size_t)max_active);
  for (auto& sl : s->slots) {
    const cp_status st = sl.res.create();
    if (st != CP_OK) {   // release what was made (destroy skips what was not)
      for (auto& q : s->slots) q.res.destroy();
      cp_ctx_destroy(s->wctx);
      return st;
    }
  }
  {
    cp_status est = CP_OK;
    s->eng = many_engine_create(ctx, max_active, &est);
    if (s->eng) {
      s->ereq.resize((size_t)max_active);
    }
  }
  cp_server* raw = s.release();
  raw->worker = std::thread([raw]() { raw->loop(); });
  *out = raw;
  return CP_OK;
}

cp_status cp_server_submit(cp_server* s, int N, const int64_t* dims, cp_dtype dtype, const void* data,
                           const cp_solve_opts* opts, const double* u0, double* u_out, uint64_t* req_id) {
  if (!s || !dims || !data || !opts || !u0 || !u_out || !req_id || N < 2 || N > CP_MAX_N) {
    set_error("cp_server_submit: bad arguments");
    return CP_ERR_ARG;
  }
  if (opts->R < 1 || opts->R > CP_MAX_R || opts->w < 1 || opts->w > CP_MAX_W || !(opts->tol > 0)) {
    set_error("cp_server_submit: bad options");
    return CP_ERR_ARG;
  }
  std::unique_ptr<Request> r(new Request());
  size_t K = 1, sumI = 0;
  for (int n = 0; n < N; ++n) {
    if (dims[n] < 1) {
      set_error("cp_server_submit: dim %d < 1", n);
      return CP_ERR_SHAPE;
    }
    r->dims[n] = dims[n];
    K *= (size_t)dims[n];
    sumI += (size_t)dims[n];
  }
  r->N = N;
  r->dtype = dtype;
  r->opts = *opts;
  const size_t esz = dtype == CP_DTYPE_F64 ? 8 : 4;
  r->data.assign((const char*)data, (const char*)data + K * esz);
  r->u0.assign(u0, u0 + sumI * (size_t)opts->R);
  r->u_out = u_out;
  r->engine_ok = many_unsupported_dims(0, N, dims, *opts) == nullptr;
  r->work = (long long)K * opts->R;
  r->footprint = r->engine_ok ? (size_t)(N + 1) * K * esz + many_state_bytes(dims, *opts)
                              : request_footprint(N, dims, dtype, *opts);
  if (r->footprint > s->budget) {
    set_error("cp_server_submit: request needs ~%zu bytes, budget %zu", r->footprint, s->budget);
    return CP_ERR_BUSY;
  }
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  if (!s->any_submit) {
    s->any_submit = true;
    s->t_first = r->t_submit;
  }
  r->id = s->next_id++;
  *req_id = r->id;
  s->pending.push_back(r.get());
  s->reqs[r->id] = std::move(r);
  return CP_OK;
}

cp_status cp_server_poll(cp_server* s, uint64_t req_id, int* done, cp_status* req_status, cp_solve_report* rep,
                         double* latency_s) {
  if (!s || !done) {
    set_error("cp_server_poll: bad arguments");
    return CP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) {
    set_error("cp_server_poll: unknown request %llu", (unsigned long long)req_id);
    return CP_ERR_ARG;
  }
  Request* r = it->second.get();
  *done = (r->state == REQ_DONE || r->state == REQ_CANCELLED) ? 1 : 0;
  if (*done) {
    if (req_status) *req_status = r->status;
    if (rep) *rep = r->rep;
    if (latency_s) *latency_s = r->state == REQ_DONE ? seconds_since(r->t_submit, r->t_done) : 0.0;
  }
  return CP_OK;
}

cp_status cp_server_cancel(cp_server* s, uint64_t req_id) {
  if (!s) return CP_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end() || it->second->state != REQ_PENDING) {
    set_error("cp_server_cancel: request %llu is not waiting", (unsigned long long)req_id);
    return CP_ERR_ARG;
  }
  it->second->state = REQ_CANCELLED;
  it->second->status = CP_ERR_ARG;
  s->cv.notify_all();
  return CP_OK;
}

cp_status cp_server_drain(cp_server* s, double timeout_s) {
  if (!s) return CP_ERR_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto all_done = [&]() {
    for (auto& kv : s->reqs)
      if (kv.second->state == REQ_PENDING || kv.second->state == REQ_RUNNING) return false;
    return true;
  };
  if (!s->cv.wait_for(lock, std::chrono::duration<double>(timeout_s), all_done)) {
    set_error("cp_server_drain: timed out");
    return CP_ERR_TIMEOUT;
  }
  return CP_OK;
}

cp_status cp_server_stats(cp_server* s, double* p50_s, double* p99_s, double* solves_per_s, int* completed,
                          size_t* peak_bytes) {
  if (!s) return CP_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    size_t i = (size_t)std::ceil(q * (double)l.size()) - 1;
    return l[std::min(i, l.size() - 1)];
  };
  if (p50_s) *p50_s = pct(0.50);
  if (p99_s) *p99_s = pct(0.99);
  if (solves_per_s) {
    const double span = s->completed ? seconds_since(s->t_first, s->t_last) : 0.0;
    *solves_per_s = span > 0 ? (double)s->completed / span : 0.0;
  }
  if (completed) *completed = s->completed;
  if (peak_bytes) *peak_bytes = s->peak;
  return CP_OK;
}

cp_status cp_server_set_engine(cp_server* s, int on, long long max_work, int max_ctas) {
  if (!s || on < 0 || on > 1) {
    set_error("cp_server_set_engine: bad arguments");
    return CP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  if (on && !s->eng) {
    set_error("cp_server_set_engine: the cluster engine is not available on this device");
    return CP_ERR_UNSUPPORTED;
  }
  s->engine_on = on != 0;
  s->engine_max_work = max_work;
  if (s->eng) many_engine_set_cta_cap(s->eng, max_ctas > 0 ? max_ctas : 0);
  return CP_OK;
}

void cp_server_destroy(cp_server* s) {
  if (!s) return;
  s->stop.store(true);
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->ctx->device);
  if (s->eng) {
    // engine requests still running finish in further rounds
    for (;;) {
      if (many_engine_in_flight(s->eng)) {
        bool idle = false;
        std::vector<int> fin;
        if (many_engine_poll(s->eng, true, &idle, &fin) != CP_OK) break;
        for (int k : fin) s->finish_engine(k);
      }
      if (many_engine_running(s->eng) == 0) break;
      if (many_engine_launch(s->eng, s->round_s) != CP_OK) break;
    }
    for (size_t k = 0; k < s->ereq.size(); ++k)
      if (s->ereq[k].r) {
        many_engine_release(s->eng, (int)k);
        tensor_release(s->ereq[k].t, s->wctx->stream);
        s->ereq[k] = cp_server::EngReq();
      }
    many_engine_destroy(s->eng);
    s->eng = nullptr;
  }
  for (auto& sl : s->slots) {
    if (sl.solver)
      while (!sl.solver->poll(true)) {
      }
    sl.solver.reset();
    if (sl.t) tensor_release(sl.t, sl.res.stream);
    sl.t = nullptr;
    sl.res.destroy();
  }
  cp_ctx_destroy(s->wctx);
  delete s;
}

cp_status cp_solve_batch(cp_ctx* ctx, int nreq, const cp_tensor* const* tensors, const cp_solve_opts* opts,
                         double* const* u, cp_solve_report* reps) {
  if (!ctx || nreq < 0 || (nreq > 0 && (!tensors || !opts || !u))) {
    set_error("cp_solve_batch: bad arguments");
    return CP_ERR_ARG;
  }
  CP_CUDA(cudaSetDevice(ctx->device));
  CP_CUDA(cudaStreamSynchronize(ctx->stream));
  std::vector<std::unique_ptr<Solver>> sv((size_t)nreq);
  std::vector<bool> dev((size_t)nreq);
  cp_status first = CP_OK;
  for (int i = 0; i < nreq; ++i) {
    if (!tensors[i] || !u[i] || tensors[i]->device != ctx->device) {
      if (first == CP_OK) {
        set_error("cp_solve_batch: request %d: null tensor or iterate, or tensor on another device", i);
        first = CP_ERR_ARG;
      }
      continue;
    }
    dev[i] = on_device(u[i]);
    sv[i].reset(new Solver());
    const cp_status st = sv[i]->start(ctx, tensors[i], opts[i], u[i], dev[i]);
    if (st != CP_OK) {
      sv[i]->finished = true;
      sv[i]->result = st;
    }
  }
  bool all = false;
  while (!all) {
    all = true;
    for (int i = 0; i < nreq; ++i)
      if (sv[i] && !sv[i]->finished && !sv[i]->poll(false)) all = false;
    if (!all) std::this_thread::sleep_for(std::chrono::microseconds(10));
  }
  for (int i = 0; i < nreq; ++i) {
    if (!sv[i]) continue;
    cp_status st = sv[i]->result;
    if (st == CP_OK) st = sv[i]->copy_out(u[i], dev[i]);
    sv[i]->rep_fill();
    if (reps) reps[i] = sv[i]->rep;
    if (st == CP_OK && !sv[i]->converged) st = CP_ERR_MAXIT;
    if (st != CP_OK && first == CP_OK) first = st;
  }
  return first;
}

}  // extern "C"
