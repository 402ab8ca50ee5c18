// serve.cpp -- a continuous-batching request server over one GPU for the hot path: log-likelihood and
// predictive-mean requests (Sec. 3.2, Sec. 3.3) on cached point sets, admitted as slots and device memory free up.
//
// The server owns a set of point sets (steps A1, A2, A5, A6 done once and cached) and `slots` workers. A
// worker is a host thread with its own context and CUDA stream; the requests of different slots run
// concurrently on the device. Requests wait in one FIFO queue. A free worker admits the request at the head
// when either it already holds an idle factor of the same point set and precision (re-used through
// gp_factor_update: no allocation), or the factor's bytes fit the server's memory budget, after idle cached
// factors of any slot have been evicted (least recently used first). A request that can never fit is refused
// at submission. Each result depends only on its request (no kernel of the path uses atomics on data), so a
// request returns the same numbers alone and in the mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "gp_internal.cuh"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// A request with its hyperparameter setting copied into storage it owns.
struct Req {
  int64_t id = 0;
  gp_request r{};
  std::vector<double> store;   // core_radius, r0, h, a, b, r
  gp_hyper th{};
  size_t need = 0;             // bytes of a new factor for (point set, precision)
  double t_submit = 0.0;
};

struct Cached {
  gp_factor_t* f = nullptr;
  int32_t ps = -1;
  gp_precision prec = GP_FP64;
  int slot = -1;
  size_t bytes = 0;
  bool busy = false;
  double last = 0.0;
};

struct Slot {
  gp_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  double* scratch = nullptr;   // device: the log-likelihood of predict requests (their alpha is what is needed)
  std::thread th;
};

void copy_theta(Req& q, const gp_hyper& t) {
  const int nb = t.n1 * t.n2;
  const size_t nh = (size_t)nb * t.bump_dims;
  q.store.assign((size_t)2 * t.d + nh + 3 * (size_t)nb, 0.0);
  double* p = q.store.data();
  auto take = [&](const double* src, size_t k) {
    double* dst = p;
    if (k) std::copy(src, src + k, dst);
    p += k;
    return dst;
  };
  q.th = t;
  q.th.core_radius = take(t.core_radius, t.d);
  q.th.r0 = take(t.r0, t.d);
  q.th.h = take(t.h, nh);
  q.th.a = take(t.a, nb);
  q.th.b = take(t.b, nb);
  q.th.r = take(t.r, nb);
}

}  // namespace

struct gp_server_s {
  int device = 0;
  size_t budget = 0;
  size_t held = 0, peak = 0;   // factor bytes reserved or held, and their maximum
  gp_ctx* ps_ctx = nullptr;
  cudaStream_t ps_stream = nullptr;
  std::vector<gp_pointset*> psets;
  std::vector<std::unique_ptr<Slot>> slots;
  std::list<Cached> cache;
  std::deque<Req*> queue;
  std::vector<gp_completion> done;
  int64_t next_id = 0, completed = 0;
  int running = 0, max_running = 0;
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv;
  std::string err;

  // Under mu: can slot k take the head request now? On success the head is popped, a cached factor is marked
  // busy or memory reserved (with victims to free handed back), and *entry points at the cache entry.
  bool admit(int k, Req** out, std::list<Cached>::iterator* entry, std::vector<gp_factor_t*>* victims) {
    if (queue.empty()) return false;
    Req* q = queue.front();
    for (auto it = cache.begin(); it != cache.end(); ++it)
      if (!it->busy && it->slot == k && it->ps == q->r.pointset && it->prec == q->r.precision) {
        it->busy = true;
        *entry = it;
        *out = q;
        queue.pop_front();
        return true;
      }
    // evict idle factors, least recently used first, until the new factor fits
    size_t freeable = 0;
    for (auto& c : cache)
      if (!c.busy) freeable += c.bytes;
    if (held + q->need > budget + freeable) return false;
    while (held + q->need > budget) {
      auto lru = cache.end();
      for (auto it = cache.begin(); it != cache.end(); ++it)
        if (!it->busy && (lru == cache.end() || it->last < lru->last)) lru = it;
      victims->push_back(lru->f);
      held -= lru->bytes;
      cache.erase(lru);
    }
    held += q->need;
    peak = std::max(peak, held);
    Cached c;
    c.ps = q->r.pointset;
    c.prec = q->r.precision;
    c.slot = k;
    c.bytes = q->need;
    c.busy = true;
    cache.push_front(c);
    *entry = cache.begin();
    *out = q;
    queue.pop_front();
    return true;
  }

  void worker(int k) {
    Slot& sl = *slots[k];
    cudaSetDevice(device);
    for (;;) {
      Req* q = nullptr;
      std::list<Cached>::iterator e;
      std::vector<gp_factor_t*> victims;
      gp_pointset* ps = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || admit(k, &q, &e, &victims); });
        if (!q) return;   // stopping
        ps = psets[q->r.pointset];
        running++;
        max_running = std::max(max_running, running);
      }
      for (gp_factor_t* v : victims) gp_factor_free(v);   // idle factors of any slot
      const double t_start = now_s();
      gp_status st = GP_OK;
      gp_factor_t* f = e->f;
      if (!f) {
        st = gp_factor(sl.ctx, ps, &q->th, 1, q->r.precision, &f);
      } else {
        st = gp_factor_update(sl.ctx, f, &q->th);
      }
      if (st == GP_OK) {
        double* ll = q->r.kind == GP_REQ_LOGLIK ? q->r.d_out : sl.scratch;
        st = gp_loglik(sl.ctx, f, q->r.d_resid, ll, q->r.d_err);
      }
      if (st == GP_OK && q->r.kind == GP_REQ_PREDICT)
        st = gp_predict(sl.ctx, f, 0, q->r.d_Xtest, q->r.m, q->r.d_mu_test, q->r.d_out);
      if (cudaStreamSynchronize(sl.stream) != cudaSuccess && st == GP_OK) st = GP_ERR_CUDA;
      const double t_done = now_s();
      size_t actual = 0;
      if (f && !e->f) {
        gp_factor_info_t fi;
        if (gp_factor_info(f, &fi, nullptr) == GP_OK) actual = (size_t)fi.bytes;
      }
      gp_factor_t* drop = nullptr;   // a new factor whose request failed
      {
        std::lock_guard<std::mutex> lk(mu);
        if (!e->f && st == GP_OK) {   // keep the new factor at its true size
          e->f = f;
          held = held - e->bytes + actual;
          e->bytes = actual;
          peak = std::max(peak, held);
        }
        if (e->f) {
          e->busy = false;
          e->last = t_done;
        } else {   // give the reservation back
          held -= e->bytes;
          cache.erase(e);
          drop = f;
        }
        gp_completion c{};
        c.id = q->id;
        c.status = st;
        c.slot = k;
        c.t_submit = q->t_submit;
        c.t_start = t_start;
        c.t_done = t_done;
        done.push_back(c);
        completed++;
        running--;
        if (st != GP_OK) err = gp_last_error(sl.ctx);
      }
      if (drop) gp_factor_free(drop);
      delete q;
      cv.notify_all();
    }
  }
};

extern "C" gp_status gp_server_create(int device, int slots, size_t mem_budget_bytes, gp_server_t** out) {
  if (!out || slots < 1 || slots > 64) return GP_ERR_ARG;
  *out = nullptr;
  auto* s = new gp_server_s();
  s->device = device;
  s->budget = mem_budget_bytes;
  gp_status st = GP_OK;
  if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&s->ps_stream, cudaStreamNonBlocking) !=
                                                  cudaSuccess) {
    cudaGetLastError();
    delete s;
    return GP_ERR_CUDA;
  }
  st = gp_create(&s->ps_ctx, device, s->ps_stream, 0);
  for (int k = 0; st == GP_OK && k < slots; k++) {
    auto sl = std::make_unique<Slot>();
    if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&sl->scratch, sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      st = GP_ERR_CUDA;
    } else {
      st = gp_create(&sl->ctx, device, sl->stream, 0);
    }
    s->slots.push_back(std::move(sl));
  }
  if (st != GP_OK) {
    gp_server_destroy(s);
    return st;
  }
  for (int k = 0; k < slots; k++) s->slots[k]->th = std::thread([s, k] { s->worker(k); });
  *out = s;
  return GP_OK;
}

extern "C" gp_status gp_server_add_pointset(gp_server_t* s, const double* d_X, int64_t n, int d,
                                            const double* core_radius, int32_t* id) {
  if (!s || !id) return GP_ERR_ARG;
  gp_pointset* ps = nullptr;
  gp_status st = gp_assemble(s->ps_ctx, d_X, n, d, core_radius, &ps);
  if (st == GP_OK) st = gp_pointset_prepare(s->ps_ctx, ps, GP_MIXED);
  std::lock_guard<std::mutex> lk(s->mu);
  if (st != GP_OK) {
    s->err = gp_last_error(s->ps_ctx);
    if (ps) gp_pointset_free(ps);
    return st;
  }
  s->psets.push_back(ps);
  *id = (int32_t)s->psets.size() - 1;
  return GP_OK;
}

extern "C" gp_status gp_server_submit(gp_server_t* s, const gp_request* r, int64_t* id) {
  if (!s || !r || !r->theta || !r->d_resid || !r->d_out) return GP_ERR_ARG;
  if (r->kind != GP_REQ_LOGLIK && r->kind != GP_REQ_PREDICT) return GP_ERR_ARG;
  if (r->kind == GP_REQ_PREDICT && (!r->d_Xtest || r->m < 1)) return GP_ERR_ARG;
  if (r->precision != GP_FP64 && r->precision != GP_MIXED) return GP_ERR_ARG;
  auto* q = new Req();
  gp_pointset* ps = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->pointset < 0 || r->pointset >= (int32_t)s->psets.size()) {
      delete q;
      return GP_ERR_ARG;
    }
    ps = s->psets[r->pointset];
  }
  q->r = *r;
  copy_theta(*q, *r->theta);
  q->r.theta = &q->th;
  if (gp_factor_bytes(ps, &q->th, 1, r->precision, &q->need) != GP_OK) {
    delete q;
    return GP_ERR_ARG;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (q->need > s->budget) {   // can never be admitted
      s->err = "request needs " + std::to_string(q->need) + " bytes, the budget is " + std::to_string(s->budget);
      delete q;
      return GP_ERR_NOMEM;
    }
    q->id = s->next_id++;
    q->t_submit = now_s();
    if (id) *id = q->id;
    s->queue.push_back(q);
  }
  s->cv.notify_all();
  return GP_OK;
}

extern "C" int gp_server_poll(gp_server_t* s, gp_completion* out, int max) {
  if (!s || !out || max < 1) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  const int k = (int)std::min<size_t>((size_t)max, s->done.size());
  std::copy(s->done.begin(), s->done.begin() + k, out);
  s->done.erase(s->done.begin(), s->done.begin() + k);
  return k;
}

extern "C" gp_status gp_server_wait(gp_server_t* s, double timeout_s) {
  if (!s) return GP_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [&] { return s->queue.empty() && s->running == 0; };
  if (timeout_s <= 0) {
    s->cv.wait(lk, idle);
    return GP_OK;
  }
  return s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), idle) ? GP_OK : GP_ERR_TIMEOUT;
}

extern "C" gp_status gp_server_stats(gp_server_t* s, gp_server_stats_t* st) {
  if (!s || !st) return GP_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  st->budget = s->budget;
  st->held = s->held;
  st->peak = s->peak;
  st->cached_factors = (int32_t)s->cache.size();
  st->queued = (int32_t)s->queue.size();
  st->running = s->running;
  st->max_running = s->max_running;
  st->completed = s->completed;
  return GP_OK;
}

extern "C" const char* gp_server_last_error(const gp_server_t* s) { return s ? s->err.c_str() : ""; }

extern "C" void gp_server_destroy(gp_server_t* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (Req* q : s->queue) delete q;
    s->queue.clear();
  }
  s->cv.notify_all();
  for (auto& sl : s->slots)
    if (sl->th.joinable()) sl->th.join();
  cudaSetDevice(s->device);
  for (auto& c : s->cache)
    if (c.f) gp_factor_free(c.f);
  s->cache.clear();
  for (gp_pointset* ps : s->psets) gp_pointset_free(ps);
  s->psets.clear();
  for (auto& sl : s->slots) {
    if (sl->ctx) gp_destroy(sl->ctx);
    if (sl->scratch) cudaFree(sl->scratch);
    if (sl->stream) cudaStreamDestroy(sl->stream);
  }
  if (s->ps_ctx) gp_destroy(s->ps_ctx);
  if (s->ps_stream) cudaStreamDestroy(s->ps_stream);
  delete s;
}
