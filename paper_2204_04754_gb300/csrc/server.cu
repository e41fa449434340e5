// Request server for projected-EM solves with continuous batching.
//
// Requests (one SR-MRA problem each: observations, sizes, noise level, iteration count
// and Algorithm 2 schedule) are queued by srmra_server_submit.  Every
// srmra_server_step call
//   1. admits queued requests in arrival order while a slot is free and the device
//      memory they need (srmra_estimate_device_bytes) fits the server's budget: the
//      request's context is created, which uploads its observations to the device where
//      they stay, with x and rho, until the request retires;
//   2. advances every admitted request by one EM iteration (+ its scheduled projection)
//      as one batch: grouped persistent launches over the work units of all requests,
//      replayed from a CUDA graph that is re-captured only when the set of requests
//      changes;
//   3. retires requests that reached their iteration count: the estimate is copied to
//      host memory, the context and its device memory are released.
// Requests that arrive while others are running join at the next iteration boundary, so
// their work shares the device with the running ones.  A server created with
// SRMRA_SERVER_AUTO picks each request's form from its size (the polyphase-FFT form where
// it exists, L/K in {8, 16, 32}, split bf16 otherwise) and keeps one batch per form.  A request's arithmetic does not
// depend on the other requests in the batch (same per-problem work decomposition, no
// cross-problem reductions), so its result equals a solve of the same problem alone.
#include <chrono>
#include <deque>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "srmra_internal.cuh"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t id = 0;
  srmra_params p{};
  std::vector<float> y;
  std::vector<float> x0;
  int32_t iters = 0, F = 0;
  double sigma_bm1 = 1.0, decay = 0.93303299153680741598;
  int64_t bytes = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  srmra_ctx* ctx = nullptr;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  srmra_status status = SRMRA_OK;
  std::string err;
  std::vector<float> x;
  std::vector<double> rho1, rho2;
  double ll_last = 0.0;
};

}  // namespace

struct srmra_server {
  int64_t budget = 0;
  int32_t max_active = 0;
  int32_t prec = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  int64_t next_id = 1;
  std::deque<Request*> queue;
  std::vector<Request*> running;
  std::unordered_map<int64_t, Request*> all;
  int64_t used = 0;
  srmra_batch* batch[4] = {nullptr, nullptr, nullptr, nullptr};  // one per precision form
  bool dirty[4] = {true, true, true, true};
  int64_t iterations = 0;
  std::string err;
};

namespace {

thread_local std::string g_server_err;

srmra_status sfail(srmra_server* s, srmra_status st, const std::string& msg) {
  if (s)
    s->err = msg;
  else
    g_server_err = msg;
  return st;
}

void retire(srmra_server* s, Request* r) {
  const int L = r->p.L_high;
  r->x.resize((size_t)L * L);
  r->rho1.resize(L);
  r->rho2.resize(L);
  double sbm = 0;
  int32_t t = 0;
  r->status = srmra_get_state(r->ctx, r->x.data(), r->rho1.data(), r->rho2.data(), &sbm, &t);
  if (r->status == SRMRA_OK)
    r->status = (cudaMemcpy(&r->ll_last, r->ctx->ll_hist, sizeof(double),
                            cudaMemcpyDeviceToHost) == cudaSuccess)
                    ? SRMRA_OK
                    : SRMRA_ECUDA;
  r->state = (r->status == SRMRA_OK) ? 2 : 3;
  srmra_destroy(r->ctx);
  r->ctx = nullptr;
  s->used -= r->bytes;
  r->t_done = now_ms();
  std::vector<float>().swap(r->y);
}

}  // namespace

extern "C" {

srmra_status srmra_server_create(int64_t device_budget_bytes, int32_t max_active, int32_t prec,
                                 void* cuda_stream, srmra_server** out) {
  if (!out) return sfail(nullptr, SRMRA_EINVAL, "out is NULL");
  *out = nullptr;
  if (device_budget_bytes <= 0 || max_active < 1)
    return sfail(nullptr, SRMRA_EINVAL, "need a positive memory budget and slot count");
  if (prec != SRMRA_FP32 && prec != SRMRA_BF16 && prec != SRMRA_BF16X3 && prec != SRMRA_FFT32 &&
      prec != SRMRA_SERVER_AUTO)
    return sfail(nullptr, SRMRA_EINVAL, "unknown precision form");
  auto* s = new (std::nothrow) srmra_server();
  if (!s) return sfail(nullptr, SRMRA_ENOMEM, "host allocation failed");
  s->budget = device_budget_bytes;
  s->max_active = max_active;
  s->prec = prec;
  s->stream = (cudaStream_t)cuda_stream;
  *out = s;
  return SRMRA_OK;
}

srmra_status srmra_server_submit(srmra_server* s, const srmra_params* p, const float* y,
                                 const float* x0, int32_t iters, int32_t F, double sigma_bm1,
                                 double decay, int64_t* request_id) {
  if (!s || !p || !y || !request_id)
    return sfail(s, SRMRA_EINVAL, "server, params, y and request_id are required");
  if (iters < 1 || F < 0 || !(decay > 0.0) || !(sigma_bm1 > 0.0))
    return sfail(s, SRMRA_EINVAL, "need iters >= 1, F >= 0, decay > 0, sigma_bm1 > 0");
  srmra_params q = *p;
  q.prec = s->prec;
  if (s->prec == SRMRA_SERVER_AUTO) {
    const int l = p->K > 0 ? p->L_high / p->K : 0;
    q.prec = (l == 8 || l == 16 || l == 32) && l * p->K == p->L_high ? SRMRA_FFT32
                                                                      : SRMRA_BF16X3;
  }
  if (F > 0 && q.L_high % 8 != 0)
    return sfail(s, SRMRA_EINVAL, "built-in denoiser needs L % 8 == 0");
  int64_t bytes = 0;
  srmra_status st = srmra_estimate_device_bytes(&q, &bytes);
  if (st != SRMRA_OK) return sfail(s, st, srmra_last_error(nullptr));
  if (bytes > s->budget) return sfail(s, SRMRA_ENOMEM, "request larger than the memory budget");
  if (!(q.sigma > 0.0)) return sfail(s, SRMRA_EINVAL, "need sigma > 0");
  auto* r = new (std::nothrow) Request();
  if (!r) return sfail(s, SRMRA_ENOMEM, "host allocation failed");
  const int64_t l = q.L_high / q.K;
  try {
    r->y.assign(y, y + q.N * l * l);
    if (x0) r->x0.assign(x0, x0 + (int64_t)q.L_high * q.L_high);
  } catch (...) {
    delete r;
    return sfail(s, SRMRA_ENOMEM, "host allocation failed");
  }
  r->p = q;
  r->iters = iters;
  r->F = F;
  r->sigma_bm1 = sigma_bm1;
  r->decay = decay;
  r->bytes = bytes;
  r->t_submit = now_ms();
  std::lock_guard<std::mutex> lock(s->mu);
  r->id = s->next_id++;
  s->queue.push_back(r);
  s->all[r->id] = r;
  *request_id = r->id;
  return SRMRA_OK;
}

srmra_status srmra_server_step(srmra_server* s, int32_t* n_running, int32_t* n_queued,
                               int32_t* n_finished) {
  if (!s) return sfail(nullptr, SRMRA_EINVAL, "server is NULL");
  std::vector<Request*> admit;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    while (!s->queue.empty() &&
           (int)(s->running.size() + admit.size()) < s->max_active &&
           s->used + s->queue.front()->bytes <= s->budget) {
      Request* r = s->queue.front();
      s->queue.pop_front();
      s->used += r->bytes;
      admit.push_back(r);
    }
  }
  for (Request* r : admit) {
    r->t_admit = now_ms();
    srmra_status st = srmra_create(&r->p, r->y.data(), 0, r->x0.empty() ? nullptr : r->x0.data(),
                                   nullptr, nullptr, (void*)s->stream, &r->ctx);
    if (st == SRMRA_OK) st = srmra_set_schedule(r->ctx, r->F, r->sigma_bm1, r->decay);
    if (st != SRMRA_OK) {
      r->status = st;
      r->err = srmra_last_error(r->ctx);
      if (r->ctx) srmra_destroy(r->ctx);
      r->ctx = nullptr;
      r->state = 3;
      r->t_done = now_ms();
      s->used -= r->bytes;
      continue;
    }
    std::vector<float>().swap(r->y);  // the observations now live on the device
    r->state = 1;
    s->running.push_back(r);
    s->dirty[r->p.prec] = true;
  }
  int32_t finished = 0;
  if (!s->running.empty()) {
    // one batch per precision form among the running requests, advanced in turn
    for (int f = 0; f < 4; ++f) {
      std::vector<srmra_ctx*> ctxs;
      for (Request* r : s->running)
        if (r->p.prec == f) ctxs.push_back(r->ctx);
      if (ctxs.empty()) continue;
      if (s->dirty[f] || !s->batch[f]) {
        if (s->batch[f]) srmra_batch_destroy(s->batch[f]);
        s->batch[f] = nullptr;
        srmra_status st =
            srmra_batch_create(ctxs.data(), (int32_t)ctxs.size(), 0, &s->batch[f]);
        if (st != SRMRA_OK) return sfail(s, st, srmra_batch_last_error(nullptr));
        s->dirty[f] = false;
      }
      srmra_status st = srmra_batch_solve(s->batch[f], 1, -1, 0.0, 1.0, nullptr);
      if (st != SRMRA_OK) return sfail(s, st, srmra_batch_last_error(s->batch[f]));
    }
    ++s->iterations;
    std::vector<Request*> still;
    for (Request* r : s->running) {
      if (r->ctx->t >= r->iters) {
        s->dirty[r->p.prec] = true;
        retire(s, r);
        ++finished;
      } else {
        still.push_back(r);
      }
    }
    s->running.swap(still);
    for (int f = 0; f < 4; ++f) {
      bool any = false;
      for (Request* r : s->running) any = any || r->p.prec == f;
      if (!any && s->batch[f]) {
        srmra_batch_destroy(s->batch[f]);
        s->batch[f] = nullptr;
      }
    }
  }
  std::lock_guard<std::mutex> lock(s->mu);
  if (n_running) *n_running = (int32_t)s->running.size();
  if (n_queued) *n_queued = (int32_t)s->queue.size();
  if (n_finished) *n_finished = finished;
  return SRMRA_OK;
}

srmra_status srmra_server_result(srmra_server* s, int64_t id, int32_t* state, float* x,
                                 double* rho1, double* rho2, double* loglik_last,
                                 double* times_ms) {
  if (!s || !state) return sfail(s, SRMRA_EINVAL, "server and state are required");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return sfail(s, SRMRA_EINVAL, "unknown request id");
  Request* r = it->second;
  *state = r->state;
  if (r->state == 2) {
    const int L = r->p.L_high;
    if (x) std::copy(r->x.begin(), r->x.end(), x);
    if (rho1) std::copy(r->rho1.begin(), r->rho1.end(), rho1);
    if (rho2) std::copy(r->rho2.begin(), r->rho2.end(), rho2);
    if (loglik_last) *loglik_last = r->ll_last;
    (void)L;
  }
  if (times_ms) {  // submit -> admit (queueing), admit -> done (running), submit -> done
    times_ms[0] = r->t_admit > 0 ? r->t_admit - r->t_submit : -1.0;
    times_ms[1] = r->t_done > 0 && r->t_admit > 0 ? r->t_done - r->t_admit : -1.0;
    times_ms[2] = r->t_done > 0 ? r->t_done - r->t_submit : -1.0;
  }
  if (r->state == 3) return sfail(s, r->status, r->err.empty() ? "request failed" : r->err);
  return SRMRA_OK;
}

srmra_status srmra_server_memory(srmra_server* s, int64_t* used, int64_t* budget) {
  if (!s) return sfail(nullptr, SRMRA_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  if (used) *used = s->used;
  if (budget) *budget = s->budget;
  return SRMRA_OK;
}

void srmra_server_destroy(srmra_server* s) {
  if (!s) return;
  for (int f = 0; f < 4; ++f)
    if (s->batch[f]) srmra_batch_destroy(s->batch[f]);
  for (auto& kv : s->all) {
    if (kv.second->ctx) srmra_destroy(kv.second->ctx);
    delete kv.second;
  }
  delete s;
}

const char* srmra_server_last_error(const srmra_server* s) {
  return s ? s->err.c_str() : g_server_err.c_str();
}

}  // extern "C"
