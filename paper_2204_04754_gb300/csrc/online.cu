// Online (mini-batch) EM over shards of the observations (declared in include/srmra.h).
//
// The statistics are those the M-step of Eqs. (x_EM), (rho_EM) consumes, in the layout
// the finalize kernels use: cfin-like [c_s (Spad) | zb_s (Spad)] and b' per (sub-image
// r, low-resolution pixel m), all float64 per-observation averages.  A step runs the
// shard's E-step (both passes and the partial-sum kernels), folds the shard's sums into
// the running statistics with weight gamma, and runs the shared M-step kernels on them
// into the online estimate.
#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "srmra_internal.cuh"

using namespace srmra;

struct srmra_online {
  std::vector<srmra_ctx*> shards;
  cudaStream_t stream = nullptr;
  Geom g;
  float* x = nullptr;        // [L*L] estimate
  double* rho1 = nullptr;    // [L]
  double* rho2 = nullptr;    // [L]
  double* sfin = nullptr;    // [2 Spad] running c_s, zb_s (per-observation averages)
  double* sb = nullptr;      // [K*K*l2] running b' (per-observation average)
  float* b1 = nullptr;       // [K*K*l2] float copy of sb for the x kernel
  double* Ar = nullptr;      // [2 K*K] coverage and zb per sub-image
  double* ll = nullptr;      // [1] batch log-likelihood of the last step
  int* status = nullptr;
  int64_t steps = 0;
  std::string err;
};

namespace {

thread_local std::string g_online_err;

srmra_status ofail(srmra_online* on, srmra_status st, const std::string& msg) {
  if (on)
    on->err = msg;
  else
    g_online_err = msg;
  return st;
}

#define OCK(on, call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ofail((on), SRMRA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// S <- (1 - gamma) S + gamma / n * (shard sums); the shard's b' partials are summed in
// a fixed order (float64).
__global__ void k_online_update(const double* __restrict__ cfin, const float* __restrict__ bpart,
                                int n_ts, int S, int Spad, int KKl2, double gamma, double inv_n,
                                double* __restrict__ sfin, double* __restrict__ sb,
                                float* __restrict__ b1) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const double keep = 1.0 - gamma, add = gamma * inv_n;
  if (j < S) {
    sfin[j] = keep * sfin[j] + add * cfin[j];
    sfin[Spad + j] = keep * sfin[Spad + j] + add * cfin[Spad + j];
  }
  if (j < KKl2) {
    double b = 0.0;
    for (int t = 0; t < n_ts; ++t) b += (double)bpart[(int64_t)t * KKl2 + j];
    const double v = keep * sb[j] + add * b;
    sb[j] = v;
    b1[j] = (float)v;
  }
}

}  // namespace

extern "C" {

srmra_status srmra_online_create(srmra_ctx* const* shards, int32_t n_shards, const float* x0,
                                 const double* rho1_0, const double* rho2_0,
                                 srmra_online** out) {
  if (!out) return ofail(nullptr, SRMRA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!shards || n_shards < 1) return ofail(nullptr, SRMRA_EINVAL, "need at least one shard");
  const srmra_ctx* c0 = shards[0];
  if (!c0) return ofail(nullptr, SRMRA_EINVAL, "NULL shard");
  for (int k = 0; k < n_shards; ++k) {
    const srmra_ctx* c = shards[k];
    if (!c) return ofail(nullptr, SRMRA_EINVAL, "NULL shard");
    for (int j = 0; j < k; ++j)
      if (shards[j] == c) return ofail(nullptr, SRMRA_EINVAL, "shard listed twice");
    if (c->g.L != c0->g.L || c->g.K != c0->g.K || c->g.sigma != c0->g.sigma ||
        c->prec != c0->prec || c->stream != c0->stream || c->device != c0->device)
      return ofail(nullptr, SRMRA_EINVAL,
                   "shards need the same L, K, sigma, precision, stream and device");
  }
  for (const double* r : {rho1_0, rho2_0}) {
    if (!r) continue;
    double s = 0.0;
    for (int k = 0; k < c0->g.L; ++k) {
      if (!(r[k] >= 0.0) || !std::isfinite(r[k]))
        return ofail(nullptr, SRMRA_EINVAL, "rho has a negative or non-finite entry");
      s += r[k];
    }
    if (!(s > 0.0)) return ofail(nullptr, SRMRA_EINVAL, "rho sums to zero");
  }
  auto* on = new (std::nothrow) srmra_online();
  if (!on) return ofail(nullptr, SRMRA_ENOMEM, "host allocation failed");
  on->shards.assign(shards, shards + n_shards);
  on->stream = c0->stream;
  on->g = c0->g;
  const Geom& g = on->g;
  const int KKl2 = g.K * g.K * g.l2;
  std::vector<void*> got;
  auto get = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes, on->stream);
    return e;
  };
  cudaError_t e = get((void**)&on->x, sizeof(float) * g.S);
  if (e == cudaSuccess) e = get((void**)&on->rho1, sizeof(double) * g.L);
  if (e == cudaSuccess) e = get((void**)&on->rho2, sizeof(double) * g.L);
  if (e == cudaSuccess) e = get((void**)&on->sfin, sizeof(double) * 2 * g.Spad);
  if (e == cudaSuccess) e = get((void**)&on->sb, sizeof(double) * KKl2);
  if (e == cudaSuccess) e = get((void**)&on->b1, sizeof(float) * KKl2);
  if (e == cudaSuccess) e = get((void**)&on->Ar, sizeof(double) * 2 * g.K * g.K);
  if (e == cudaSuccess) e = get((void**)&on->ll, sizeof(double));
  if (e == cudaSuccess) e = get((void**)&on->status, sizeof(int));
  // the starting estimate: the given one, else shard 0's
  auto put = [&](void* dst, const void* host, const void* dev, size_t bytes) {
    if (e != cudaSuccess) return;
    e = host ? cudaMemcpyAsync(dst, host, bytes, cudaMemcpyHostToDevice, on->stream)
             : cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToDevice, on->stream);
  };
  std::vector<double> r1n, r2n;
  auto normalised = [&](const double* r, std::vector<double>& v) -> const double* {
    if (!r) return nullptr;
    double s = 0.0;
    for (int k = 0; k < g.L; ++k) s += r[k];
    v.resize(g.L);
    for (int k = 0; k < g.L; ++k) v[k] = r[k] / s;
    return v.data();
  };
  put(on->x, x0, c0->x, sizeof(float) * g.S);
  put(on->rho1, normalised(rho1_0, r1n), c0->rho1, sizeof(double) * g.L);
  put(on->rho2, normalised(rho2_0, r2n), c0->rho2, sizeof(double) * g.L);
  if (e == cudaSuccess) e = cudaStreamSynchronize(on->stream);
  if (e != cudaSuccess) {
    srmra_online_destroy(on);
    return ofail(nullptr, SRMRA_ECUDA, std::string("online state: ") + cudaGetErrorString(e));
  }
  *out = on;
  return SRMRA_OK;
}

srmra_status srmra_online_step(srmra_online* on, int32_t shard, double gamma,
                               double* loglik_out) {
  if (!on) return ofail(nullptr, SRMRA_EINVAL, "online is NULL");
  if (shard < 0 || shard >= (int32_t)on->shards.size())
    return ofail(on, SRMRA_EINVAL, "shard index out of range");
  if (!(gamma > 0.0 && gamma <= 1.0)) return ofail(on, SRMRA_EINVAL, "need 0 < gamma <= 1");
  srmra_ctx* c = on->shards[shard];
  const Geom& g = on->g;
  const cudaStream_t st = on->stream;
  // theta into the shard, its E-step, the shard's sums into S, the M-step on S
  OCK(on, cudaMemcpyAsync(c->x, on->x, sizeof(float) * g.S, cudaMemcpyDeviceToDevice, st));
  OCK(on, cudaMemcpyAsync(c->rho1, on->rho1, sizeof(double) * g.L, cudaMemcpyDeviceToDevice, st));
  OCK(on, cudaMemcpyAsync(c->rho2, on->rho2, sizeof(double) * g.L, cudaMemcpyDeviceToDevice, st));
  srmra_status s = run_estep_stats(c);
  if (s != SRMRA_OK) return ofail(on, s, srmra_last_error(c));
  const double gm = on->steps == 0 ? 1.0 : gamma;
  const int KKl2 = g.K * g.K * g.l2;
  const int n = std::max(g.Spad, KKl2);
  k_online_update<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(
      c->cfin, c->bpart, stats_t_splits(c), g.S, g.Spad, KKl2, gm, 1.0 / (double)c->g.N,
      on->sfin, on->sb, on->b1);
  c->launches++;
  launch_mstep(c, on->sfin, on->b1, 1, c->llpart, c->plan.ll_blocks, on->rho1, on->rho2, on->Ar,
               on->ll, on->x, on->status, st);
  OCK(on, cudaGetLastError());
  on->steps += 1;
  if (loglik_out) {
    int status = 0;
    OCK(on, cudaMemcpyAsync(loglik_out, on->ll, sizeof(double), cudaMemcpyDeviceToHost, st));
    OCK(on, cudaMemcpyAsync(&status, on->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    OCK(on, cudaStreamSynchronize(st));
    if (status & STATUS_NUMERIC)
      return ofail(on, SRMRA_ENUMERIC, "NaN or Inf in the log-likelihood, x or rho");
    if (status) return ofail(on, SRMRA_ETIMEOUT, "a bounded device wait timed out");
  }
  return SRMRA_OK;
}

srmra_status srmra_online_project(srmra_online* on, double sigma_bm) {
  if (!on) return ofail(nullptr, SRMRA_EINVAL, "online is NULL");
  srmra_ctx* c = on->shards[0];
  const Geom& g = on->g;
  OCK(on, cudaMemcpyAsync(c->x, on->x, sizeof(float) * g.S, cudaMemcpyDeviceToDevice, on->stream));
  srmra_status s = srmra_project(c, sigma_bm, nullptr, nullptr);
  if (s != SRMRA_OK) return ofail(on, s, srmra_last_error(c));
  OCK(on, cudaMemcpyAsync(on->x, c->x, sizeof(float) * g.S, cudaMemcpyDeviceToDevice, on->stream));
  return SRMRA_OK;
}

srmra_status srmra_online_get_state(srmra_online* on, float* x, double* rho1, double* rho2,
                                    int64_t* steps_done) {
  if (!on) return ofail(nullptr, SRMRA_EINVAL, "online is NULL");
  const Geom& g = on->g;
  if (x) OCK(on, cudaMemcpyAsync(x, on->x, sizeof(float) * g.S, cudaMemcpyDeviceToHost, on->stream));
  if (rho1)
    OCK(on, cudaMemcpyAsync(rho1, on->rho1, sizeof(double) * g.L, cudaMemcpyDeviceToHost, on->stream));
  if (rho2)
    OCK(on, cudaMemcpyAsync(rho2, on->rho2, sizeof(double) * g.L, cudaMemcpyDeviceToHost, on->stream));
  OCK(on, cudaStreamSynchronize(on->stream));
  if (steps_done) *steps_done = on->steps;
  return SRMRA_OK;
}

void srmra_online_destroy(srmra_online* on) {
  if (!on) return;
  cudaStreamSynchronize(on->stream);
  for (void* p : {(void*)on->x, (void*)on->rho1, (void*)on->rho2, (void*)on->sfin, (void*)on->sb,
                  (void*)on->b1, (void*)on->Ar, (void*)on->ll, (void*)on->status})
    if (p) cudaFree(p);
  delete on;
}

const char* srmra_online_last_error(const srmra_online* on) {
  return on ? on->err.c_str() : g_online_err.c_str();
}

}  // extern "C"
