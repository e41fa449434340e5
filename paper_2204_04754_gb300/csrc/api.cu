// Host driver and C ABI of libsrmra (declared in include/srmra.h).
//
// One EM iteration (Sec. 2) is enqueued as:
//   prep      sub-image statistics, logit column terms, centred templates
//   pass 1    logits + online log-sum-exp partials              (Eq. weights_EM)
//   combine   lse per observation, float64 log-likelihood       (Eq. likelihood_EM)
//   pass 2    recomputed weights -> M-step partial sums         (Eqs. x_EM, rho_EM)
//   finalize  rho (marginals of the joint update), coverage, x = b / A
// and Algorithm 2 adds the denoiser x <- D(x, sigma_BM) after every F iterations with
// sigma_BM decayed by Eq. (decaying_function).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "srmra_internal.cuh"

using namespace srmra;

namespace {

thread_local std::string g_create_err;

srmra_status fail(srmra_ctx* c, srmra_status st, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_err = msg;
  return st;
}

srmra_status cuda_fail(srmra_ctx* c, cudaError_t e, const char* what) {
  const srmra_status st =
      (e == cudaErrorMemoryAllocation) ? SRMRA_ENOMEM : SRMRA_ECUDA;
  return fail(c, st, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(c, call)                                            \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail((c), e_, #call);   \
  } while (0)

// Allocation cap used by the failure-injection tests (SRMRA_ALLOC_LIMIT_BYTES).
int64_t alloc_limit() {
  const char* s = std::getenv("SRMRA_ALLOC_LIMIT_BYTES");
  return s ? std::atoll(s) : -1;
}

struct Allocator {
  srmra_ctx* c;
  int64_t used = 0;
  int64_t limit = alloc_limit();
  std::vector<void*>* owned;
  bool dry = false;  // count bytes only (admission estimates)
  template <typename T>
  cudaError_t get(T** p, int64_t count) {
    const int64_t bytes = count * (int64_t)sizeof(T);
    if (dry) {
      used += round_up(bytes, 256);
      *p = nullptr;
      return cudaSuccess;
    }
    if (limit >= 0 && used + bytes > limit) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc((void**)p, (size_t)bytes);
    if (e != cudaSuccess) return e;
    owned->push_back(*p);
    used += bytes;
    return cudaMemsetAsync(*p, 0, (size_t)bytes, c->stream);
  }
};

srmra_status check_rho(srmra_ctx* c, const double* r, int L, std::vector<double>& out) {
  out.assign(L, 1.0 / L);
  if (!r) return SRMRA_OK;
  double s = 0.0;
  for (int k = 0; k < L; ++k) {
    if (!(r[k] >= 0.0) || !std::isfinite(r[k]))
      return fail(c, SRMRA_EINVAL, "rho has a negative or non-finite entry");
    s += r[k];
  }
  if (std::fabs(s - 1.0) > 1e-6) return fail(c, SRMRA_EINVAL, "rho does not sum to 1");
  for (int k = 0; k < L; ++k) out[k] = r[k] / s;
  return SRMRA_OK;
}

srmra_status read_status(srmra_ctx* c) {
  int st = 0;
  CK(c, cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (st) {
    CK(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    if (st & STATUS_TIMEOUT) return fail(c, SRMRA_ETIMEOUT, "a bounded device wait timed out");
    if (st & STATUS_NUMERIC) return fail(c, SRMRA_ENUMERIC, "NaN/Inf in log-likelihood, x or rho");
  }
  return SRMRA_OK;
}

cudaEvent_t take_event(srmra_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t ev = c->event_pool.back();
    c->event_pool.pop_back();
    return ev;
  }
  cudaEvent_t ev = nullptr;
  cudaEventCreate(&ev);
  return ev;
}

// Records an event pair around one phase when profiling is on.
struct PhaseTimer {
  srmra_ctx* c;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseTimer(srmra_ctx* c_, int p) : c(c_), phase(p) {
    if (c->profiling) {
      a = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~PhaseTimer() {
    if (a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, c->stream);
      c->marks.push_back({phase, a, b});
    }
  }
};

// The E-step of theta_t over the context's observations, up to the sums the M-step
// needs (launch_stats); shared by the EM iteration and the online step.
srmra_status run_estep_passes(srmra_ctx* c) {
  cudaError_t e = cudaSuccess;
  { PhaseTimer t(c, SRMRA_PHASE_PREP); launch_prep_iter(c); }
  const bool tc = is_tc_prec(c->prec), fft = c->prec == SRMRA_FFT32;
  {
    PhaseTimer t(c, SRMRA_PHASE_PASS1);
    if (tc)
      e = launch_pass1_tc(c);
    else if (fft)
      launch_pass1_fft(c);
    else
      launch_pass1_f32(c);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "pass 1 launch");
  { PhaseTimer t(c, SRMRA_PHASE_COMBINE); launch_lse_combine(c, c->plan.p1_groups); }
  {
    PhaseTimer t(c, SRMRA_PHASE_PASS2);
    e = tc ? launch_pass2_tc(c) : fft ? launch_pass2_fft(c) : launch_pass2_f32(c);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "pass 2 launch");
  return SRMRA_OK;
}

}  // namespace

srmra_status srmra::run_estep_stats(srmra_ctx* c) {
  srmra_status st = run_estep_passes(c);
  if (st != SRMRA_OK) return st;
  { PhaseTimer t(c, SRMRA_PHASE_FINAL); launch_stats(c); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "E-step launch");
  c->have_estep = true;
  return SRMRA_OK;
}

namespace {

// One EM iteration theta_t -> theta_{t+1}; LL(theta_t) goes to ll_hist[ll_index].
srmra_status run_iteration(srmra_ctx* c, int ll_index) {
  srmra_status st = run_estep_passes(c);
  if (st != SRMRA_OK) return st;
  { PhaseTimer t(c, SRMRA_PHASE_FINAL); launch_finalize(c, ll_index); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "EM iteration launch");
  c->t += 1;
  c->have_estep = true;
  return SRMRA_OK;
}

srmra_status ensure_ll(srmra_ctx* c, int n) {
  if (n <= c->ll_cap) return SRMRA_OK;
  double* p = nullptr;
  CK(c, cudaMalloc((void**)&p, sizeof(double) * (size_t)n));
  if (c->ll_hist) {
    CK(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->ll_hist);
  }
  c->ll_hist = p;
  c->ll_cap = n;
  return SRMRA_OK;
}

// Geometry and work plan of a context; caps receives the partial-buffer capacities
// (pass-1 groups, Z' slices, c/zb slices) the buffers are sized for.
void setup_ctx(srmra_ctx* c, const srmra_params* p, int num_sms, int caps[3]) {
  c->num_sms = num_sms;
  c->prec = p->prec;
  c->flags = p->flags;
  c->no_cluster = (p->flags & SRMRA_FLAG_NO_CLUSTER) != 0;
  Geom& g = c->g;
  g.L = p->L_high;
  g.K = p->K;
  g.l = g.L / g.K;
  g.l2 = g.l * g.l;
  g.S = g.L * g.L;
  g.Spad = (int)round_up(g.S, SPAD);
  g.ldy = (int)round_up(g.l2, 16);
  g.ldk = (int)round_up(g.l2, 64);
  g.N = p->N;
  g.Npad = round_up(g.N, NPAD);
  g.sigma = p->sigma;
  if (c->prec == SRMRA_FFT32) {
    plan_fft(c);
    caps[0] = c->plan.p1_groups;
    caps[1] = 0;
    caps[2] = c->plan.nparts_c;
  } else if (is_tc_prec(c->prec)) {
    c->plan.p2_comp = tc_comp_mstep(g, c->prec, c->flags);
    c->plan.p2_pair = tc_pair_form(g, c->prec, c->flags, c->plan.p2_comp);
    if (c->flags & SRMRA_FLAG_P1_TILE128) c->plan.p1_bn = 128;
    // size the partial buffers for the finest decomposition the batch tuner may pick
    plan_tc(c, 2, 2);
    c->plan.cap_p1_groups = c->plan.p1_groups;
    c->plan.cap_nsplit = c->plan.p2_nsplit;
    caps[0] = c->plan.p1_groups;
    caps[1] = c->plan.nparts_z;
    caps[2] = c->plan.nparts_c;
    plan_tc(c, 1, 1);
  } else {
    plan_simt(c);
    caps[0] = c->plan.p1_groups;
    caps[1] = c->plan.nparts_z;
    caps[2] = c->plan.nparts_c;
  }
}

// Every device buffer of a context (or, with A.dry, just their total size).
cudaError_t allocate_buffers(srmra_ctx* c, Allocator& A, const int caps[3], const char** what) {
  const Geom& g = c->g;
  const Plan& pl = c->plan;
  const bool tc = is_tc_prec(c->prec);
#define AL(ptr, count)                                   \
  do {                                                   \
    cudaError_t e2 = A.get(&(ptr), (int64_t)(count));    \
    if (e2 != cudaSuccess) {                             \
      *what = "allocate " #ptr;                          \
      return e2;                                         \
    }                                                    \
  } while (0)
  AL(c->Yc, g.Npad * g.ldy);
  if (tc) {
    AL(c->Yh, g.Npad * g.ldk);
    AL(c->YTf, g.Npad * g.l2);
    if (pl.p2_comp) AL(c->YTfl, g.Npad * g.l2);
    AL(c->Ah, (int64_t)g.Spad * g.ldk);
    AL(c->d_ustart, 4);
    {
      unsigned char* di = nullptr;
      AL(di, (int64_t)tc_inst_bytes());
      c->d_inst = di;
    }
    if (c->prec == SRMRA_BF16X3) {
      AL(c->Yl, g.Npad * g.ldk);
      AL(c->Al, (int64_t)g.Spad * g.ldk);
    }
  } else if (c->prec == SRMRA_FFT32) {
    AL(c->Yf, g.Npad * g.l2);
    AL(c->Xf, (int64_t)g.K * g.K * g.l2);
    AL(c->Gp, (int64_t)pl.fft_blocks * g.K * g.K * g.l2);
  } else {
    AL(c->YcT, g.Npad * g.ldy);
    AL(c->AxT, (int64_t)g.ldy * g.Spad);
  }
  AL(c->ybar, g.Npad);
  AL(c->yy, g.Npad);
  AL(c->x, g.S);
  AL(c->rho1, g.L);
  AL(c->rho2, g.L);
  AL(c->sub, 2 * g.K * g.K);
  AL(c->colb, g.Spad);
  AL(c->colm, g.Spad);
  AL(c->pm, (int64_t)caps[0] * g.Npad);
  AL(c->ps, (int64_t)caps[0] * g.Npad);
  AL(c->lse2, g.Npad);
  AL(c->lse, g.Npad);
  AL(c->llpart, pl.ll_blocks);
  if (caps[1] > 0) AL(c->Zp, (int64_t)caps[1] * g.Spad * g.ldy);
  AL(c->cp, (int64_t)caps[2] * g.Spad);
  AL(c->zbp, (int64_t)caps[2] * g.Spad);
  AL(c->cfin, 2 * (int64_t)g.Spad);
  AL(c->bpart, (int64_t)fin_t_splits(g, c->num_sms) * g.S);
  AL(c->Ar, 2 * g.K * g.K);
  AL(c->dstats, 3 * (int64_t)g.S + 1);
  AL(c->status, 1);
  AL(c->d_sched, 1);
#undef AL
  return cudaSuccess;
}

}  // namespace

// Mean-upsampled initial guess x0[q] = mean_i y_i[q1 / K, q2 / K] (nearest neighbour).
__global__ void k_mean_upsample(const float* __restrict__ Yc, const float* __restrict__ ybar,
                                int64_t N, int ldy, int L, int K, int l,
                                float* __restrict__ x) {
  __shared__ double red[256];
  const int n = blockIdx.x;  // low-resolution pixel
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += 256) s += (double)Yc[i * ldy + n] + (double)ybar[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const float v = (float)(red[0] / (double)N);
  const int n1 = n / l, n2 = n % l;
  for (int k = threadIdx.x; k < K * K; k += 256)
    x[(n1 * K + k / K) * L + n2 * K + k % K] = v;
}

extern "C" {

const char* srmra_version(void) { return "srmra 0.1 (sm_103a)"; }

const char* srmra_last_error(const srmra_ctx* c) {
  return c ? c->err.c_str() : g_create_err.c_str();
}

srmra_status srmra_create(const srmra_params* p, const float* y, int32_t y_is_device,
                          const float* x0, const double* rho1_0, const double* rho2_0,
                          void* cuda_stream, srmra_ctx** out) {
  if (!out) return fail(nullptr, SRMRA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!p || !y) return fail(nullptr, SRMRA_EINVAL, "params or y is NULL");
  if (p->L_high < 2 || p->K < 1 || p->L_high % p->K != 0)
    return fail(nullptr, SRMRA_EINVAL, "need L >= 2, K >= 1 and K dividing L");
  if (p->N < 1) return fail(nullptr, SRMRA_EINVAL, "need N >= 1");
  if (!(p->sigma > 0.0) || !std::isfinite(p->sigma))
    return fail(nullptr, SRMRA_EINVAL, "need sigma > 0");
  if (p->prec != SRMRA_FP32 && p->prec != SRMRA_BF16 && p->prec != SRMRA_BF16X3 &&
      p->prec != SRMRA_FFT32)
    return fail(nullptr, SRMRA_EINVAL, "unknown precision form");
  if (p->prec == SRMRA_FFT32 && !fft_supported(p->L_high / p->K))
    return fail(nullptr, SRMRA_EINVAL, "the FFT form needs l = L/K in {8, 16, 32}");

  std::vector<double> r1, r2;
  {
    srmra_status st = check_rho(nullptr, rho1_0, p->L_high, r1);
    if (st == SRMRA_OK) st = check_rho(nullptr, rho2_0, p->L_high, r2);
    if (st != SRMRA_OK) return st;
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceProperties");
  if (prop.major * 10 + prop.minor != 103)
    return fail(nullptr, SRMRA_ECUDA, "libsrmra is built for sm_103a (GB300) only");

  srmra_ctx* c = new (std::nothrow) srmra_ctx();
  if (!c) return fail(nullptr, SRMRA_ENOMEM, "host allocation failed");
  c->device = dev;
  c->stream = (cudaStream_t)cuda_stream;
  int caps[3];
  setup_ctx(c, p, prop.multiProcessorCount, caps);
  const Geom& g = c->g;
  const bool tc = is_tc_prec(c->prec);
  Allocator A{c, 0, alloc_limit(), &c->owned};
  const char* what = nullptr;
  e = allocate_buffers(c, A, caps, &what);
  if (e != cudaSuccess) {
    srmra_status s2 = cuda_fail(nullptr, e, what);
    srmra_destroy(c);
    return s2;
  }
  c->device_bytes = A.used;
  auto bail = [&](cudaError_t err, const char* w) {
    srmra_status s2 = cuda_fail(nullptr, err, w);
    srmra_destroy(c);
    return s2;
  };
  float* ytmp = nullptr;
  if (!y_is_device) {
    e = cudaMalloc((void**)&ytmp, sizeof(float) * (size_t)(g.N * g.l2));
    if (e != cudaSuccess) return bail(e, "allocate upload buffer");
    e = cudaMemcpyAsync(ytmp, y, sizeof(float) * (size_t)(g.N * g.l2), cudaMemcpyHostToDevice,
                        c->stream);
    if (e != cudaSuccess) {
      cudaFree(ytmp);
      return bail(e, "upload y");
    }
  }
  launch_center_obs(c, y_is_device ? y : ytmp);
  if (tc || c->prec == SRMRA_FFT32) {
    e = tc ? prep_obs_tc(c) : prep_obs_fft(c);
    if (e != cudaSuccess) {
      if (ytmp) cudaFree(ytmp);
      return bail(e, tc ? "prepare tensor-core operands" : "transform the observations");
    }
  }
  if (x0) {
    e = cudaMemcpyAsync(c->x, x0, sizeof(float) * (size_t)g.S, cudaMemcpyHostToDevice,
                        c->stream);
  } else {
    k_mean_upsample<<<g.l2, 256, 0, c->stream>>>(c->Yc, c->ybar, g.N, g.ldy, g.L, g.K, g.l,
                                                  c->x);
    c->launches++;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->rho1, r1.data(), sizeof(double) * g.L, cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->rho2, r2.data(), sizeof(double) * g.L, cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (ytmp) cudaFree(ytmp);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return bail(e, "initialise context");
  if (ensure_ll(c, 64) != SRMRA_OK) {
    g_create_err = c->err;
    srmra_destroy(c);
    return SRMRA_ENOMEM;
  }
  *out = c;
  return SRMRA_OK;
}

srmra_status srmra_em_iter(srmra_ctx* c, int32_t n_iters, double* loglik_out) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  if (n_iters < 0) return fail(c, SRMRA_EINVAL, "n_iters < 0");
  srmra_status st = ensure_ll(c, n_iters > 0 ? n_iters : 1);
  if (st != SRMRA_OK) return st;
  for (int k = 0; k < n_iters; ++k) {
    st = run_iteration(c, k);
    if (st != SRMRA_OK) return st;
  }
  if (loglik_out && n_iters > 0) {
    CK(c, cudaMemcpyAsync(loglik_out, c->ll_hist, sizeof(double) * n_iters,
                          cudaMemcpyDeviceToHost, c->stream));
    return read_status(c);
  }
  if (c->flags & SRMRA_FLAG_CHECK_NUMERIC) return read_status(c);
  return SRMRA_OK;
}

srmra_status srmra_stats_length(const srmra_ctx* c, int64_t* len) {
  if (!c || !len) return fail(nullptr, SRMRA_EINVAL, "ctx or len is NULL");
  *len = 3 * (int64_t)c->g.S + 1;
  return SRMRA_OK;
}

srmra_status srmra_estep_stats(srmra_ctx* c, double* stats, int32_t stats_is_device) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  if (!stats) return fail(c, SRMRA_EINVAL, "stats is NULL");
  srmra_status st = run_estep_stats(c);
  if (st != SRMRA_OK) return st;
  launch_pack_stats(c, stats_is_device ? stats : c->dstats);
  CK(c, cudaGetLastError());
  if (stats_is_device) return SRMRA_OK;
  CK(c, cudaMemcpyAsync(stats, c->dstats, sizeof(double) * (3 * (size_t)c->g.S + 1),
                        cudaMemcpyDeviceToHost, c->stream));
  return read_status(c);
}

srmra_status srmra_mstep_stats(srmra_ctx* c, const double* stats, int32_t stats_is_device,
                               double* loglik_out) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  if (!stats) return fail(c, SRMRA_EINVAL, "stats is NULL");
  srmra_status st = ensure_ll(c, 1);
  if (st != SRMRA_OK) return st;
  if (!stats_is_device)
    CK(c, cudaMemcpyAsync(c->dstats, stats, sizeof(double) * (3 * (size_t)c->g.S + 1),
                          cudaMemcpyHostToDevice, c->stream));
  launch_unpack_stats(c, stats_is_device ? stats : c->dstats);
  launch_mstep(c, c->cfin, c->bpart, 1, c->llpart, 1, c->rho1, c->rho2, c->Ar, c->ll_hist, c->x,
               c->status, c->stream);
  CK(c, cudaGetLastError());
  c->t += 1;
  // Algorithm 2 on the context's own schedule (srmra_set_schedule): the projection after
  // every F-th M-step, then sigma_BM <- decay sigma_BM (Eq. decaying_function)
  if (c->sched_F > 0 && c->t % c->sched_F == 0) {
    PhaseTimer tm(c, SRMRA_PHASE_DENOISE);
    launch_dct_denoise(c, c->sigma_bm, c->dn_thr);
    c->sigma_bm *= c->sched_decay;
    CK(c, cudaGetLastError());
  }
  if (loglik_out) {
    CK(c, cudaMemcpyAsync(loglik_out, c->ll_hist, sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
    return read_status(c);
  }
  if (c->flags & SRMRA_FLAG_CHECK_NUMERIC) return read_status(c);
  return SRMRA_OK;
}

srmra_status srmra_project(srmra_ctx* c, double sigma_bm, srmra_denoiser_fn fn, void* user) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  if (!(sigma_bm >= 0.0)) return fail(c, SRMRA_EINVAL, "sigma_bm < 0");
  if (fn) {
    if (fn(c->x, c->g.L, sigma_bm, (void*)c->stream, user) != 0)
      return fail(c, SRMRA_EINVAL, "denoiser callback failed");
  } else {
    if (c->g.L % 8 != 0) return fail(c, SRMRA_EINVAL, "built-in denoiser needs L % 8 == 0");
    PhaseTimer t(c, SRMRA_PHASE_DENOISE);
    launch_dct_denoise(c, sigma_bm, 2.7);
  }
  CK(c, cudaGetLastError());
  return SRMRA_OK;
}

srmra_status srmra_solve(srmra_ctx* c, int32_t iters, int32_t F, double sigma_bm1,
                         double decay, srmra_denoiser_fn fn, void* user, double* loglik_out) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  if (iters < 0 || F < 0 || !(decay > 0.0))
    return fail(c, SRMRA_EINVAL, "need iters >= 0, F >= 0, decay > 0");
  if (F > 0 && !fn && c->g.L % 8 != 0)
    return fail(c, SRMRA_EINVAL, "built-in denoiser needs L % 8 == 0");
  srmra_status st = ensure_ll(c, iters > 0 ? iters : 1);
  if (st != SRMRA_OK) return st;
  if (sigma_bm1 > 0.0) c->sigma_bm = sigma_bm1;
  for (int k = 0; k < iters; ++k) {
    st = run_iteration(c, k);
    if (st != SRMRA_OK) return st;
    if (F > 0 && c->t % F == 0) {
      st = srmra_project(c, c->sigma_bm, fn, user);
      if (st != SRMRA_OK) return st;
      c->sigma_bm *= decay;
    }
  }
  if (loglik_out && iters > 0) {
    CK(c, cudaMemcpyAsync(loglik_out, c->ll_hist, sizeof(double) * iters,
                          cudaMemcpyDeviceToHost, c->stream));
    return read_status(c);
  }
  if (c->flags & SRMRA_FLAG_CHECK_NUMERIC) return read_status(c);
  return SRMRA_OK;
}

srmra_status srmra_get_state(srmra_ctx* c, float* x, double* rho1, double* rho2,
                             double* sigma_bm, int32_t* t) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  const Geom& g = c->g;
  if (x) CK(c, cudaMemcpyAsync(x, c->x, sizeof(float) * g.S, cudaMemcpyDeviceToHost, c->stream));
  if (rho1)
    CK(c, cudaMemcpyAsync(rho1, c->rho1, sizeof(double) * g.L, cudaMemcpyDeviceToHost, c->stream));
  if (rho2)
    CK(c, cudaMemcpyAsync(rho2, c->rho2, sizeof(double) * g.L, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (sigma_bm) *sigma_bm = c->sigma_bm;
  if (t) *t = c->t;
  return SRMRA_OK;
}

srmra_status srmra_set_state(srmra_ctx* c, const float* x, const double* rho1,
                             const double* rho2, double sigma_bm, int32_t t) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  if (!x || !rho1 || !rho2) return fail(c, SRMRA_EINVAL, "x, rho1 and rho2 are required");
  std::vector<double> r1, r2;
  srmra_status st = check_rho(c, rho1, c->g.L, r1);
  if (st == SRMRA_OK) st = check_rho(c, rho2, c->g.L, r2);
  if (st != SRMRA_OK) return st;
  const Geom& g = c->g;
  CK(c, cudaMemcpyAsync(c->x, x, sizeof(float) * g.S, cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(c->rho1, r1.data(), sizeof(double) * g.L, cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(c->rho2, r2.data(), sizeof(double) * g.L, cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->sigma_bm = sigma_bm;
  c->t = t;
  return SRMRA_OK;
}

srmra_status srmra_get_estep(srmra_ctx* c, double* lse, double* cs) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  if (!c->have_estep) return fail(c, SRMRA_EINVAL, "no E-step has run yet");
  if (lse)
    CK(c, cudaMemcpyAsync(lse, c->lse, sizeof(double) * (size_t)c->g.N, cudaMemcpyDeviceToHost,
                          c->stream));
  if (cs)
    CK(c, cudaMemcpyAsync(cs, c->cfin, sizeof(double) * (size_t)c->g.S, cudaMemcpyDeviceToHost,
                          c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return SRMRA_OK;
}

srmra_status srmra_estimate_device_bytes(const srmra_params* p, int64_t* bytes) {
  if (!p || !bytes) return fail(nullptr, SRMRA_EINVAL, "params or bytes is NULL");
  if (p->L_high < 2 || p->K < 1 || p->L_high % p->K != 0 || p->N < 1 ||
      (p->prec != SRMRA_FP32 && p->prec != SRMRA_BF16 && p->prec != SRMRA_BF16X3 &&
       p->prec != SRMRA_FFT32) ||
      (p->prec == SRMRA_FFT32 && !fft_supported(p->L_high / p->K)))
    return fail(nullptr, SRMRA_EINVAL, "invalid problem parameters");
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  srmra_ctx c;
  int caps[3];
  setup_ctx(&c, p, sms, caps);
  Allocator A{&c, 0, -1, &c.owned};
  A.dry = true;
  const char* what = nullptr;
  allocate_buffers(&c, A, caps, &what);
  *bytes = A.used + 64 * (int64_t)sizeof(double);  // + the log-likelihood history
  return SRMRA_OK;
}

srmra_status srmra_device_bytes(const srmra_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return fail(nullptr, SRMRA_EINVAL, "ctx or bytes is NULL");
  *bytes = c->device_bytes + (int64_t)c->ll_cap * (int64_t)sizeof(double);
  return SRMRA_OK;
}

srmra_status srmra_set_schedule(srmra_ctx* c, int32_t F, double sigma_bm, double decay) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  if (F < 0 || !(decay > 0.0) || !(sigma_bm >= 0.0))
    return fail(c, SRMRA_EINVAL, "need F >= 0, sigma_bm >= 0, decay > 0");
  if (F > 0 && c->g.L % 8 != 0)
    return fail(c, SRMRA_EINVAL, "built-in denoiser needs L % 8 == 0");
  c->sched_F = F;
  c->sigma_bm = sigma_bm;
  c->sched_decay = decay;
  return SRMRA_OK;
}

srmra_status srmra_set_denoiser(srmra_ctx* c, int32_t mode, double threshold, int32_t spin) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  if ((mode != SRMRA_DENOISE_HARD && mode != SRMRA_DENOISE_SOFT) || !(threshold >= 0.0))
    return fail(c, SRMRA_EINVAL, "unknown denoiser mode or negative threshold");
  if (spin && !c->dn_acc) {
    cudaError_t e = cudaMalloc((void**)&c->dn_acc, sizeof(double) * 64 * (size_t)c->g.S);
    if (e != cudaSuccess) return cuda_fail(c, e, "allocate cycle-spinning buffer");
    c->owned.push_back(c->dn_acc);
    c->device_bytes += (int64_t)sizeof(double) * 64 * c->g.S;
  }
  c->dn_mode = mode;
  c->dn_thr = threshold;
  c->dn_spin = spin != 0;
  return SRMRA_OK;
}

srmra_status srmra_launch_count(const srmra_ctx* c, int64_t* count) {
  if (!c || !count) return fail(nullptr, SRMRA_EINVAL, "ctx or count is NULL");
  *count = c->launches;
  return SRMRA_OK;
}

srmra_status srmra_set_wait_limit(srmra_ctx* c, int64_t limit_ns, int32_t test_hook) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  if (limit_ns < 1000 || limit_ns > 60000000000ll)
    return fail(c, SRMRA_EINVAL, "need 1e3 <= limit_ns <= 6e10");
  if (test_hook < 0 || test_hook > 2) return fail(c, SRMRA_EINVAL, "test_hook must be 0, 1 or 2");
  c->wait_ns = (uint64_t)limit_ns;
  c->test_hook = test_hook;
  if (is_tc_prec(c->prec)) CK(c, tc_upload_inst(c));
  return SRMRA_OK;
}

srmra_status srmra_get_plan(const srmra_ctx* c, int32_t* out, int32_t n) {
  if (!c || !out || n < 0) return fail(nullptr, SRMRA_EINVAL, "ctx or out is NULL");
  const Plan& p = c->plan;
  int form = SRMRA_P2_FP32;
  if (is_tc_prec(c->prec))
    form = p.p2_comp   ? SRMRA_P2_PER_CHUNK_COMP
           : p.p2_pair ? SRMRA_P2_PAIR
           : p.p2_gc <= 1 ? SRMRA_P2_PER_CHUNK
                          : (p.p2_gc <= 4 ? SRMRA_P2_RING : SRMRA_P2_INTERLEAVED);
  else if (c->prec == SRMRA_FFT32)
    form = SRMRA_P2_FFT;
  const int32_t v[7] = {p.p1_groups, p.p1_tiles_per_group, p.p2_gc, p.p2_chunk_groups, form,
                        p.p2_nsplit, is_tc_prec(c->prec) ? p.p1_bn : 0};
  for (int k = 0; k < n && k < 7; ++k) out[k] = v[k];
  return SRMRA_OK;
}

srmra_status srmra_profile(srmra_ctx* c, int32_t enable) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  c->profiling = enable != 0;
  return SRMRA_OK;
}

srmra_status srmra_profile_read(srmra_ctx* c, double* ms, int64_t* count) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  CK(c, cudaStreamSynchronize(c->stream));
  for (const auto& m : c->marks) {
    float t = 0.f;
    CK(c, cudaEventElapsedTime(&t, m.a, m.b));
    if (ms) ms[m.phase] += (double)t;
    if (count) count[m.phase] += 1;
    c->event_pool.push_back(m.a);
    c->event_pool.push_back(m.b);
  }
  c->marks.clear();
  return SRMRA_OK;
}

srmra_status srmra_sync(srmra_ctx* c) {
  if (!c) return fail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  CK(c, cudaStreamSynchronize(c->stream));
  return SRMRA_OK;
}

void srmra_destroy(srmra_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (void* p : c->owned) cudaFree(p);
  for (const auto& m : c->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (cudaEvent_t ev : c->event_pool) cudaEventDestroy(ev);
  if (c->ll_hist) cudaFree(c->ll_hist);
  delete c;
}

}  // extern "C"
