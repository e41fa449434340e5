// Batched projected EM: many independent SR-MRA problems advanced together.
//
// Each EM iteration of a batch runs the per-problem preparation kernels, ONE grouped
// persistent launch of pass 1 over the work units of every problem, the per-problem
// log-sum-exp combine, ONE grouped launch of pass 2, the per-problem finalize and the
// projection step of Algorithm 2 read from a per-problem schedule in device memory
// (t, F, sigma_BM, decay).  Because nothing in the sequence depends on host state, one
// iteration is captured once into a CUDA graph and replayed.  The work decomposition of
// the grouped launches (shift groups of pass 1, observation ranges of pass 2, order of
// the problems in the unit list) is chosen by a small autotuner that times candidate
// decompositions with CUDA events and keeps the fastest.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "srmra_internal.cuh"

using namespace srmra;

struct srmra_batch {
  std::vector<srmra_ctx*> given;  // caller's order
  std::vector<srmra_ctx*> ctxs;   // launch order
  std::vector<int64_t> graph_launches;  // kernels per replay, per context (launch order)
  int prec = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  uint32_t flags = 0;
  void* d_insts = nullptr;        // grouped descriptors (tensor-core forms)
  int64_t* d_ustart = nullptr;    // pass 1: [n+1]; pass 2: [len+1] per cluster-size range
  int64_t total1 = 0;
  struct P2Range { int G, k0, k1; int64_t off, total; };
  std::vector<P2Range> p2;        // pass-2 launches, one per cluster size
  std::vector<unsigned char> h_insts;
  std::vector<int64_t> h_ustart;
  int64_t ustart_cap = 0;
  int* d_status = nullptr;
  cudaStream_t cap_stream = nullptr;  // capture stream (the contexts' may be legacy)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // around the grouped passes
  // side streams for the per-problem kernels (preparation, combine, finalize and
  // projection): independent problems run concurrently, forked from and joined to the
  // batch stream with events (branches of the captured graph)
  static constexpr int kSide = 8;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kSide] = {};
  int tuned_s1 = 1, tuned_s2 = 1, tuned_order = 0, tuned_bn = 256;
  double tuned_ms = 0.0;
  std::string err;
};

namespace {

thread_local std::string g_batch_err;

srmra_status bfail(srmra_batch* b, srmra_status st, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    g_batch_err = msg;
  return st;
}

srmra_status bcuda(srmra_batch* b, cudaError_t e, const char* what) {
  return bfail(b, e == cudaErrorMemoryAllocation ? SRMRA_ENOMEM : SRMRA_ECUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

#define BCK(b, call)                                       \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return bcuda((b), e_, #call);   \
  } while (0)

bool is_tc(int prec) { return is_tc_prec(prec); }

// Estimated cost of one pass-2 unit of a context (pixels x logit depth x observations).
double unit_cost(const srmra_ctx* c) {
  const Geom& g = c->g;
  return (double)c->plan.p2_iblk_per_split * (double)g.l2 * 3.0 + 1.0;
}

// Rebuild the grouped descriptor table and unit prefix sums in the batch order.
srmra_status upload_group(srmra_batch* b) {
  if (!is_tc(b->prec)) return SRMRA_OK;
  const size_t isz = tc_inst_bytes();
  const int n = (int)b->ctxs.size();
  b->h_insts.assign(isz * n + 64, 0);
  unsigned char* base =
      (unsigned char*)(((uintptr_t)b->h_insts.data() + 63) & ~(uintptr_t)63);
  // pass 2 launches once per kernel (cluster size, or the compensated per-chunk kernel):
  // keep contexts of one kernel contiguous
  std::stable_sort(b->ctxs.begin(), b->ctxs.end(), [](const srmra_ctx* x, const srmra_ctx* y) {
    return tc_p2_key(x) < tc_p2_key(y);
  });
  b->h_ustart.assign(n + 1, 0);
  for (int k = 0; k < n; ++k) {
    tc_fill_inst(b->ctxs[k], base + isz * k);
    b->h_ustart[k + 1] = b->h_ustart[k] + tc_units(b->ctxs[k], 1);
  }
  b->total1 = b->h_ustart[n];
  b->p2.clear();
  for (int k0 = 0; k0 < n;) {
    const int G = tc_p2_key(b->ctxs[k0]);
    int k1 = k0;
    while (k1 < n && tc_p2_key(b->ctxs[k1]) == G) ++k1;
    srmra_batch::P2Range rg{G, k0, k1, (int64_t)b->h_ustart.size(), 0};
    b->h_ustart.push_back(0);
    for (int k = k0; k < k1; ++k) b->h_ustart.push_back(b->h_ustart.back() + tc_units(b->ctxs[k], 2));
    rg.total = b->h_ustart.back();
    b->p2.push_back(rg);
    k0 = k1;
  }
  if (b->h_ustart.size() > (size_t)b->ustart_cap) {
    if (b->d_ustart) cudaFree(b->d_ustart);
    b->d_ustart = nullptr;
    BCK(b, cudaMalloc((void**)&b->d_ustart, sizeof(int64_t) * b->h_ustart.size()));
    b->ustart_cap = (int64_t)b->h_ustart.size();
  }
  BCK(b, cudaMemcpyAsync(b->d_insts, base, isz * n, cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaMemcpyAsync(b->d_ustart, b->h_ustart.data(), sizeof(int64_t) * b->h_ustart.size(),
                         cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  return SRMRA_OK;
}

cudaError_t launch_pass(srmra_batch* b, int pass) {
  const int n = (int)b->ctxs.size();
  if (is_tc(b->prec)) {
    for (auto* c : b->ctxs) c->launches++;
    if (pass == 1)
      return tc_launch_group(1, b->prec, b->ctxs[0]->plan.p1_bn, b->d_insts, b->d_ustart, n,
                             b->total1, b->d_status,
                             b->stream, b->num_sms);
    const size_t isz = tc_inst_bytes();
    for (const auto& rg : b->p2) {
      cudaError_t e = tc_launch_group_p2(rg.G, b->prec, (const char*)b->d_insts + isz * rg.k0,
                                         b->d_ustart + rg.off, rg.k1 - rg.k0, rg.total,
                                         b->d_status, b->stream, b->num_sms);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (auto* c : b->ctxs) {
    const bool fft = c->prec == SRMRA_FFT32;
    if (pass == 1) {
      if (fft)
        launch_pass1_fft(c);
      else
        launch_pass1_f32(c);
    } else {
      cudaError_t e = fft ? launch_pass2_fft(c) : launch_pass2_f32(c);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

// Runs `work(c)` for every context of the batch, problem k on side stream k mod kSide
// (each problem's kernels stay in order on one stream), after everything enqueued on
// the batch stream so far; the batch stream then waits for all of them.
template <typename Work>
cudaError_t per_problem(srmra_batch* b, Work work) {
  cudaError_t e = cudaEventRecord(b->fork_ev, b->stream);
  const int ns = std::min<int>(srmra_batch::kSide, (int)b->ctxs.size());
  for (int k = 0; k < ns && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->fork_ev, 0);
  for (size_t i = 0; i < b->ctxs.size() && e == cudaSuccess; ++i) {
    srmra_ctx* c = b->ctxs[i];
    const cudaStream_t own = c->stream;
    c->stream = b->side[i % srmra_batch::kSide];
    work(c);
    c->stream = own;
    e = cudaGetLastError();
  }
  for (int k = 0; k < ns && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->join_ev[k], b->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join_ev[k], 0);
  }
  return e;
}

// One EM iteration + scheduled projection for every context of the batch.
cudaError_t enqueue_iteration(srmra_batch* b) {
  cudaError_t e = per_problem(b, [](srmra_ctx* c) { launch_prep_iter(c); });
  if (e != cudaSuccess) return e;
  cudaEventRecord(b->ev[0], b->stream);
  e = launch_pass(b, 1);
  if (e != cudaSuccess) return e;
  cudaEventRecord(b->ev[1], b->stream);
  e = per_problem(b, [](srmra_ctx* c) { launch_lse_combine(c, c->plan.p1_groups); });
  if (e != cudaSuccess) return e;
  cudaEventRecord(b->ev[2], b->stream);
  e = launch_pass(b, 2);
  if (e != cudaSuccess) return e;
  cudaEventRecord(b->ev[3], b->stream);
  e = per_problem(b, [](srmra_ctx* c) {
    launch_finalize(c, 0);
    launch_dct_sched(c, 2.7);
  });
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

srmra_status capture_graph(srmra_batch* b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  if (!b->cap_stream) BCK(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  // Capture on the batch's own stream (the contexts may use the legacy stream, which
  // cannot be captured); the graph is replayed on the contexts' stream.
  std::vector<int64_t> before;
  for (auto* c : b->ctxs) {
    before.push_back(c->launches);
    c->stream = b->cap_stream;
  }
  const cudaStream_t real = b->stream;
  b->stream = b->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = enqueue_iteration(b);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
  b->stream = real;
  b->graph_launches.assign(b->ctxs.size(), 0);
  for (size_t k = 0; k < b->ctxs.size(); ++k) {  // capturing enqueues nothing yet
    b->ctxs[k]->stream = real;
    b->graph_launches[k] = b->ctxs[k]->launches - before[k];
    b->ctxs[k]->launches = before[k];
  }
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bcuda(b, e, "capture iteration");
  }
  if (e2 != cudaSuccess) return bcuda(b, e2, "end capture");
  b->graph = g;
  BCK(b, cudaGraphInstantiate(&b->exec, g, 0));
  return SRMRA_OK;
}

// Time the two grouped passes (with the combine between them) for the current
// decomposition.  Reads the current estimates, writes only per-iteration scratch.
srmra_status time_passes(srmra_batch* b, int reps, double* ms) {
  cudaEvent_t e0, e1;
  BCK(b, cudaEventCreate(&e0));
  BCK(b, cudaEventCreate(&e1));
  float best = 1e30f;
  for (int r = 0; r < reps + 1; ++r) {
    BCK(b, cudaEventRecord(e0, b->stream));
    BCK(b, launch_pass(b, 1));
    BCK(b, per_problem(b, [](srmra_ctx* c) { launch_lse_combine(c, c->plan.p1_groups); }));
    BCK(b, launch_pass(b, 2));
    BCK(b, cudaEventRecord(e1, b->stream));
    BCK(b, cudaEventSynchronize(e1));
    float t = 0.f;
    BCK(b, cudaEventElapsedTime(&t, e0, e1));
    if (r > 0) best = std::min(best, t);  // the first repetition warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return SRMRA_OK;
}

srmra_status apply_decomposition(srmra_batch* b, int s1, int s2, int order, int bn) {
  b->ctxs = b->given;
  if (order == 1)
    std::stable_sort(b->ctxs.begin(), b->ctxs.end(), [](const srmra_ctx* x, const srmra_ctx* y) {
      return unit_cost(x) > unit_cost(y);
    });
  for (auto* c : b->ctxs) BCK(b, tc_replan(c, s1, s2, bn));
  return upload_group(b);
}

// The autotuner: times the grouped passes for every candidate (pass-1 tile width 256 or
// 128 shifts) x (pass-1 shift groups x1, x2) x (pass-2 observation ranges x1, x2) x
// (problem order as given, costliest units first) on the current estimates (no state
// changes) and keeps the fastest.
srmra_status autotune(srmra_batch* b) {
  for (auto* c : b->ctxs) launch_prep_iter(c);  // operands of the current estimates
  BCK(b, cudaGetLastError());
  double best = 1e300;
  int bs1 = 1, bs2 = 1, bo = 0, bbn = 256;
  for (int bn : {256, 128})
    for (int order = 0; order < 2; ++order)
      for (int s1 : {1, 2})
        for (int s2 : {1, 2}) {
          srmra_status st = apply_decomposition(b, s1, s2, order, bn);
          if (st != SRMRA_OK) return st;
          double ms = 0.0;
          st = time_passes(b, 2, &ms);
          if (st != SRMRA_OK) return st;
          if (ms < best) {
            best = ms;
            bs1 = s1;
            bs2 = s2;
            bo = order;
            bbn = bn;
          }
        }
  b->tuned_s1 = bs1;
  b->tuned_s2 = bs2;
  b->tuned_order = bo;
  b->tuned_bn = bbn;
  b->tuned_ms = best;
  return apply_decomposition(b, bs1, bs2, bo, bbn);
}

}  // namespace

extern "C" {

srmra_status srmra_batch_create(srmra_ctx** ctxs, int32_t count, uint32_t flags,
                                srmra_batch** out) {
  if (!out) return bfail(nullptr, SRMRA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctxs || count < 1) return bfail(nullptr, SRMRA_EINVAL, "need at least one context");
  for (int k = 0; k < count; ++k) {
    if (!ctxs[k]) return bfail(nullptr, SRMRA_EINVAL, "NULL context in the batch");
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return bfail(nullptr, SRMRA_EINVAL, "context listed twice");
    if (ctxs[k]->prec != ctxs[0]->prec)
      return bfail(nullptr, SRMRA_EINVAL, "all contexts of a batch need the same precision");
    if (ctxs[k]->stream != ctxs[0]->stream || ctxs[k]->device != ctxs[0]->device)
      return bfail(nullptr, SRMRA_EINVAL, "all contexts of a batch need the same stream");
  }
  if (is_tc_prec(ctxs[0]->prec) && !(flags & SRMRA_BATCH_AUTOTUNE))
    for (int k = 1; k < count; ++k)
      if (ctxs[k]->plan.p1_bn != ctxs[0]->plan.p1_bn)
        return bfail(nullptr, SRMRA_EINVAL,
                     "contexts with different pass-1 tile widths need SRMRA_BATCH_AUTOTUNE");
  auto* b = new (std::nothrow) srmra_batch();
  if (!b) return bfail(nullptr, SRMRA_ENOMEM, "host allocation failed");
  b->ctxs.assign(ctxs, ctxs + count);
  b->given = b->ctxs;
  b->prec = ctxs[0]->prec;
  b->stream = ctxs[0]->stream;
  b->num_sms = ctxs[0]->num_sms;
  b->flags = flags;
  b->tuned_bn = ctxs[0]->plan.p1_bn;
  cudaError_t e = is_tc(b->prec)                ? tc_set_attributes(b->prec)
                  : b->prec == SRMRA_FFT32 ? fft_set_attributes()
                                           : simt_set_attributes();
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&b->ev[k]);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
  for (int k = 0; k < srmra_batch::kSide && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream);
  if (e == cudaSuccess && is_tc(b->prec)) {
    e = cudaMalloc(&b->d_insts, tc_inst_bytes() * count);
  }
  srmra_status st = SRMRA_OK;
  if (e != cudaSuccess) st = bcuda(nullptr, e, "batch buffers");
  if (st == SRMRA_OK) {
    st = upload_group(b);
    if (st == SRMRA_OK && is_tc(b->prec) && (flags & SRMRA_BATCH_AUTOTUNE)) st = autotune(b);
    if (st != SRMRA_OK) g_batch_err = b->err;
  }
  if (st != SRMRA_OK) {
    srmra_batch_destroy(b);
    return st;
  }
  *out = b;
  return SRMRA_OK;
}

srmra_status srmra_batch_solve(srmra_batch* b, int32_t iters, int32_t F, double sigma_bm1,
                               double decay, double* loglik_last) {
  if (!b) return bfail(nullptr, SRMRA_EINVAL, "batch is NULL");
  if (iters < 0 || (F >= 0 && !(decay > 0.0)))
    return bfail(b, SRMRA_EINVAL, "need iters >= 0 and decay > 0");
  for (auto* c : b->ctxs)
    if ((F > 0 || (F < 0 && c->sched_F > 0)) && c->g.L % 8 != 0)
      return bfail(b, SRMRA_EINVAL, "built-in denoiser needs L % 8 == 0");
  // the Algorithm 2 schedule of every context goes to device memory
  std::vector<DevSched> sched(b->ctxs.size());
  for (size_t k = 0; k < b->ctxs.size(); ++k) {
    srmra_ctx* c = b->ctxs[k];
    if (sigma_bm1 > 0.0) c->sigma_bm = sigma_bm1;
    sched[k] = (F >= 0) ? DevSched{c->t, F, c->sigma_bm, decay}
                        : DevSched{c->t, c->sched_F, c->sigma_bm, c->sched_decay};
    BCK(b, cudaMemcpyAsync(c->d_sched, &sched[k], sizeof(DevSched), cudaMemcpyHostToDevice,
                           b->stream));
  }
  const bool use_graph = !(b->flags & SRMRA_BATCH_NO_GRAPH);
  if (use_graph && !b->exec && iters > 0) {
    srmra_status st = capture_graph(b);
    if (st != SRMRA_OK) return st;
  }
  for (int it = 0; it < iters; ++it) {
    if (use_graph) {
      BCK(b, cudaGraphLaunch(b->exec, b->stream));
      for (size_t k = 0; k < b->ctxs.size(); ++k) b->ctxs[k]->launches += b->graph_launches[k];
    } else {
      BCK(b, enqueue_iteration(b));
    }
  }
  std::vector<double> ll(b->ctxs.size(), 0.0);
  for (size_t k = 0; k < b->ctxs.size(); ++k) {
    srmra_ctx* c = b->ctxs[k];
    BCK(b, cudaMemcpyAsync(&sched[k], c->d_sched, sizeof(DevSched), cudaMemcpyDeviceToHost,
                           b->stream));
    if (loglik_last)
      BCK(b, cudaMemcpyAsync(&ll[k], c->ll_hist, sizeof(double), cudaMemcpyDeviceToHost,
                             b->stream));
  }
  int st_dev = 0;
  BCK(b, cudaMemcpyAsync(&st_dev, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  for (size_t k = 0; k < b->ctxs.size(); ++k) {
    srmra_ctx* c = b->ctxs[k];
    c->t = sched[k].t;
    c->sigma_bm = sched[k].sigma_bm;
    if (iters > 0) c->have_estep = true;
  }
  if (st_dev & STATUS_TIMEOUT) return bfail(b, SRMRA_ETIMEOUT, "a bounded device wait timed out");
  if (loglik_last) {  // in the order of srmra_batch_create's input
    for (size_t k = 0; k < b->ctxs.size(); ++k) {
      const size_t pos =
          std::find(b->given.begin(), b->given.end(), b->ctxs[k]) - b->given.begin();
      loglik_last[pos] = ll[k];
    }
  }
  return SRMRA_OK;
}

srmra_status srmra_batch_tuning(const srmra_batch* b, int32_t* p1_scale, int32_t* p2_scale,
                                int32_t* order, double* ms) {
  if (!b) return bfail(nullptr, SRMRA_EINVAL, "batch is NULL");
  if (p1_scale) *p1_scale = b->tuned_s1;
  if (p2_scale) *p2_scale = b->tuned_s2;
  if (order) *order = b->tuned_order;
  if (ms) *ms = b->tuned_ms;
  return SRMRA_OK;
}

srmra_status srmra_batch_tiles(const srmra_batch* b, int32_t* p1_shift_tile) {
  if (!b) return bfail(nullptr, SRMRA_EINVAL, "batch is NULL");
  if (p1_shift_tile) *p1_shift_tile = b->tuned_bn;
  return SRMRA_OK;
}

srmra_status srmra_batch_pass_ms(srmra_batch* b, double* ms_pass1, double* ms_pass2) {
  if (!b) return bfail(nullptr, SRMRA_EINVAL, "batch is NULL");
  BCK(b, cudaStreamSynchronize(b->stream));
  float t1 = 0.f, t2 = 0.f;
  BCK(b, cudaEventElapsedTime(&t1, b->ev[0], b->ev[1]));
  BCK(b, cudaEventElapsedTime(&t2, b->ev[2], b->ev[3]));
  if (ms_pass1) *ms_pass1 = t1;
  if (ms_pass2) *ms_pass2 = t2;
  return SRMRA_OK;
}

void srmra_batch_destroy(srmra_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (int k = 0; k < 4; ++k)
    if (b->ev[k]) cudaEventDestroy(b->ev[k]);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  for (int k = 0; k < srmra_batch::kSide; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
  }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->d_insts) cudaFree(b->d_insts);
  if (b->d_ustart) cudaFree(b->d_ustart);
  if (b->d_status) cudaFree(b->d_status);
  delete b;
}

const char* srmra_batch_last_error(const srmra_batch* b) {
  return b ? b->err.c_str() : g_batch_err.c_str();
}

srmra_status srmra_em_iter_batch(srmra_ctx** ctxs, int32_t count, int32_t n_iters) {
  srmra_batch* b = nullptr;
  srmra_status st = srmra_batch_create(ctxs, count, SRMRA_BATCH_NO_GRAPH, &b);
  if (st != SRMRA_OK) return st;
  st = srmra_batch_solve(b, n_iters, 0, 0.0, 1.0, nullptr);
  if (st != SRMRA_OK) g_batch_err = b->err;
  srmra_batch_destroy(b);
  return st;
}

}  // extern "C"
