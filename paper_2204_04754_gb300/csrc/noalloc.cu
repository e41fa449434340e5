// Allocation-free evaluation of the per-observation log-likelihood terms.
//
// Some callers cannot call cudaMalloc: services that size all device memory once at
// start-up so that no request can fail later on an allocation, host code that must not
// block on the allocator (cudaMalloc can synchronise the device), and embedders whose
// own allocator owns every byte of device memory.  srmra_loglik_noalloc serves them: it
// runs the
// float32 E-step normaliser (observation centring, template preparation, the pass-1
// kernel and the log-sum-exp combine) with every intermediate buffer placed in one
// fixed, file-scope device array instead of memory obtained from an allocator.
#include <cuda.h>

#include <mutex>

#include "srmra_internal.cuh"

namespace srmra {
namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB per device, held until exit
constexpr int kMaxDevices = 64;

// Shared by every call on a device; holds the last call's intermediates.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context the address belongs to

// Unique id of the CUDA context current on this thread (0 if none is current or the
// driver cannot tell).  A device reset destroys the context and the module with the
// array, and the next context may place the array elsewhere: the id tells the cached
// address apart from a stale one.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {  // under g_setup_mutex
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) ==
            cudaSuccess &&
        qa == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) ==
            cudaSuccess &&
        qb == cudaDriverEntryPointSuccess) {
      get_current = (GetCurrent)a;
      get_id = (GetId)b;
    }
    cudaGetLastError();
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array for the current device, looked up with that
// device current the first time (and again whenever the device's context is no longer
// the one the address was taken in, e.g. after a device reset).  Host code must not use
// the symbol itself: on the host it names a stand-in object, not device memory.
cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  const unsigned long long id = current_context_id();
  if (g_scratch_ptr[dev] && id != 0 && id == g_scratch_ctx[dev]) {
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  g_scratch_ptr[dev] = p;
  g_scratch_ctx[dev] = current_context_id();
  *out = p;
  return cudaSuccess;
}

thread_local std::string g_noalloc_err;

srmra_status noalloc_fail(srmra_status st, const std::string& msg) {
  g_noalloc_err = msg;
  return st;
}

// Carves 256-byte aligned pieces out of the scratch array.
struct Carver {
  unsigned char* base;
  size_t used = 0;
  template <typename T>
  T* take(int64_t count) {
    T* p = reinterpret_cast<T*>(base + used);
    used += (size_t)round_up(count * (int64_t)sizeof(T), 256);
    return p;
  }
};

}  // namespace
}  // namespace srmra

using namespace srmra;

extern "C" srmra_status srmra_loglik_noalloc(const float* y_dev, int64_t N, int32_t L,
                                             int32_t K, double sigma, const float* x_dev,
                                             const double* rho1_dev, const double* rho2_dev,
                                             double* lse_dev, double* ll_dev,
                                             void* cuda_stream) {
  if (!y_dev || !x_dev || !rho1_dev || !rho2_dev || !lse_dev || !ll_dev)
    return noalloc_fail(SRMRA_EINVAL, "a required pointer is NULL");
  if (L < 2 || K < 1 || L % K != 0 || N < 1 || !(sigma > 0.0))
    return noalloc_fail(SRMRA_EINVAL, "need L >= 2, K dividing L, N >= 1, sigma > 0");

  srmra_ctx c;  // a view: every buffer pointer below points into the scratch array
  Geom& g = c.g;
  g.L = L;
  g.K = K;
  g.l = L / K;
  g.l2 = g.l * g.l;
  g.S = L * L;
  g.Spad = (int)round_up(g.S, SPAD);
  g.ldy = (int)round_up(g.l2, 16);
  g.ldk = (int)round_up(g.l2, 64);
  g.N = N;
  g.Npad = round_up(N, NPAD);
  g.sigma = sigma;
  c.prec = SRMRA_FP32;
  c.stream = (cudaStream_t)cuda_stream;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return noalloc_fail(SRMRA_ECUDA, cudaGetErrorString(e));
  plan_simt(&c);

  void* scratch = nullptr;
  e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess)
    return noalloc_fail(SRMRA_ECUDA, std::string("scratch lookup: ") + cudaGetErrorString(e));
  Carver cv{static_cast<unsigned char*>(scratch)};
  c.Yc = cv.take<float>(g.Npad * g.ldy);
  c.YcT = cv.take<float>(g.Npad * g.ldy);
  c.ybar = cv.take<float>(g.Npad);
  c.yy = cv.take<double>(g.Npad);
  c.x = const_cast<float*>(x_dev);
  c.rho1 = const_cast<double*>(rho1_dev);
  c.rho2 = const_cast<double*>(rho2_dev);
  c.sub = cv.take<double>(2 * K * K);
  c.colb = cv.take<float>(g.Spad);
  c.colm = cv.take<float>(g.Spad);
  c.AxT = cv.take<float>((int64_t)g.ldy * g.Spad);
  c.pm = cv.take<float>((int64_t)c.plan.p1_groups * g.Npad);
  c.ps = cv.take<float>((int64_t)c.plan.p1_groups * g.Npad);
  c.lse2 = cv.take<float>(g.Npad);
  c.llpart = cv.take<double>(c.plan.ll_blocks);
  c.lse = lse_dev;  // the combine kernel writes entries 0..N-1 only
  const size_t ybar_bytes = (size_t)g.Npad * sizeof(float);
  const size_t yy_bytes = (size_t)g.Npad * sizeof(double);
  if (cv.used > kScratchBytes)
    return noalloc_fail(SRMRA_EINVAL, "problem needs " + std::to_string(cv.used) +
                                          " bytes of scratch; the fixed array holds " +
                                          std::to_string(kScratchBytes));
  // zero what the kernels read without writing: the padding observation rows
  e = cudaMemsetAsync(c.Yc, 0, (size_t)g.Npad * g.ldy * sizeof(float), c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.ybar, 0, ybar_bytes, c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.yy, 0, yy_bytes, c.stream);
  if (e != cudaSuccess) return noalloc_fail(SRMRA_ECUDA, cudaGetErrorString(e));

  launch_center_obs(&c, y_dev);
  launch_prep_iter(&c);
  launch_pass1_f32(&c);
  launch_lse_combine(&c, c.plan.p1_groups);
  // LL = sum of the combine kernel's block partials, reduced in a fixed order
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_sum_f64(c.llpart, c.plan.ll_blocks, ll_dev, c.stream);
  if (e != cudaSuccess) return noalloc_fail(SRMRA_ECUDA, cudaGetErrorString(e));
  return SRMRA_OK;
}

extern "C" const char* srmra_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

extern "C" int64_t srmra_noalloc_scratch_bytes(void) { return (int64_t)kScratchBytes; }
