// Projected method of moments (Algorithm 1) on a context's device-resident observations;
// declared in include/srmra.h.
//
//   empirical moments (Eq. empiric_MOM, D = 2), once, in one pass over the observations
//   y_i = y'_i + ybar_i:   M1^ = (1/N) sum_i y_i,   M2^ = (1/N) Y^T Y;
//   per step, at theta = (x, rho = rho1 rho2^T) with the templates t_s = P R_s x (rows of
//   T, L^2 x l^2):
//     M1 = T^T rho,  M2 = T^T diag(rho) T + sigma^2 I,  R = M2 - M2^,  r = M1 - M1^,
//     f  = ||R||_F^2 + lambda ||r||^2,  lambda = 1 / (L^2 (1 + sigma^2))   (Eq. LS_SR),
//     U  = T R (rows R t_s),  df/drho_s = 2 u_s . t_s + 2 lambda t_s . r,
//     df/dx = sum_s rho_s (P R_s)^T (4 u_s + 2 lambda r),
//   then x <- x - mu_x df/dx, rho1 and rho2 <- simplex projections of a gradient step of
//   size mu_rho (df/drho1 = G rho2, df/drho2 = G^T rho1 with G[s1][s2] = df/drho_s), and
//   every F steps x <- D(x, sigma_BM), sigma_BM <- decay sigma_BM.
// The products Y^T Y, T^T diag(rho) T and T R run through one float32 tile kernel
// (k-major operands, 128 x 128 tiles, packed FMA, k split into partials that are summed in
// float64 in a fixed order); every other reduction is float64 in a fixed order.
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "srmra_internal.cuh"

using namespace srmra;

namespace {

using f2 = unsigned long long;
__device__ __forceinline__ void ffma2(f2& d, f2 a, f2 b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}
__device__ __forceinline__ f2 dup2(float x) {
  f2 r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lo2(f2 v) { return __uint_as_float((unsigned)(v & 0xffffffffull)); }
__device__ __forceinline__ float hi2(f2 v) { return __uint_as_float((unsigned)(v >> 32)); }

constexpr int GT = 128;  // product tile (rows and columns)

struct GemmArgs {
  const float* A;        // [K][lda], element (k, m)
  int lda, Mvalid;
  const float* B;        // [K][ldb], element (k, n)
  int ldb, Nvalid;
  const float* off;      // per-k offset added to row k of A and of B (nullable)
  const float* scale;    // per-k scale of row k of A (nullable)
  int Kvalid, kchunk;    // split z covers k in [z kchunk, min(Kvalid, (z + 1) kchunk))
  float* C;              // [split][Mpad][ldc]
  int ldc;
  int64_t c_split;       // elements between splits
};

// C[m][n] = sum_k (A[k][m] + off[k]) scale[k] (B[k][n] + off[k]) over one 128 x 128 tile
// and one k range; 256 threads with 8 x 8 outputs each, k staged 8 rows at a time in a
// double-buffered shared tile.  Rows and columns past Mvalid / Nvalid and k past the range
// read as zero; the whole tile is written.
__global__ void __launch_bounds__(256) k_mom_gemm(GemmArgs g) {
  __shared__ __align__(16) float As[2][8][GT];
  __shared__ __align__(16) float Bs[2][8][GT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * GT, n0 = blockIdx.y * GT;
  const int k0 = blockIdx.z * g.kchunk, k1 = min(g.Kvalid, k0 + g.kchunk);
  const int lk = tid >> 5, lc = (tid & 31) * 4;
  auto load = [&](int k, float (&ra)[4], float (&rb)[4]) {
    const bool kv = k < k1;
    const float o = (kv && g.off) ? g.off[k] : 0.f;
    const float sc = (kv && g.scale) ? g.scale[k] : 1.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int m = m0 + lc + e, n = n0 + lc + e;
      ra[e] = (kv && m < g.Mvalid) ? (g.A[(int64_t)k * g.lda + m] + o) * sc : 0.f;
      rb[e] = (kv && n < g.Nvalid) ? g.B[(int64_t)k * g.ldb + n] + o : 0.f;
    }
  };
  f2 acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[j][c] = 0ull;
  float ra[4], rb[4];
  load(k0 + lk, ra, rb);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    As[0][lk][lc + e] = ra[e];
    Bs[0][lk][lc + e] = rb[e];
  }
  __syncthreads();
  int cur = 0;
  for (int kc = k0; kc < k1; kc += 8) {
    const bool more = kc + 8 < k1;
    if (more) load(kc + 8 + lk, ra, rb);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
      const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(&Bs[cur][kk][tx * 4]);
      const ulonglong2 b1 = *reinterpret_cast<const ulonglong2*>(&Bs[cur][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const f2 b[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const f2 aj = dup2(a[j]);
#pragma unroll
        for (int c = 0; c < 4; ++c) ffma2(acc[j][c], aj, b[c]);
      }
    }
    if (more) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        As[cur ^ 1][lk][lc + e] = ra[e];
        Bs[cur ^ 1][lk][lc + e] = rb[e];
      }
    }
    __syncthreads();
    cur ^= 1;
  }
  float* C = g.C + (int64_t)blockIdx.z * g.c_split;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int m = m0 + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int n = n0 + (c < 2 ? tx * 4 + 2 * c : 64 + tx * 4 + 2 * (c - 2));
      *reinterpret_cast<float2*>(&C[(int64_t)m * g.ldc + n]) =
          make_float2(lo2(acc[j][c]), hi2(acc[j][c]));
    }
  }
}

// part[z][n] = sum over rows k of split z of (A[k][n] + off[k]) scale[k]  (float64).
__global__ void k_mom_colsum(const float* __restrict__ A, int lda, int cols,
                             const float* __restrict__ off, const float* __restrict__ scale,
                             int64_t rows, int64_t chunk, double* __restrict__ part) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= cols) return;
  const int64_t k0 = blockIdx.y * chunk, k1 = rows < k0 + chunk ? rows : k0 + chunk;
  double s = 0.0;
  for (int64_t k = k0; k < k1; ++k) {
    const double v = (double)A[k * lda + n] + (off ? (double)off[k] : 0.0);
    s += scale ? v * (double)scale[k] : v;
  }
  part[(int64_t)blockIdx.y * cols + n] = s;
}

// Empirical moments from the split partials: M2^ [l2][l2] and M1^ [l2], float64.
__global__ void k_mom_hat(const float* __restrict__ part, int nsplit, int64_t split_stride,
                          int l2, int l2p, const double* __restrict__ part1, int nsplit1,
                          double inv_n, double* __restrict__ M2h, double* __restrict__ M1h) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (int64_t)l2 * l2) {
    const int m = (int)(idx / l2), n = (int)(idx % l2);
    double s = 0.0;
    for (int p = 0; p < nsplit; ++p) s += (double)part[p * split_stride + (int64_t)m * l2p + n];
    M2h[idx] = s * inv_n;
  }
  if (idx < l2) {
    double s = 0.0;
    for (int p = 0; p < nsplit1; ++p) s += part1[(int64_t)p * l2 + idx];
    M1h[idx] = s * inv_n;
  }
}

// Templates t_s = P R_s x in both layouts, T[s][n] and TT[n][s] (zero padding), and the
// joint prior rho_s = rho1[s1] rho2[s2] (block row 0).
__global__ void k_mom_templates(const float* __restrict__ x, const double* __restrict__ rho1,
                                const double* __restrict__ rho2, int L, int K, int l, int S,
                                int Spad, int l2p, float* __restrict__ T, float* __restrict__ TT,
                                float* __restrict__ rho) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = blockIdx.y;
  if (s >= Spad) return;
  float v = 0.f;
  if (s < S && n < l * l) {
    const int s1 = s / L, s2 = s % L, n1 = n / l, n2 = n % l;
    v = x[((n1 * K - s1) % L + L) % L * L + ((n2 * K - s2) % L + L) % L];
  }
  T[(int64_t)s * l2p + n] = v;
  TT[(int64_t)n * Spad + s] = v;
  if (n == 0) rho[s] = s < S ? (float)(rho1[s / L] * rho2[s % L]) : 0.f;
}

// R = M2 - M2^ (float32 copy for the next product, zero padding), r = M1 - M1^, and the
// block partials of f = ||R||^2 + lambda ||r||^2.
__global__ void __launch_bounds__(256) k_mom_residual(
    const float* __restrict__ part, int nsplit, int64_t split_stride, int l2, int l2p,
    double sigma2, const double* __restrict__ M2h, const double* __restrict__ part1,
    int nsplit1, const double* __restrict__ M1h, double lambda, float* __restrict__ R,
    double* __restrict__ r1, double* __restrict__ fpart) {
  __shared__ double red[256];
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double f = 0.0;
  if (idx < (int64_t)l2p * l2p) {
    const int m = (int)(idx / l2p), n = (int)(idx % l2p);
    float rv = 0.f;
    if (m < l2 && n < l2) {
      double s = 0.0;
      for (int p = 0; p < nsplit; ++p) s += (double)part[p * split_stride + idx];
      const double d = s + (m == n ? sigma2 : 0.0) - M2h[(int64_t)m * l2 + n];
      f = d * d;
      rv = (float)d;
    }
    R[idx] = rv;
  }
  if (idx < l2) {
    double s = 0.0;
    for (int p = 0; p < nsplit1; ++p) s += part1[(int64_t)p * l2 + idx];
    const double d = s - M1h[idx];
    r1[idx] = d;
    f += lambda * d * d;
  }
  red[threadIdx.x] = f;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) fpart[blockIdx.x] = red[0];
}

// One warp per shift s: u_s from the split partials of U = T R,
// gs[s] = df/drho_s = 2 u_s . t_s + 2 lambda t_s . r, and the back-projection operand
// W[s][n] = rho_s (4 u_s[n] + 2 lambda r[n]).
__global__ void k_mom_gshift(const float* __restrict__ Upart, int nsplit, int64_t split_stride,
                             const float* __restrict__ T, const float* __restrict__ rho, int l2,
                             int l2p, int S, const double* __restrict__ r1, double lambda,
                             double* __restrict__ gs, float* __restrict__ W) {
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= S) return;
  const double rs = (double)rho[s];
  double a = 0.0, b = 0.0;
  for (int n = lane; n < l2; n += 32) {
    double u = 0.0;
    for (int p = 0; p < nsplit; ++p) u += (double)Upart[p * split_stride + (int64_t)s * l2p + n];
    const double t = (double)T[(int64_t)s * l2p + n];
    a += u * t;
    b += t * r1[n];
    W[(int64_t)s * l2p + n] = (float)(rs * (4.0 * u + 2.0 * lambda * r1[n]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) gs[s] = 2.0 * a + 2.0 * lambda * b;
}

// df/dx[q1][q2] = sum_{n1, n2} W[s(n1, q1) L + s(n2, q2)][n1 l + n2] with
// s(n, q) = (n K - q) mod L per axis (the adjoint of t_s = P R_s x).  One block per row
// q1; for each n1 and each 32-column chunk of n2 the slab of all L shifts s2 is staged in
// shared memory (pitch 33) so that the global reads are row-contiguous.
constexpr int GX_THREADS = 256;
constexpr int GX_MAXQ = 4;  // L <= GX_THREADS * GX_MAXQ
__global__ void __launch_bounds__(GX_THREADS) k_mom_gx(const float* __restrict__ W, int L, int K,
                                                       int l, int l2p, double* __restrict__ gx) {
  extern __shared__ float slab[];  // [L][33]
  const int q1 = blockIdx.x, tid = threadIdx.x;
  double acc[GX_MAXQ];
#pragma unroll
  for (int j = 0; j < GX_MAXQ; ++j) acc[j] = 0.0;
  for (int n1 = 0; n1 < l; ++n1) {
    const int s1 = ((n1 * K - q1) % L + L) % L;
    for (int c0 = 0; c0 < l; c0 += 32) {
      const int cw = min(32, l - c0);
      __syncthreads();
      for (int e = tid; e < L * 32; e += GX_THREADS) {
        const int s2 = e >> 5, j = e & 31;
        slab[s2 * 33 + j] = j < cw ? W[(int64_t)(s1 * L + s2) * l2p + n1 * l + c0 + j] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int jq = 0; jq < GX_MAXQ; ++jq) {
        const int q2 = tid + jq * GX_THREADS;
        if (q2 < L) {
          double a = 0.0;
          for (int j = 0; j < cw; ++j) {
            const int s2 = (((c0 + j) * K - q2) % L + L) % L;
            a += (double)slab[s2 * 33 + j];
          }
          acc[jq] += a;
        }
      }
    }
  }
#pragma unroll
  for (int jq = 0; jq < GX_MAXQ; ++jq) {
    const int q2 = tid + jq * GX_THREADS;
    if (q2 < L) gx[(int64_t)q1 * L + q2] = acc[jq];
  }
}

// Euclidean projection of v[0..n) onto the probability simplex, in place, by one block of
// at least n threads.  With the values ranked decreasingly (ties by index) and c_k the sum
// of the k largest, k* = max{k : u_k > (c_k - 1) / k} and the result is max(v - tau, 0)
// with tau = (c_k* - 1) / k*.
__device__ void simplex_project(double* v, int n, double* css, int* kk, double* tau) {
  const int t = threadIdx.x;
  if (t < n) {
    int rank = 0;
    double c = 0.0;
    for (int k = 0; k < n; ++k)
      if (v[k] > v[t] || (v[k] == v[t] && k < t)) {
        ++rank;
        c += v[k];
      }
    c += v[t];
    css[t] = c;
    kk[t] = (v[t] - (c - 1.0) / (rank + 1) > 0.0) ? rank + 1 : 0;
  }
  __syncthreads();
  if (t == 0) {
    int kb = 0;
    double cb = 0.0;
    for (int k = 0; k < n; ++k)
      if (kk[k] > kb) {
        kb = kk[k];
        cb = css[k];
      }
    *tau = kb > 0 ? (cb - 1.0) / kb : 0.0;
  }
  __syncthreads();
  if (t < n) v[t] = fmax(v[t] - *tau, 0.0);
  __syncthreads();
}

// f (from the block partials) into f_out; df/drho1 = G rho2 and df/drho2 = G^T rho1 into
// g12 (both at the current rho); with apply: x <- x - mu_x gx and rho1, rho2 <- their
// simplex projections after a step mu_rho.  One block of 1024 threads (L <= 1024).
__global__ void __launch_bounds__(1024) k_mom_step(
    const double* __restrict__ fpart, int nfp, const double* __restrict__ gs,
    const double* __restrict__ gx, int L, int apply, double mu_x, double mu_rho,
    float* __restrict__ x, double* __restrict__ rho1, double* __restrict__ rho2,
    double* __restrict__ g12, double* __restrict__ f_out, int* __restrict__ status) {
  __shared__ double red[1024], v1[1024], v2[1024], css[1024];
  __shared__ int kk[1024];
  __shared__ double tau;
  const int t = threadIdx.x;
  double f = 0.0;
  for (int k = t; k < nfp; k += 1024) f += fpart[k];
  red[t] = f;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) {
    *f_out = red[0];
    if (!isfinite(red[0])) atomicOr(status, STATUS_NUMERIC);
  }
  if (t < L) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < L; ++k) {
      a += gs[(int64_t)t * L + k] * rho2[k];
      b += gs[(int64_t)k * L + t] * rho1[k];
    }
    g12[t] = a;
    g12[L + t] = b;
    v1[t] = rho1[t] - mu_rho * a;
    v2[t] = rho2[t] - mu_rho * b;
  }
  __syncthreads();
  if (!apply) return;
  for (int q = t; q < L * L; q += 1024) x[q] = (float)((double)x[q] - mu_x * gx[q]);
  simplex_project(v1, L, css, kk, &tau);
  simplex_project(v2, L, css, kk, &tau);
  if (t < L) {
    rho1[t] = v1[t];
    rho2[t] = v2[t];
  }
}

}  // namespace

struct srmra_mom {
  srmra_ctx* ctx = nullptr;
  int l2p = 0, Mpad_u = 0;
  int ns_y = 1, ns_t = 1, ns_u = 1;  // k splits of the three products
  int ns_c1 = 1, ns_ct = 1;          // row splits of the two column sums
  double lambda = 0.0;
  double* M2h = nullptr;    // [l2][l2]
  double* M1h = nullptr;    // [l2]
  float* T = nullptr;       // [Spad][l2p]
  float* TT = nullptr;      // [l2p][Spad]
  float* rho = nullptr;     // [Spad]
  float* part = nullptr;    // split partials of the products
  double* part1 = nullptr;  // split partials of the column sums [ns][l2]
  float* R = nullptr;       // [l2p][l2p]
  float* W = nullptr;       // [Spad][l2p] back-projection operand
  double* r1 = nullptr;     // [l2]
  double* fpart = nullptr;  // [nfp]
  int nfp = 0;
  double* gs = nullptr;     // [S]
  double* gx = nullptr;     // [L*L]
  double* g12 = nullptr;    // [2L]
  double* fhist = nullptr;  // [fcap]
  int fcap = 0;
  int* status = nullptr;
  size_t gx_smem = 0;
  std::string err;
  std::vector<void*> owned;
};

namespace {

thread_local std::string g_mom_err;

srmra_status mfail(srmra_mom* m, srmra_status st, const std::string& msg) {
  if (m)
    m->err = msg;
  else
    g_mom_err = msg;
  return st;
}

#define MCK(m, call)                                                                    \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return mfail((m), SRMRA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
cudaError_t mget(srmra_mom* m, T** p, int64_t count) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)count);
  if (e != cudaSuccess) return e;
  m->owned.push_back(*p);
  return cudaMemsetAsync(*p, 0, sizeof(T) * (size_t)count, m->ctx->stream);
}

// k splits of a product with `tiles` output tiles: about two blocks per SM, at least
// 256 k per split.
int product_splits(int64_t tiles, int64_t kdim, int sms) {
  int64_t s = (2 * (int64_t)sms + tiles - 1) / tiles;
  const int64_t kmax = (kdim + 255) / 256;
  s = std::min(s, kmax);
  return (int)std::max<int64_t>(1, s);
}

// row splits of a column sum over `cols` columns: about two blocks per SM, at least 64
// rows per split.
int colsum_splits(int cols, int64_t rows, int sms) {
  const int64_t cb = ceil_div(cols, 256);
  int64_t s = (2 * (int64_t)sms + cb - 1) / cb;
  s = std::min(s, (rows + 63) / 64);
  return (int)std::max<int64_t>(1, s);
}

void gemm(srmra_mom* m, const GemmArgs& a, int Mpad, int Npad, int nsplit, cudaStream_t st) {
  dim3 grid((unsigned)(Mpad / GT), (unsigned)(Npad / GT), (unsigned)nsplit);
  k_mom_gemm<<<grid, 256, 0, st>>>(a);
  m->ctx->launches++;
}

void colsum(srmra_mom* m, const float* A, int lda, int cols, const float* off,
            const float* scale, int64_t rows, int nsplit, cudaStream_t st) {
  const int64_t chunk = ceil_div(rows, nsplit);
  k_mom_colsum<<<dim3((unsigned)ceil_div(cols, 256), (unsigned)nsplit), 256, 0, st>>>(
      A, lda, cols, off, scale, rows, chunk, m->part1);
  m->ctx->launches++;
}

// The empirical moments of the context's observations.
void launch_moments(srmra_mom* m) {
  srmra_ctx* c = m->ctx;
  const Geom& g = c->g;
  const cudaStream_t st = c->stream;
  const int l2p = m->l2p;
  GemmArgs a{c->Yc, g.ldy, g.l2, c->Yc, g.ldy, g.l2, c->ybar, nullptr, (int)g.N,
             (int)ceil_div(g.N, m->ns_y), m->part, l2p, (int64_t)l2p * l2p};
  gemm(m, a, l2p, l2p, m->ns_y, st);
  colsum(m, c->Yc, g.ldy, g.l2, c->ybar, nullptr, g.N, m->ns_c1, st);
  const int64_t n = (int64_t)g.l2 * g.l2;
  k_mom_hat<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(
      m->part, m->ns_y, (int64_t)l2p * l2p, g.l2, l2p, m->part1, m->ns_c1, 1.0 / (double)g.N,
      m->M2h, m->M1h);
  c->launches++;
}

// f and the gradient at the context's theta; with apply, the projected gradient step.
void launch_step(srmra_mom* m, int apply, double mu_x, double mu_rho, double* f_out) {
  srmra_ctx* c = m->ctx;
  const Geom& g = c->g;
  const cudaStream_t st = c->stream;
  const int l2p = m->l2p;
  k_mom_templates<<<dim3((unsigned)ceil_div(g.Spad, 256), (unsigned)l2p), 256, 0, st>>>(
      c->x, c->rho1, c->rho2, g.L, g.K, g.l, g.S, g.Spad, l2p, m->T, m->TT, m->rho);
  c->launches++;
  // M2 - sigma^2 I = T^T diag(rho) T and M1 = T^T rho
  GemmArgs a2{m->T, l2p, g.l2, m->T, l2p, g.l2, nullptr, m->rho, g.S,
              (int)ceil_div(g.S, m->ns_t), m->part, l2p, (int64_t)l2p * l2p};
  gemm(m, a2, l2p, l2p, m->ns_t, st);
  colsum(m, m->T, l2p, g.l2, nullptr, m->rho, g.S, m->ns_ct, st);
  k_mom_residual<<<(unsigned)m->nfp, 256, 0, st>>>(
      m->part, m->ns_t, (int64_t)l2p * l2p, g.l2, l2p, g.sigma * g.sigma, m->M2h, m->part1,
      m->ns_ct, m->M1h, m->lambda, m->R, m->r1, m->fpart);
  // U = T R (rows R t_s), then the shift gradient and the back-projection operand
  GemmArgs au{m->TT, g.Spad, g.S, m->R, l2p, g.l2, nullptr, nullptr, g.l2,
              (int)ceil_div(g.l2, m->ns_u), m->part, l2p, (int64_t)m->Mpad_u * l2p};
  gemm(m, au, m->Mpad_u, l2p, m->ns_u, st);
  k_mom_gshift<<<(unsigned)ceil_div(g.S, 8), 256, 0, st>>>(
      m->part, m->ns_u, (int64_t)m->Mpad_u * l2p, m->T, m->rho, g.l2, l2p, g.S, m->r1,
      m->lambda, m->gs, m->W);
  k_mom_gx<<<(unsigned)g.L, GX_THREADS, m->gx_smem, st>>>(m->W, g.L, g.K, g.l, l2p, m->gx);
  k_mom_step<<<1, 1024, 0, st>>>(m->fpart, m->nfp, m->gs, m->gx, g.L, apply, mu_x, mu_rho, c->x,
                                 c->rho1, c->rho2, m->g12, f_out, m->status);
  c->launches += 4;
}

srmra_status check_status(srmra_mom* m) {
  int status = 0;
  MCK(m, cudaMemcpyAsync(&status, m->status, sizeof(int), cudaMemcpyDeviceToHost,
                         m->ctx->stream));
  MCK(m, cudaStreamSynchronize(m->ctx->stream));
  if (status & STATUS_NUMERIC) return mfail(m, SRMRA_ENUMERIC, "NaN or Inf in the objective");
  return SRMRA_OK;
}

}  // namespace

extern "C" {

srmra_status srmra_mom_create(srmra_ctx* ctx, srmra_mom** out) {
  if (!out) return mfail(nullptr, SRMRA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctx) return mfail(nullptr, SRMRA_EINVAL, "ctx is NULL");
  const Geom& g = ctx->g;
  if (g.L > GX_THREADS * GX_MAXQ) return mfail(nullptr, SRMRA_EINVAL, "MoM needs L <= 1024");
  if (g.l2 > 8192) return mfail(nullptr, SRMRA_EINVAL, "MoM needs (L/K)^2 <= 8192");
  auto* m = new (std::nothrow) srmra_mom();
  if (!m) return mfail(nullptr, SRMRA_ENOMEM, "host allocation failed");
  m->ctx = ctx;
  m->l2p = (int)round_up(g.l2, GT);
  m->Mpad_u = (int)round_up(g.Spad, GT);
  m->lambda = 1.0 / ((double)g.L * g.L * (1.0 + g.sigma * g.sigma));
  const int l2p = m->l2p;
  const int sms = ctx->num_sms;
  const int64_t tiles2 = (int64_t)(l2p / GT) * (l2p / GT);
  m->ns_y = product_splits(tiles2, g.N, sms);
  m->ns_t = product_splits(tiles2, g.S, sms);
  m->ns_u = product_splits((int64_t)(m->Mpad_u / GT) * (l2p / GT), g.l2, sms);
  m->ns_c1 = colsum_splits(g.l2, g.N, sms);
  m->ns_ct = colsum_splits(g.l2, g.S, sms);
  const int64_t part = std::max({(int64_t)m->ns_y * l2p * l2p, (int64_t)m->ns_t * l2p * l2p,
                                 (int64_t)m->ns_u * m->Mpad_u * l2p});
  m->nfp = (int)ceil_div((int64_t)l2p * l2p, 256);
  m->gx_smem = sizeof(float) * (size_t)g.L * 33;
  cudaError_t e = mget(m, &m->M2h, (int64_t)g.l2 * g.l2);
  if (e == cudaSuccess) e = mget(m, &m->M1h, g.l2);
  if (e == cudaSuccess) e = mget(m, &m->T, (int64_t)g.Spad * l2p);
  if (e == cudaSuccess) e = mget(m, &m->TT, (int64_t)l2p * g.Spad);
  if (e == cudaSuccess) e = mget(m, &m->rho, g.Spad);
  if (e == cudaSuccess) e = mget(m, &m->part, part);
  if (e == cudaSuccess) e = mget(m, &m->part1, (int64_t)std::max(m->ns_c1, m->ns_ct) * g.l2);
  if (e == cudaSuccess) e = mget(m, &m->R, (int64_t)l2p * l2p);
  if (e == cudaSuccess) e = mget(m, &m->W, (int64_t)g.Spad * l2p);
  if (e == cudaSuccess) e = mget(m, &m->r1, g.l2);
  if (e == cudaSuccess) e = mget(m, &m->fpart, m->nfp);
  if (e == cudaSuccess) e = mget(m, &m->gs, g.S);
  if (e == cudaSuccess) e = mget(m, &m->gx, g.S);
  if (e == cudaSuccess) e = mget(m, &m->g12, 2 * g.L);
  if (e == cudaSuccess) e = mget(m, &m->status, 1);
  if (e == cudaSuccess && m->gx_smem > 48 * 1024)
    e = cudaFuncSetAttribute(k_mom_gx, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)m->gx_smem);
  if (e != cudaSuccess) {
    const std::string msg = std::string("MoM buffers: ") + cudaGetErrorString(e);
    srmra_mom_destroy(m);
    return mfail(nullptr, SRMRA_ENOMEM, msg);
  }
  launch_moments(m);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    const std::string msg = std::string("MoM moments: ") + cudaGetErrorString(e);
    srmra_mom_destroy(m);
    return mfail(nullptr, SRMRA_ECUDA, msg);
  }
  *out = m;
  return SRMRA_OK;
}

srmra_status srmra_mom_moments(srmra_mom* m, double* M1h, double* M2h) {
  if (!m) return mfail(nullptr, SRMRA_EINVAL, "mom is NULL");
  const Geom& g = m->ctx->g;
  const cudaStream_t st = m->ctx->stream;
  if (M1h) MCK(m, cudaMemcpyAsync(M1h, m->M1h, sizeof(double) * g.l2, cudaMemcpyDeviceToHost, st));
  if (M2h)
    MCK(m, cudaMemcpyAsync(M2h, m->M2h, sizeof(double) * g.l2 * g.l2, cudaMemcpyDeviceToHost, st));
  MCK(m, cudaStreamSynchronize(st));
  return SRMRA_OK;
}

srmra_status srmra_mom_recompute_moments(srmra_mom* m) {
  if (!m) return mfail(nullptr, SRMRA_EINVAL, "mom is NULL");
  launch_moments(m);
  MCK(m, cudaGetLastError());
  return SRMRA_OK;
}

srmra_status srmra_mom_eval(srmra_mom* m, double* f, double* gx, double* g1, double* g2) {
  if (!m) return mfail(nullptr, SRMRA_EINVAL, "mom is NULL");
  const Geom& g = m->ctx->g;
  const cudaStream_t st = m->ctx->stream;
  if (m->fcap < 1) {
    double* p = nullptr;
    MCK(m, cudaMalloc((void**)&p, sizeof(double)));
    m->owned.push_back(p);
    m->fhist = p;
    m->fcap = 1;
  }
  launch_step(m, 0, 0.0, 0.0, m->fhist);
  MCK(m, cudaGetLastError());
  if (f) MCK(m, cudaMemcpyAsync(f, m->fhist, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (gx) MCK(m, cudaMemcpyAsync(gx, m->gx, sizeof(double) * g.S, cudaMemcpyDeviceToHost, st));
  if (g1) MCK(m, cudaMemcpyAsync(g1, m->g12, sizeof(double) * g.L, cudaMemcpyDeviceToHost, st));
  if (g2)
    MCK(m, cudaMemcpyAsync(g2, m->g12 + g.L, sizeof(double) * g.L, cudaMemcpyDeviceToHost, st));
  return check_status(m);
}

srmra_status srmra_mom_run(srmra_mom* m, int32_t iters, int32_t F, double mu_x, double mu_rho,
                           double sigma_bm1, double decay, srmra_denoiser_fn fn, void* user,
                           double* f_out) {
  if (!m) return mfail(nullptr, SRMRA_EINVAL, "mom is NULL");
  srmra_ctx* c = m->ctx;
  if (iters < 0 || F < 0 || !(decay > 0.0) || !(sigma_bm1 >= 0.0) || !std::isfinite(mu_x) ||
      !std::isfinite(mu_rho))
    return mfail(m, SRMRA_EINVAL, "need iters >= 0, F >= 0, sigma_bm1 >= 0, decay > 0");
  if (F > 0 && !fn && c->g.L % 8 != 0)
    return mfail(m, SRMRA_EINVAL, "built-in denoiser needs L % 8 == 0");
  const cudaStream_t st = c->stream;
  if (iters > m->fcap) {
    double* p = nullptr;
    MCK(m, cudaMalloc((void**)&p, sizeof(double) * (size_t)iters));
    m->owned.push_back(p);
    m->fhist = p;
    m->fcap = iters;
  }
  double sbm = sigma_bm1;
  for (int t = 0; t < iters; ++t) {
    launch_step(m, 1, mu_x, mu_rho, m->fhist + t);
    MCK(m, cudaGetLastError());
    if (F > 0 && (t + 1) % F == 0) {
      const srmra_status s = srmra_project(c, sbm, fn, user);
      if (s != SRMRA_OK) return mfail(m, s, srmra_last_error(c));
      sbm *= decay;
    }
  }
  if (f_out && iters > 0)
    MCK(m, cudaMemcpyAsync(f_out, m->fhist, sizeof(double) * (size_t)iters,
                           cudaMemcpyDeviceToHost, st));
  return check_status(m);
}

void srmra_mom_destroy(srmra_mom* m) {
  if (!m) return;
  if (m->ctx) cudaStreamSynchronize(m->ctx->stream);
  for (void* p : m->owned) cudaFree(p);
  delete m;
}

const char* srmra_mom_last_error(const srmra_mom* m) {
  return m ? m->err.c_str() : g_mom_err.c_str();
}

}  // extern "C"
