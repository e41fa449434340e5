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
#include <atomic>
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
  const float* A;        // [K][lda], element (k, m); lda % 4 == 0, 16-byte aligned
  int lda, Mvalid;
  const float* B;        // [K][ldb], element (k, n); ldb % 4 == 0, 16-byte aligned
  int ldb, Nvalid;
  int Kvalid, kchunk;    // split z covers k in [z kchunk, min(Kvalid, (z + 1) kchunk))
  float* C;              // [split][Mpad][ldc]
  int ldc;
  int64_t c_split;       // elements between splits
  int sym;               // 1: C is symmetric; only the tiles (bi <= bj) of an nt x nt tile
  int nt;                //    grid are computed, enumerated row by row by blockIdx.x
};

// 16-byte asynchronous copy global -> shared that reads `bytes` (0..16) and zero-fills the
// rest; with bytes == 0 nothing is read.
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

constexpr int GK = 16;     // k rows per stage
constexpr int GSTAGE = 3;  // stages in flight

// C[m][n] = sum_k A[k][m] B[k][n] over one 128 x 128 tile and one k range: 256 threads
// with 8 x 8 outputs each (packed FMA), operands staged GK rows at a time through a
// GSTAGE-deep cp.async ring.  Rows and columns past Mvalid / Nvalid and k past the range
// read as zero (zero-filled copies); the whole tile is written.
__global__ void __launch_bounds__(256) k_mom_gemm(GemmArgs g) {
  __shared__ __align__(16) float As[GSTAGE][GK][GT];
  __shared__ __align__(16) float Bs[GSTAGE][GK][GT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int bi = blockIdx.x, bj = blockIdx.y;
  if (g.sym) {
    int t = blockIdx.x;
    bi = 0;
    while (t >= g.nt - bi) {
      t -= g.nt - bi;
      ++bi;
    }
    bj = bi + t;
  }
  const int m0 = bi * GT, n0 = bj * GT;
  const int k0 = blockIdx.z * g.kchunk, k1 = min(g.Kvalid, k0 + g.kchunk);
  const int nk = k1 > k0 ? (k1 - k0 + GK - 1) / GK : 0;
  // each thread copies two 16-byte chunks of A and two of B per stage
  auto issue = [&](int it) {
    const int st = it % GSTAGE;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = tid + h * 256, row = c >> 5, col = (c & 31) * 4;
      const int k = k0 + it * GK + row;
      const bool kv = k < k1;
      const int va = kv ? max(0, min(4, g.Mvalid - (m0 + col))) : 0;
      const int vb = kv ? max(0, min(4, g.Nvalid - (n0 + col))) : 0;
      cp_async16(&As[st][row][col], va ? g.A + (int64_t)k * g.lda + m0 + col : g.A, va * 4);
      cp_async16(&Bs[st][row][col], vb ? g.B + (int64_t)k * g.ldb + n0 + col : g.B, vb * 4);
    }
  };
  f2 acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[j][c] = 0ull;
#pragma unroll
  for (int it = 0; it < GSTAGE - 1; ++it) {
    if (it < nk) issue(it);
    cp_async_commit();
  }
  for (int it = 0; it < nk; ++it) {
    cp_async_wait<GSTAGE - 2>();
    __syncthreads();
    if (it + GSTAGE - 1 < nk) issue(it + GSTAGE - 1);
    cp_async_commit();
    const int st = it % GSTAGE;
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[st][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[st][kk][64 + ty * 4]);
      const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(&Bs[st][kk][tx * 4]);
      const ulonglong2 b1 = *reinterpret_cast<const ulonglong2*>(&Bs[st][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const f2 b[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const f2 aj = dup2(a[j]);
#pragma unroll
        for (int c = 0; c < 4; ++c) ffma2(acc[j][c], aj, b[c]);
      }
    }
  }
  cp_async_wait<0>();
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

// Column sums of the centred observations for the moments, per row split z:
//   part[z][n]       = sum_i y'_i[n],   part[z][l2 + n] = sum_i ybar_i y'_i[n],
//   part[z][2 l2]    = sum_i ybar_i,    part[z][2 l2 + 1] = sum_i ybar_i^2
// (float32 inside a split of at most 256 rows in four interleaved chains, float64 across
// chains).
__global__ void k_mom_colsum(const float* __restrict__ Y, int ldy, int l2,
                             const float* __restrict__ ybar, int64_t rows, int64_t chunk,
                             double* __restrict__ part) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t k0 = blockIdx.y * chunk, k1 = rows < k0 + chunk ? rows : k0 + chunk;
  double* out = part + (int64_t)blockIdx.y * (2 * l2 + 2);
  if (n < l2) {
    float a[4] = {0.f, 0.f, 0.f, 0.f}, b[4] = {0.f, 0.f, 0.f, 0.f};
    int64_t k = k0;
    for (; k + 4 <= k1; k += 4) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float v = Y[(k + j) * ldy + n];
        a[j] += v;
        b[j] = fmaf(ybar[k + j], v, b[j]);
      }
    }
    for (int j = 0; k < k1; ++k, ++j) {
      const float v = Y[k * ldy + n];
      a[j] += v;
      b[j] = fmaf(ybar[k], v, b[j]);
    }
    out[n] = ((double)a[0] + a[1]) + ((double)a[2] + a[3]);
    out[l2 + n] = ((double)b[0] + b[1]) + ((double)b[2] + b[3]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0, q = 0.0;
    for (int64_t k = k0; k < k1; ++k) {
      const double v = (double)ybar[k];
      s += v;
      q += v * v;
    }
    out[2 * l2] = s;
    out[2 * l2 + 1] = q;
  }
}

// The consumers of a symmetric product walk the 32 x 32 tiles (ti <= tj) of its upper
// triangle (inside the computed 128 x 128 tiles), one block of 32 x 8 threads per tile,
// and write the mirrored tile through shared memory.
__device__ __forceinline__ void upper_tile(int nt32, int& ti, int& tj) {
  int t = blockIdx.x;
  ti = 0;
  while (t >= nt32 - ti) {
    t -= nt32 - ti;
    ++ti;
  }
  tj = ti + t;
}

// The column sums of k_mom_colsum reduced over the splits in a fixed order:
// cs[n] = sum_i y'_i[n], cs[l2 + n] = sum_i ybar_i y'_i[n], cs[2 l2] = sum_i ybar_i,
// cs[2 l2 + 1] = sum_i ybar_i^2.
__global__ void k_mom_colsum_fin(const double* __restrict__ part, int nsplit, int l2,
                                 double* __restrict__ cs) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int w = 2 * l2 + 2;
  if (n >= w) return;
  double s = 0.0;
  for (int p = 0; p < nsplit; ++p) s += part[(int64_t)p * w + n];
  cs[n] = s;
}

// Empirical second moment from the split partials of Y'^T Y' (y_i = y'_i + ybar_i 1):
//   M2^[r][c] = (sum_i y'_i[r] y'_i[c] + v[r] + v[c] + q) / N,
//   v = sum_i ybar_i y'_i,  q = sum_i ybar_i^2   (float64);
// and M1^[n] = (sum_i y'_i[n] + sum_i ybar_i) / N.
__global__ void __launch_bounds__(256) k_mom_hat(const float* __restrict__ part, int nsplit,
                                                 int64_t split_stride, int l2, int l2p,
                                                 const double* __restrict__ cs, double inv_n,
                                                 double* __restrict__ M2h,
                                                 double* __restrict__ M1h) {
  __shared__ double tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  int ti, tj;
  upper_tile(l2p / 32, ti, tj);
  const double q = cs[2 * l2 + 1];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = ti * 32 + ty + 8 * j, c = tj * 32 + tx;
    double s = 0.0;
    if (r < l2 && c < l2) {
      for (int p = 0; p < nsplit; ++p) s += (double)part[p * split_stride + (int64_t)r * l2p + c];
      s = (s + (cs[l2 + r] + cs[l2 + c]) + q) * inv_n;  // symmetric in (r, c) bit for bit
      M2h[(int64_t)r * l2 + c] = s;
    }
    tile[ty + 8 * j][tx] = s;
  }
  if (ti != tj) {
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = tj * 32 + ty + 8 * j, c = ti * 32 + tx;
      if (r < l2 && c < l2) M2h[(int64_t)r * l2 + c] = tile[tx][ty + 8 * j];
    }
  }
  const int n = blockIdx.x * 256 + threadIdx.x;  // the first blocks also write M1^
  if (n < l2) M1h[n] = (cs[n] + cs[2 * l2]) * inv_n;
}

// Templates t_s = P R_s x, t_s[n1 l + n2] = x[(n1 K - s1) mod L][(n2 K - s2) mod L], in the
// layouts T[s][n], TS[s][n] = rho_s t_s[n] and TT[n][s] (zero padding), one block of
// 32 x 8 threads per 32 x 32 (shift, pixel) tile, the transposed copy through shared
// memory; and the joint prior rho_s = rho1[s1] rho2[s2] (float, zero padding).
__global__ void __launch_bounds__(256) k_mom_templates(
    const float* __restrict__ x, const double* __restrict__ rho1, const double* __restrict__ rho2,
    int L, int K, int l, int S, int Spad, int l2p, float* __restrict__ T, float* __restrict__ TS,
    float* __restrict__ TT, float* __restrict__ rho) {
  __shared__ float tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int s0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int s = s0 + ty + 8 * j, n = n0 + tx;
    float v = 0.f, r = 0.f;
    if (s < S && n < l * l) {
      const int s1 = s / L, s2 = s % L, n1 = n / l, n2 = n % l;
      v = x[((n1 * K - s1) % L + L) % L * L + ((n2 * K - s2) % L + L) % L];
      r = (float)(rho1[s1] * rho2[s2]);
    }
    T[(int64_t)s * l2p + n] = v;
    TS[(int64_t)s * l2p + n] = r * v;
    tile[ty + 8 * j][tx] = v;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n = n0 + ty + 8 * j, s = s0 + tx;
    TT[(int64_t)n * Spad + s] = tile[tx][ty + 8 * j];
  }
  if (blockIdx.y == 0 && ty == 0) {
    const int s = s0 + tx;
    rho[s] = s < S ? (float)(rho1[s / L] * rho2[s % L]) : 0.f;
  }
}

// M1 = sum_s rho_s t_s in separable form (float64):
//   Y1[q1][n2] = sum_{s2} rho2[s2] x[q1][(n2 K - s2) mod L]                (k_mom_m1_rows)
//   M1[n1][n2] = sum_{s1} rho1[s1] Y1[(n1 K - s1) mod L][n2],  r = M1 - M1^   (k_mom_m1)
__global__ void k_mom_m1_rows(const float* __restrict__ x, const double* __restrict__ rho2,
                              int L, int K, int l, double* __restrict__ Y1) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L * l) return;
  const int q1 = j / l, n2 = j % l;
  double a = 0.0;
#pragma unroll 8
  for (int s2 = 0; s2 < L; ++s2) a += rho2[s2] * (double)x[q1 * L + ((n2 * K - s2) % L + L) % L];
  Y1[j] = a;
}

__global__ void k_mom_m1(const double* __restrict__ Y1, const double* __restrict__ rho1, int L,
                         int K, int l, const double* __restrict__ M1h, double* __restrict__ r1) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= l * l) return;
  const int n1 = n / l, n2 = n % l;
  double a = 0.0;
#pragma unroll 8
  for (int s1 = 0; s1 < L; ++s1) a += rho1[s1] * Y1[((n1 * K - s1) % L + L) % L * l + n2];
  r1[n] = a - M1h[n];
}

// R = M2 - M2^ (float32, zero padding; both triangles) and the block partials of
// ||R||_F^2 (an off-diagonal tile counts twice).
__global__ void __launch_bounds__(256) k_mom_residual(const float* __restrict__ part, int nsplit,
                                                      int64_t split_stride, int l2, int l2p,
                                                      double sigma2, const double* __restrict__ M2h,
                                                      float* __restrict__ R,
                                                      double* __restrict__ fpart) {
  __shared__ float tile[32][33];
  __shared__ double red[256];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  int ti, tj;
  upper_tile(l2p / 32, ti, tj);
  double f = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = ti * 32 + ty + 8 * j, c = tj * 32 + tx;
    float rv = 0.f;
    if (r < l2 && c < l2) {
      // the split partials in float32 pairs (each already float32-rounded), then float64
      const float* pp = part + (int64_t)r * l2p + c;
      double s = 0.0;
      int p = 0;
      for (; p + 2 <= nsplit; p += 2) s += (double)(pp[p * split_stride] + pp[(p + 1) * split_stride]);
      if (p < nsplit) s += (double)pp[p * split_stride];
      const double d = s + (r == c ? sigma2 : 0.0) - M2h[(int64_t)r * l2 + c];
      f += d * d;
      rv = (float)d;
    }
    R[(int64_t)r * l2p + c] = rv;
    tile[ty + 8 * j][tx] = rv;
  }
  if (ti != tj) {
    f *= 2.0;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = tj * 32 + ty + 8 * j, c = ti * 32 + tx;
      R[(int64_t)r * l2p + c] = tile[tx][ty + 8 * j];
    }
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
  const float rs = rho[s], lam2 = (float)(2.0 * lambda);
  float af = 0.f, bf = 0.f;  // per-lane partial dot products (float32), float64 across lanes
#pragma unroll 4
  for (int n = lane; n < l2; n += 32) {
    float u = 0.f;
    for (int p = 0; p < nsplit; ++p) u += Upart[p * split_stride + (int64_t)s * l2p + n];
    const float t = T[(int64_t)s * l2p + n];
    const float rn = (float)r1[n];
    af = fmaf(u, t, af);
    bf = fmaf(t, rn, bf);
    W[(int64_t)s * l2p + n] = rs * fmaf(4.f, u, lam2 * rn);
  }
  double a = af, b = bf;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) gs[s] = 2.0 * a + 2.0 * lambda * b;
}

// Partial df/dx over a range of n1: gxp[z][q1 L + q2] = sum_{n1 in range z, n2}
// W[s(n1, q1) L + s(n2, q2)][n1 l + n2] with s(n, q) = (n K - q) mod L per axis (the
// adjoint of t_s = P R_s x).  One block per (row q1, range z); for each n1 and each
// 32-column chunk of n2 the slab of all L shifts s2 is staged in shared memory (pitch 33)
// so that the global reads are row-contiguous.
constexpr int GX_THREADS = 256;
constexpr int GX_MAXQ = 4;  // L <= GX_THREADS * GX_MAXQ
__global__ void __launch_bounds__(GX_THREADS) k_mom_gx(const float* __restrict__ W, int L, int K,
                                                       int l, int l2p, int nz,
                                                       double* __restrict__ gxp) {
  extern __shared__ float slab[];  // [L][33]
  const int q1 = blockIdx.x, z = blockIdx.y, tid = threadIdx.x;
  const int na = z * l / nz, nb = (z + 1) * l / nz;
  double acc[GX_MAXQ];
#pragma unroll
  for (int j = 0; j < GX_MAXQ; ++j) acc[j] = 0.0;
  for (int n1 = na; n1 < nb; ++n1) {
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
          float a = 0.f;  // at most 32 terms in float32, then float64
          int s2 = ((c0 * K - q2) % L + L) % L;  // (n2 K - q2) mod L, stepped by K
          for (int j = 0; j < cw; ++j) {
            a += slab[s2 * 33 + j];
            s2 += K;
            if (s2 >= L) s2 -= L;
          }
          acc[jq] += (double)a;
        }
      }
    }
  }
#pragma unroll
  for (int jq = 0; jq < GX_MAXQ; ++jq) {
    const int q2 = tid + jq * GX_THREADS;
    if (q2 < L) gxp[(int64_t)z * L * L + (int64_t)q1 * L + q2] = acc[jq];
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

// df/dx = the sum of the nz partials (fixed order) into gx; with apply,
// x <- x - mu_x df/dx.  One thread per pixel.
__global__ void k_mom_xstep(const double* __restrict__ gxp, int nz, int S, int apply,
                            double mu_x, float* __restrict__ x, double* __restrict__ gx) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= S) return;
  double g = 0.0;
  for (int z = 0; z < nz; ++z) g += gxp[(int64_t)z * S + q];
  gx[q] = g;
  if (apply) x[q] = (float)((double)x[q] - mu_x * g);
}

// f = ||R||^2 (block partials) + lambda ||r||^2 into f_out; df/drho1 = G rho2 and
// df/drho2 = G^T rho1 into g12 (both at the current rho); with apply, rho1, rho2 <- their
// simplex projections after a step mu_rho.  One block of 1024 threads (L <= 1024).
__global__ void __launch_bounds__(1024) k_mom_step(
    const double* __restrict__ fpart, int nfp, const double* __restrict__ r1, int l2,
    double lambda, const double* __restrict__ gs, int L, int apply, double mu_rho,
    double* __restrict__ rho1, double* __restrict__ rho2, double* __restrict__ g12,
    double* __restrict__ f_out, int* __restrict__ status) {
  __shared__ double red[1024], v1[1024], v2[1024], css[1024];
  __shared__ int kk[1024];
  __shared__ double tau;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double f = 0.0;
  for (int k = t; k < nfp; k += 1024) f += fpart[k];
  for (int n = t; n < l2; n += 1024) f += lambda * r1[n] * r1[n];
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
  // df/drho1[a] = sum_b G[a][b] rho2[b]: one warp per row a (row-contiguous reads)
  for (int a = warp; a < L; a += 32) {
    double g = 0.0;
#pragma unroll 4
    for (int b = lane; b < L; b += 32) g += gs[(int64_t)a * L + b] * rho2[b];
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    if (lane == 0) {
      g12[a] = g;
      v1[a] = rho1[a] - mu_rho * g;
    }
  }
  // df/drho2[b] = sum_a G[a][b] rho1[a]: one thread per column b
  if (t < L) {
    double g = 0.0;
#pragma unroll 8
    for (int a = 0; a < L; ++a) g += gs[(int64_t)a * L + t] * rho1[a];
    g12[L + t] = g;
    v2[t] = rho2[t] - mu_rho * g;
  }
  __syncthreads();
  if (!apply) return;
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
  int ns_c1 = 1;                     // row splits of the observation column sum
  int nz = 1;                        // n1 ranges of the df/dx gather
  double lambda = 0.0;
  double* M2h = nullptr;    // [l2][l2]
  double* M1h = nullptr;    // [l2]
  float* T = nullptr;       // [Spad][l2p]
  float* TS = nullptr;      // [Spad][l2p] rho_s t_s
  float* TT = nullptr;      // [l2p][Spad]
  float* rho = nullptr;     // [Spad]
  float* part = nullptr;    // split partials of the products
  double* part1 = nullptr;  // split partials of the observation column sums [ns_c1][2 l2 + 2]
  double* cs = nullptr;     // [2 l2 + 2] their totals
  double* Y1 = nullptr;     // [L][l] first stage of M1
  float* R = nullptr;       // [l2p][l2p]
  float* W = nullptr;       // [Spad][l2p] back-projection operand
  double* r1 = nullptr;     // [l2]
  double* fpart = nullptr;  // [nfp]
  int nfp = 0;
  double* gs = nullptr;     // [S]
  double* gx = nullptr;     // [L*L]
  double* gxp = nullptr;    // [nz][L*L] partials of df/dx
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

// Co-resident blocks of the product kernel on the device (SMs x blocks per SM).
int gemm_slots(int sms) {
  // occupancy of a kernel without opt-in shared memory: the same on every GB300
  static std::atomic<int> per_sm{0};
  int b = per_sm.load();
  if (b == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mom_gemm, 256, 0) != cudaSuccess ||
        b < 1)
      b = 1;
    per_sm.store(b);
  }
  return b * sms;
}

// k splits of a product with `tiles` output tiles: as many as keep all blocks in one
// wave of co-resident blocks (no partly filled second wave), at least 256 k per split.
int product_splits(int64_t tiles, int64_t kdim, int slots) {
  int64_t s = slots / tiles;
  s = std::min(s, (kdim + 255) / 256);
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

int tri(int n) { return n * (n + 1) / 2; }

void gemm(srmra_mom* m, const GemmArgs& a, int Mpad, int Npad, int nsplit, cudaStream_t st) {
  const dim3 grid = a.sym ? dim3((unsigned)tri(a.nt), 1u, (unsigned)nsplit)
                          : dim3((unsigned)(Mpad / GT), (unsigned)(Npad / GT), (unsigned)nsplit);
  k_mom_gemm<<<grid, 256, 0, st>>>(a);
  m->ctx->launches++;
}



// The empirical moments of the context's observations.
void launch_moments(srmra_mom* m) {
  srmra_ctx* c = m->ctx;
  const Geom& g = c->g;
  const cudaStream_t st = c->stream;
  const int l2p = m->l2p;
  // Y'^T Y' (upper-triangle tiles), the column sums for the ybar terms, then M2^ and M1^
  GemmArgs a{c->Yc, g.ldy, g.l2, c->Yc, g.ldy, g.l2, (int)g.N, (int)ceil_div(g.N, m->ns_y),
             m->part, l2p, (int64_t)l2p * l2p, 1, l2p / GT};
  gemm(m, a, l2p, l2p, m->ns_y, st);
  k_mom_colsum<<<dim3((unsigned)ceil_div(g.l2, 256), (unsigned)m->ns_c1), 256, 0, st>>>(
      c->Yc, g.ldy, g.l2, c->ybar, g.N, ceil_div(g.N, m->ns_c1), m->part1);
  k_mom_colsum_fin<<<(unsigned)ceil_div(2 * g.l2 + 2, 256), 256, 0, st>>>(m->part1, m->ns_c1,
                                                                          g.l2, m->cs);
  k_mom_hat<<<(unsigned)tri(l2p / 32), 256, 0, st>>>(m->part, m->ns_y, (int64_t)l2p * l2p, g.l2,
                                                     l2p, m->cs, 1.0 / (double)g.N, m->M2h,
                                                     m->M1h);
  c->launches += 3;
}

// f and the gradient at the context's theta; with apply, the projected gradient step.
void launch_step(srmra_mom* m, int apply, double mu_x, double mu_rho, double* f_out) {
  srmra_ctx* c = m->ctx;
  const Geom& g = c->g;
  const cudaStream_t st = c->stream;
  const int l2p = m->l2p;
  k_mom_templates<<<dim3((unsigned)(g.Spad / 32), (unsigned)(l2p / 32)), 256, 0, st>>>(
      c->x, c->rho1, c->rho2, g.L, g.K, g.l, g.S, g.Spad, l2p, m->T, m->TS, m->TT, m->rho);
  // M1 = T^T rho (separable form) and r = M1 - M1^
  k_mom_m1_rows<<<(unsigned)ceil_div((int64_t)g.L * g.l, 128), 128, 0, st>>>(c->x, c->rho2, g.L,
                                                                            g.K, g.l, m->Y1);
  k_mom_m1<<<(unsigned)ceil_div(g.l2, 128), 128, 0, st>>>(m->Y1, c->rho1, g.L, g.K, g.l, m->M1h,
                                                          m->r1);
  c->launches += 3;
  // M2 - sigma^2 I = T^T diag(rho) T, then R = M2 - M2^ and ||R||^2
  GemmArgs a2{m->TS, l2p, g.l2, m->T, l2p, g.l2, g.S, (int)ceil_div(g.S, m->ns_t), m->part,
              l2p, (int64_t)l2p * l2p, 1, l2p / GT};
  gemm(m, a2, l2p, l2p, m->ns_t, st);
  k_mom_residual<<<(unsigned)m->nfp, 256, 0, st>>>(m->part, m->ns_t, (int64_t)l2p * l2p, g.l2,
                                                   l2p, g.sigma * g.sigma, m->M2h, m->R,
                                                   m->fpart);
  // U = T R (rows R t_s), then the shift gradient and the back-projection operand
  GemmArgs au{m->TT, g.Spad, g.S, m->R, l2p, g.l2, g.l2, (int)ceil_div(g.l2, m->ns_u), m->part,
              l2p, (int64_t)m->Mpad_u * l2p, 0, 0};
  gemm(m, au, m->Mpad_u, l2p, m->ns_u, st);
  k_mom_gshift<<<(unsigned)ceil_div(g.S, 8), 256, 0, st>>>(
      m->part, m->ns_u, (int64_t)m->Mpad_u * l2p, m->T, m->rho, g.l2, l2p, g.S, m->r1,
      m->lambda, m->gs, m->W);
  k_mom_gx<<<dim3((unsigned)g.L, (unsigned)m->nz), GX_THREADS, m->gx_smem, st>>>(
      m->W, g.L, g.K, g.l, l2p, m->nz, m->gxp);
  // rho first: its gradient reads nothing the x step writes
  k_mom_step<<<1, 1024, 0, st>>>(m->fpart, m->nfp, m->r1, g.l2, m->lambda, m->gs, g.L, apply,
                                 mu_rho, c->rho1, c->rho2, m->g12, f_out, m->status);
  k_mom_xstep<<<(unsigned)ceil_div(g.S, 256), 256, 0, st>>>(m->gxp, m->nz, g.S, apply, mu_x, c->x,
                                                           m->gx);
  c->launches += 5;
}

srmra_status check_status(srmra_mom* m) {
  int status = 0;
  MCK(m, cudaMemcpyAsync(&status, m->status, sizeof(int), cudaMemcpyDeviceToHost,
                         m->ctx->stream));
  MCK(m, cudaStreamSynchronize(m->ctx->stream));
  if (status) {  // reported once, then cleared (as for a context's status word)
    MCK(m, cudaMemsetAsync(m->status, 0, sizeof(int), m->ctx->stream));
    if (status & STATUS_NUMERIC) return mfail(m, SRMRA_ENUMERIC, "NaN or Inf in the objective");
  }
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
  const int slots = gemm_slots(sms);
  const int64_t tiles2 = tri(l2p / GT);  // symmetric products: upper-triangle tiles
  m->ns_y = product_splits(tiles2, g.N, slots);
  m->ns_t = product_splits(tiles2, g.S, slots);
  m->ns_u = product_splits((int64_t)(m->Mpad_u / GT) * (l2p / GT), g.l2, slots);
  m->ns_c1 = (int)std::max<int64_t>(colsum_splits(g.l2, g.N, sms), ceil_div(g.N, 256));
  m->nz = (int)std::min<int64_t>(g.l, ceil_div(4 * (int64_t)sms, g.L));
  const int64_t part = std::max({(int64_t)m->ns_y * l2p * l2p, (int64_t)m->ns_t * l2p * l2p,
                                 (int64_t)m->ns_u * m->Mpad_u * l2p});
  m->nfp = tri(l2p / 32);  // one f partial per upper-triangle 32 x 32 tile
  m->gx_smem = sizeof(float) * (size_t)g.L * 33;
  cudaError_t e = mget(m, &m->M2h, (int64_t)g.l2 * g.l2);
  if (e == cudaSuccess) e = mget(m, &m->M1h, g.l2);
  if (e == cudaSuccess) e = mget(m, &m->T, (int64_t)g.Spad * l2p);
  if (e == cudaSuccess) e = mget(m, &m->TT, (int64_t)l2p * g.Spad);
  if (e == cudaSuccess) e = mget(m, &m->rho, g.Spad);
  if (e == cudaSuccess) e = mget(m, &m->part, part);
  if (e == cudaSuccess) e = mget(m, &m->part1, (int64_t)m->ns_c1 * (2 * g.l2 + 2));
  if (e == cudaSuccess) e = mget(m, &m->cs, 2 * (int64_t)g.l2 + 2);
  if (e == cudaSuccess) e = mget(m, &m->TS, (int64_t)g.Spad * l2p);
  if (e == cudaSuccess) e = mget(m, &m->Y1, (int64_t)g.L * g.l);
  if (e == cudaSuccess) e = mget(m, &m->gxp, (int64_t)m->nz * g.S);
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
