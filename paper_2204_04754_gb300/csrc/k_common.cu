// Kernels shared by every precision form: observation centring, per-iteration
// operand preparation, the log-sum-exp combine, the M-step finalisation and the
// built-in block-DCT denoiser.
//
// Notation (Sec. 1-2 of the paper): x is L x L, K = L / l, the template of shift
// s = (s1, s2) is T_s = P R_s x with T_s[n] = x[(n1 K - s1) mod L, (n2 K - s2) mod L].
// Writing s = t K - r (mod L, per axis) with r = (-s) mod K, T_s is the low-resolution
// circular translate by t of the sub-image x_r[m] = x[r + m K] (proof of Theorem 1).
// The kernels use centred operands: y'_i = y_i - ybar_i and x'_r = x_r - m_r, which
// turns ||y_i - T_s||^2 into ||y'_i||^2 - 2 <y'_i, T'_s> + nu'_r + l^2 (ybar_i - m_r)^2
// with nu'_r = ||x'_r||^2 (exact algebra; it shrinks the operands of the contraction).
#include <math.h>

#include <algorithm>

#include <mutex>
#include <set>
#include <utility>

#include "srmra_internal.cuh"

namespace srmra {

cudaError_t once_per_device(int key, cudaError_t (*set)()) {
  static std::mutex mu;
  static std::set<std::pair<int, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({dev, key})) return cudaSuccess;
  e = set();
  if (e == cudaSuccess) done.insert({dev, key});
  return e;
}

namespace {

constexpr double kLog2e = 1.4426950408889634073599246810019;
constexpr double kLn2 = 0.69314718055994530941723212145818;

__device__ __forceinline__ int mod_pos(int a, int m) {
  int r = a % m;
  return r < 0 ? r + m : r;
}

// Block-wide float64 sum with a fixed reduction tree (deterministic).
template <int NT>
__device__ double block_sum_f64(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
#pragma unroll 1
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

// y'_i = y_i - mean(y_i); per-row mean and ||y'_i||^2 (float64 accumulation).
__global__ void __launch_bounds__(128) k_center_obs(const float* __restrict__ y, int l2,
                                                    int ldy, float* __restrict__ Yc,
                                                    float* __restrict__ ybar,
                                                    double* __restrict__ yy) {
  __shared__ double red[128];
  const int64_t i = blockIdx.x;
  const float* yi = y + i * (int64_t)l2;
  double s = 0.0;
  for (int n = threadIdx.x; n < l2; n += 128) s += (double)yi[n];
  const double mean = block_sum_f64<128>(s, red) / (double)l2;
  double q = 0.0;
  for (int n = threadIdx.x; n < ldy; n += 128) {
    float v = 0.f;
    if (n < l2) {
      const double d = (double)yi[n] - mean;
      v = (float)d;
      q += d * d;
    }
    Yc[i * ldy + n] = v;
  }
  const double qq = block_sum_f64<128>(q, red);
  if (threadIdx.x == 0) {
    ybar[i] = (float)mean;
    yy[i] = qq;
  }
}

// out[c][r] = in[r][c] for an R x C row-major matrix (32 x 32 tiles).
__global__ void k_transpose(const float* __restrict__ in, int64_t R, int64_t C,
                            float* __restrict__ out) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int64_t r = r0 + k, c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < R && c < C) ? in[r * C + c] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int64_t c = c0 + k, r = r0 + threadIdx.x;
    if (c < C && r < R) out[c * R + r] = tile[threadIdx.x][k];
  }
}

// Sub-image statistics: m_r = mean(x_r), nu'_r = ||x_r - m_r||^2 (float64).
__global__ void __launch_bounds__(256) k_sub_stats(const float* __restrict__ x, int L, int K,
                                                   int l, double* __restrict__ sub) {
  __shared__ double red[256];
  const int r = blockIdx.x, r1 = r / K, r2 = r % K, l2 = l * l;
  double s = 0.0;
  for (int m = threadIdx.x; m < l2; m += 256)
    s += (double)x[(r1 + (m / l) * K) * L + r2 + (m % l) * K];
  const double mean = block_sum_f64<256>(s, red) / (double)l2;
  double q = 0.0;
  for (int m = threadIdx.x; m < l2; m += 256) {
    const double d = (double)x[(r1 + (m / l) * K) * L + r2 + (m % l) * K] - mean;
    q += d * d;
  }
  const double nu = block_sum_f64<256>(q, red);
  if (threadIdx.x == 0) {
    sub[r] = mean;
    sub[K * K + r] = nu;
  }
}

// Column terms of the logit: colb[s] = log2(e) (-nu'_r / (2 sigma^2) + log rho1[s1] +
// log rho2[s2]), colm[s] = m_r.  Padding columns get -inf / 0.
__global__ void k_columns(const double* __restrict__ sub, const double* __restrict__ rho1,
                          const double* __restrict__ rho2, int L, int K, int S, int Spad,
                          double inv2s2, float* __restrict__ colb, float* __restrict__ colm) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Spad) return;
  if (s >= S) {
    colb[s] = -INFINITY;
    colm[s] = 0.f;
    return;
  }
  const int s1 = s / L, s2 = s % L;
  const int r = mod_pos(-s1, K) * K + mod_pos(-s2, K);
  const double lr = log(rho1[s1]) + log(rho2[s2]);  // -inf for a zero entry
  colb[s] = (float)(kLog2e * (lr - sub[K * K + r] * inv2s2));
  colm[s] = (float)sub[r];
}

// Centred templates, pixel-major: AxT[n][s] = x'_r(s)[n - t(s)] (zero for padding).
// Shift s = (s1, s2) has phase r = (-s1 mod K, -s2 mod K) and low-resolution lag
// t = ((s1 + r1) / K mod l, (s2 + r2) / K mod l); each thread holds one shift and walks
// the pixels n2 of row n1 = blockIdx.y (blockIdx.y = l writes the padding rows), so the
// index arithmetic is per shift, and the subtraction of the sub-image mean is float32
// (a rounding of the mean common to all pixels of a sub-image cancels in <y', T'>,
// since every y' sums to zero).
__global__ void k_templates_T(const float* __restrict__ x, const double* __restrict__ sub,
                              int L, int K, int l, int S, int Spad, int l2, int ldy,
                              float* __restrict__ AxT) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int n1 = blockIdx.y;
  if (s >= Spad) return;
  if (n1 == l) {  // padding rows
    for (int n = l2; n < ldy; ++n) AxT[(int64_t)n * Spad + s] = 0.f;
    return;
  }
  float* out = AxT + (int64_t)n1 * l * Spad + s;
  if (s >= S) {
    for (int n2 = 0; n2 < l; ++n2) out[(int64_t)n2 * Spad] = 0.f;
    return;
  }
  const int s1 = s / L, s2 = s % L;
  const int r1 = mod_pos(-s1, K), r2 = mod_pos(-s2, K);
  const int t1 = ((s1 + r1) / K) % l, t2 = ((s2 + r2) / K) % l;
  const int m1 = mod_pos(n1 - t1, l);
  const float mr = (float)sub[r1 * K + r2];
  const float* row = x + (r1 + m1 * K) * L + r2;
  int m2 = mod_pos(-t2, l);
  for (int n2 = 0; n2 < l; ++n2) {
    out[(int64_t)n2 * Spad] = row[m2 * K] - mr;
    if (++m2 == l) m2 = 0;
  }
}

// Combine the per-group (max, sum) partials of pass 1 into lse2[i] (base 2, of the
// centred logits) and the per-observation log-likelihood
//   lse[i] = ln 2 * lse2[i] - ||y'_i||^2 / (2 sigma^2)
// = log sum_s rho[s] exp(-||y_i - T_s||^2 / (2 sigma^2)); block partial sums in float64.
__global__ void __launch_bounds__(256) k_lse_combine(
    const float* __restrict__ pm, const float* __restrict__ ps, int groups, int64_t Npad,
    int64_t N, const double* __restrict__ yy, double inv2s2, float* __restrict__ lse2,
    double* __restrict__ lse, double* __restrict__ llpart) {
  __shared__ double red[256];
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  double ll = 0.0;
  if (i < N) {
    float m = -INFINITY;
    for (int gI = 0; gI < groups; ++gI) m = fmaxf(m, pm[gI * Npad + i]);
    // the group scale factors 2^(mg - m) lie in (0, 1]: float32 exp2 (float64
    // transcendentals are slow on this GPU), sums in float64
    double s = 0.0;
    if (m != -INFINITY)
      for (int gI = 0; gI < groups; ++gI) {
        const float mg = pm[gI * Npad + i];
        if (mg != -INFINITY) s += (double)ps[gI * Npad + i] * (double)exp2f(mg - m);
      }
    const double l2v = (double)m + log2(s);
    lse2[i] = (float)l2v;
    ll = kLn2 * l2v - yy[i] * inv2s2;
    lse[i] = ll;
  } else if (i < Npad) {
    lse2[i] = 0.f;
  }
  const double tot = block_sum_f64<256>(ll, red);
  if (threadIdx.x == 0) llpart[blockIdx.x] = tot;
}

// c_s = sum of the partial weight sums over the observation ranges, zb_s likewise
// (float64, fixed order).
__global__ void k_fin_sums(const float* __restrict__ cp, const float* __restrict__ zbp,
                           int nparts, int Spad, int S, double* __restrict__ cfin) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  double c = 0.0, z = 0.0;
#pragma unroll 8  // loads issued ahead; the additions keep their order
  for (int p = 0; p < nparts; ++p) {
    c += (double)cp[(int64_t)p * Spad + s];
    z += (double)zbp[(int64_t)p * Spad + s];
  }
  cfin[s] = c;
  cfin[Spad + s] = z;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// M-step totals in a fixed order, over K^2 + 1 blocks of 1024 threads:
//   blocks r < K^2: coverage A_r = sum_t c_{(r,t)} and ZB_r = sum_t zb_{(r,t)} of
//     sub-image r (each thread a few lags, then a block reduction);
//   block K^2: rho (Eq. rho_EM) = joint c_s / sum c with its marginals rho1 (rows) and
//     rho2 (columns), one warp per row / column, and LL(theta_t) = the sum of the
//     lse-combine block partials.
__global__ void __launch_bounds__(1024) k_fin_counts(
    const double* __restrict__ cfin, int Spad, int S, int L, int K, int l,
    const double* __restrict__ llpart, int ll_blocks, double* __restrict__ rho1,
    double* __restrict__ rho2, double* __restrict__ Ar, double* __restrict__ ll_out,
    int* __restrict__ status) {
  __shared__ double red[1024];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KK = K * K;
  if ((int)blockIdx.x < KK) {
    const int r = blockIdx.x, r1 = r / K, r2 = r % K, l2 = l * l;
    double a = 0.0, z = 0.0;
    for (int t = threadIdx.x; t < l2; t += 1024) {
      const int s1 = mod_pos((t / l) * K - r1, L), s2 = mod_pos((t % l) * K - r2, L);
      a += cfin[s1 * L + s2];
      z += cfin[Spad + s1 * L + s2];
    }
    a = block_sum_f64<1024>(a, red);
    z = block_sum_f64<1024>(z, red);
    if (threadIdx.x == 0) {
      Ar[r] = a;
      Ar[KK + r] = z;
    }
    return;
  }
  double loc = 0.0;
  for (int s = threadIdx.x; s < S; s += 1024) loc += cfin[s];
  const double ctot = block_sum_f64<1024>(loc, red);
  for (int j = warp; j < 2 * L; j += 32) {  // one warp per row (rho1) / column (rho2)
    double acc = 0.0;
    if (j < L)
      for (int k = lane; k < L; k += 32) acc += cfin[j * L + k];
    else
      for (int k = lane; k < L; k += 32) acc += cfin[k * L + (j - L)];
    acc = warp_sum_f64(acc);
    if (lane == 0) {
      if (j < L)
        rho1[j] = acc / ctot;
      else
        rho2[j - L] = acc / ctot;
    }
  }
  if (warp == 0) {
    double ll = 0.0;
    for (int b = lane; b < ll_blocks; b += 32) ll += llpart[b];
    ll = warp_sum_f64(ll);
    if (lane == 0) {
      *ll_out = ll;
      if (!isfinite(ll) || !(ctot > 0.0) || !isfinite(ctot)) atomicOr(status, STATUS_NUMERIC);
    }
  }
}

// Partial right-hand side of Eq. x_EM on sub-image r (pixel q = r + m K):
//   b'_r[m] = sum_t Z'[s(r,t)][(m + t) mod l],   s(r,t) = t K - r (mod L, per axis),
// over a range of lags t and all partial slices.  For a fixed (r, t) the row
// Z'[s(r,t)] is read contiguously and added at a circular offset, so the loads are
// coalesced.  Float32 with compensated (Kahan) summation; one partial per t-range.
__global__ void __launch_bounds__(256) k_fin_b(const float* __restrict__ Zp, int nparts, int Spad,
                                               int ldy, int L, int K, int l, int t_per,
                                               float* __restrict__ bpart) {
  constexpr int MPT = 4;  // pixels per thread per pass; the (lag, slice) arithmetic is shared
  const int r = blockIdx.x, ts = blockIdx.y;
  const int r1 = r / K, r2 = r % K, l2 = l * l;
  const int t0 = ts * t_per, t1 = min(l2, t0 + t_per);
  const int total = (t1 - t0) * nparts;  // (lag, slice) pairs of this range
  for (int mb = threadIdx.x; mb < l2; mb += 256 * MPT) {
    int m1[MPT], m2[MPT];
    float acc[MPT], comp[MPT];
#pragma unroll
    for (int k = 0; k < MPT; ++k) {
      const int m = mb + 256 * k;
      m1[k] = m < l2 ? m / l : 0;
      m2[k] = m < l2 ? m % l : 0;
      acc[k] = comp[k] = 0.f;
    }
    for (int j = 0; j < total; ++j) {
      const int t = t0 + j / nparts, p = j % nparts;
      const int tt1 = t / l, tt2 = t % l;
      const int s = mod_pos(tt1 * K - r1, L) * L + mod_pos(tt2 * K - r2, L);
      const float* row = Zp + ((int64_t)p * Spad + s) * ldy;
      float v[MPT];
#pragma unroll
      for (int k = 0; k < MPT; ++k) {  // independent loads, then the sums in order
        int a1 = m1[k] + tt1, a2 = m2[k] + tt2;
        a1 -= (a1 >= l) ? l : 0;
        a2 -= (a2 >= l) ? l : 0;
        v[k] = (mb + 256 * k < l2) ? row[a1 * l + a2] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < MPT; ++k) {
        const float y = v[k] - comp[k];
        const float tsum = acc[k] + y;
        comp[k] = (tsum - acc[k]) - y;
        acc[k] = tsum;
      }
    }
#pragma unroll
    for (int k = 0; k < MPT; ++k) {
      const int m = mb + 256 * k;
      if (m < l2) bpart[((int64_t)ts * K * K + r) * l2 + m] = acc[k];
    }
  }
}

// x_{t+1}[q] = (b'[q] + ZB_r) / A_r with b'[q] the fixed-order float64 sum of the
// lag-range partials (Eq. x_EM); a pixel with A_r = 0 keeps its value (uncovered pixel).
// One thread per (sub-image r, low-resolution pixel m): the partials are read coalesced.
// x = b / A per pixel q = r + m K of sub-image r (pixels with A = 0 keep their value):
// eight threads per pixel sum the t-range partials of b' (thread g takes partials g,
// g + 8, ...), then combine them with a fixed butterfly.
__global__ void __launch_bounds__(256) k_fin_x(const float* __restrict__ bpart, int n_ts, int L,
                                               int K, int l, const double* __restrict__ Ar,
                                               float* __restrict__ x, int* __restrict__ status) {
  const int l2 = l * l;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int idx = gid >> 3, g = gid & 7;  // idx = r * l2 + m
  const bool valid = idx < K * K * l2;
  double b = 0.0;
  if (valid)
    for (int ts = g; ts < n_ts; ts += 8) b += (double)bpart[(int64_t)ts * K * K * l2 + idx];
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
  if (!valid || g != 0) return;
  const int r = idx / l2, m = idx % l2;
  const int q = ((r / K) + (m / l) * K) * L + (r % K) + (m % l) * K;
  const double A = Ar[r];
  if (A > 0.0) {
    const double v = (b + Ar[K * K + r]) / A;
    x[q] = (float)v;
    if (!isfinite(v)) atomicOr(status, STATUS_NUMERIC);
  }
}

// Built-in denoiser: per 8x8 block, orthonormal 2D DCT-II in float64, DC kept, the AC
// coefficients thresholded at thr: hard (keep iff |c| > thr) or soft
// (c <- sign(c) max(|c| - thr, 0), the prox of thr * ||AC||_1).  The block grid is
// offset by (d1, d2): block pixel (u, v) of block (b1, b2) is image pixel
// ((8 b1 + u - d1) mod L, (8 b2 + v - d2) mod L).  Reads `in`, writes `out` (float or
// double); one block of 64 threads per 8x8 image block.
template <typename OutT>
__device__ __forceinline__ void dct8_block(const float* __restrict__ in, OutT* __restrict__ out,
                                           int L, double thr, int mode, int d1, int d2) {
  __shared__ double C[8][8], B[8][8], T[8][8];
  const int u = threadIdx.x >> 3, v = threadIdx.x & 7;
  const int b1 = blockIdx.x / (L / 8), b2 = blockIdx.x % (L / 8);
  C[u][v] = (u == 0 ? sqrt(0.125) : 0.5) * cospi((double)((2 * v + 1) * u) / 16.0);
  const int p1 = (b1 * 8 + u - d1 + L) % L, p2 = (b2 * 8 + v - d2 + L) % L;
  B[u][v] = (double)in[p1 * L + p2];
  __syncthreads();
  double a = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) a += C[u][k] * B[k][v];  // C B
  T[u][v] = a;
  __syncthreads();
  double X = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) X += T[u][k] * C[v][k];  // (C B) C^T
  double Xd;
  if (u == 0 && v == 0)
    Xd = X;
  else if (mode == 0)
    Xd = fabs(X) > thr ? X : 0.0;
  else
    Xd = (X > 0.0 ? 1.0 : (X < 0.0 ? -1.0 : 0.0)) * fmax(fabs(X) - thr, 0.0);
  __syncthreads();
  B[u][v] = Xd;
  __syncthreads();
  a = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) a += C[k][u] * B[k][v];  // C^T X
  T[u][v] = a;
  __syncthreads();
  double o = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) o += T[u][k] * C[k][v];  // (C^T X) C
  out[p1 * L + p2] = (OutT)o;
}

__global__ void __launch_bounds__(64) k_dct8(float* __restrict__ x, int L, double thr, int mode) {
  dct8_block<float>(x, x, L, thr, mode, 0, 0);
}

// Cycle spinning: the block denoiser for all 64 grid offsets (blockIdx.y = offset),
// each offset's full image into acc[offset][L*L] (float64).
__global__ void __launch_bounds__(64) k_dct8_spin(const float* __restrict__ x, int L,
                                                  double thr, int mode,
                                                  double* __restrict__ acc) {
  const int d = blockIdx.y;
  dct8_block<double>(x, acc + (int64_t)d * L * L, L, thr, mode, d / 8, d % 8);
}

// x[q] = mean over the 64 offsets (fixed order).
__global__ void k_spin_mean(const double* __restrict__ acc, int S, float* __restrict__ x) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= S) return;
  double m = 0.0;
  for (int d = 0; d < 64; ++d) m += acc[(int64_t)d * S + q];
  x[q] = (float)(m / 64.0);
}

// out = sum_{k<n} in[k] in float64, one warp, fixed order.
__global__ void k_sum_f64(const double* __restrict__ in, int n, double* __restrict__ out) {
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += 32) v += in[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) *out = v;
}

// Algorithm 2 step in device memory (for graph replay): project iff F > 0 and the
// iteration that just finished is the F-th, with threshold thr * sigma_BM.
__global__ void __launch_bounds__(64) k_dct8_sched(float* __restrict__ x, int L, double thr,
                                                   int mode, const DevSched* __restrict__ sc) {
  const int t = sc->t, F = sc->F;
  if (F <= 0 || (t + 1) % F != 0) return;
  dct8_block<float>(x, x, L, thr * sc->sigma_bm, mode, 0, 0);
}
__global__ void __launch_bounds__(64) k_dct8_spin_sched(const float* __restrict__ x, int L,
                                                        double thr, int mode,
                                                        const DevSched* __restrict__ sc,
                                                        double* __restrict__ acc) {
  const int t = sc->t, F = sc->F;
  if (F <= 0 || (t + 1) % F != 0) return;
  const int d = blockIdx.y;
  dct8_block<double>(x, acc + (int64_t)d * L * L, L, thr * sc->sigma_bm, mode, d / 8, d % 8);
}
__global__ void k_spin_mean_sched(const double* __restrict__ acc, int S, float* __restrict__ x,
                                  const DevSched* __restrict__ sc) {
  const int t = sc->t, F = sc->F;
  if (F <= 0 || (t + 1) % F != 0) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= S) return;
  double m = 0.0;
  for (int d = 0; d < 64; ++d) m += acc[(int64_t)d * S + q];
  x[q] = (float)(m / 64.0);
}

// Advance the schedule after an iteration: t <- t + 1, and decay sigma_BM if this
// iteration projected (Eq. decaying_function).
__global__ void k_sched_advance(DevSched* sc) {
  const int t = sc->t, F = sc->F;
  if (F > 0 && (t + 1) % F == 0) sc->sigma_bm *= sc->decay;
  sc->t = t + 1;
}

}  // namespace

// Number of lag ranges of the b' partial sums: about two blocks per SM.
int fin_t_splits(const Geom& g, int num_sms) {
  int n = (int)ceil_div(2 * (int64_t)num_sms, (int64_t)g.K * g.K);
  if (n > g.l2) n = g.l2;
  return n < 1 ? 1 : n;
}

cudaError_t launch_sum_f64(const double* in, int n, double* out, cudaStream_t stream) {
  k_sum_f64<<<1, 32, 0, stream>>>(in, n, out);
  return cudaGetLastError();
}

LogitScalars logit_scalars(const Geom& g) {
  LogitScalars s;
  const double inv_s2 = 1.0 / (g.sigma * g.sigma);
  s.a2 = (float)(kLog2e * inv_s2);
  s.c2 = (float)(kLog2e * (double)g.l2 * 0.5 * inv_s2);
  return s;
}

void launch_center_obs(srmra_ctx* c, const float* y_dev) {
  const Geom& g = c->g;
  k_center_obs<<<(unsigned)g.N, 128, 0, c->stream>>>(y_dev, g.l2, g.ldy, c->Yc, c->ybar, c->yy);
  c->launches++;
  if (c->YcT) {
    dim3 grid((unsigned)ceil_div(g.ldy, 32), (unsigned)ceil_div(g.Npad, 32));
    k_transpose<<<grid, dim3(32, 8), 0, c->stream>>>(c->Yc, g.Npad, g.ldy, c->YcT);
    c->launches++;
  }
}

void launch_prep_iter(srmra_ctx* c) {
  const Geom& g = c->g;
  k_sub_stats<<<g.K * g.K, 256, 0, c->stream>>>(c->x, g.L, g.K, g.l, c->sub);
  k_columns<<<(unsigned)ceil_div(g.Spad, 256), 256, 0, c->stream>>>(
      c->sub, c->rho1, c->rho2, g.L, g.K, g.S, g.Spad, 0.5 / (g.sigma * g.sigma), c->colb,
      c->colm);
  c->launches += 2;
  if (c->AxT) {
    dim3 grid((unsigned)ceil_div(g.Spad, 256), (unsigned)(g.l + 1));
    k_templates_T<<<grid, 256, 0, c->stream>>>(c->x, c->sub, g.L, g.K, g.l, g.S, g.Spad,
                                                g.l2, g.ldy, c->AxT);
    c->launches++;
  } else if (c->prec == SRMRA_FFT32) {
    launch_templates_fft(c);
  } else {
    launch_templates_tc(c);
  }
}

void launch_lse_combine(srmra_ctx* c, int groups) {
  const Geom& g = c->g;
  k_lse_combine<<<c->plan.ll_blocks, 256, 0, c->stream>>>(
      c->pm, c->ps, groups, g.Npad, g.N, c->yy, 0.5 / (g.sigma * g.sigma), c->lse2, c->lse,
      c->llpart);
  c->launches++;
}

int stats_t_splits(const srmra_ctx* c) {
  return c->prec == SRMRA_FFT32 ? 1 : fin_t_splits(c->g, c->num_sms);
}

// Zp[0][s][:] = sum_k Zp[k][s][:] over the nparts partial slices of pass 2 (s < S):
// float4 rows, one coalesced pass, so that the gather of k_fin_b reads a single slice.
// The slices are added in order with a compensated (Kahan) float32 sum; eight loads are
// issued before their additions so that the pass runs at memory speed.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}
__global__ void __launch_bounds__(256) k_sum_parts(float* __restrict__ Zp, int nparts,
                                                    int64_t slice, int64_t n4) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n4) return;
  const float4* base = reinterpret_cast<const float4*>(Zp) + q;
  const int64_t step = slice / 4;
  float4 s = base[0];
  float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k0 = 1; k0 < nparts; k0 += 8) {
    float4 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (k0 + j < nparts) v[j] = base[(int64_t)(k0 + j) * step];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (k0 + j < nparts) {
        kahan_add(s.x, c.x, v[j].x);
        kahan_add(s.y, c.y, v[j].y);
        kahan_add(s.z, c.z, v[j].z);
        kahan_add(s.w, c.w, v[j].w);
      }
  }
  reinterpret_cast<float4*>(Zp)[q] = s;
}

// The E-step sums of the iteration: c_s, zb_s (float64, cfin) and the partials of b'
// (bpart, stats_t_splits of them).
void launch_stats(srmra_ctx* c) {
  const Geom& g = c->g;
  k_fin_sums<<<(unsigned)ceil_div(g.S, 256), 256, 0, c->stream>>>(c->cp, c->zbp,
                                                                  c->plan.nparts_c, g.Spad,
                                                                  g.S, c->cfin);
  c->launches++;
  if (c->prec == SRMRA_FFT32) {
    launch_fin_b_fft(c);  // b' from the frequency-domain sums: one partial
  } else {
    int nparts = c->plan.nparts_z;
    if (nparts > 1) {
      const int64_t n4 = (int64_t)g.S * g.ldy / 4;  // ldy is a multiple of 16
      k_sum_parts<<<(unsigned)ceil_div(n4, 256), 256, 0, c->stream>>>(
          c->Zp, nparts, (int64_t)g.Spad * g.ldy, n4);
      c->launches++;
      nparts = 1;
    }
    const int n_ts = fin_t_splits(g, c->num_sms);
    const int t_per = (int)ceil_div(g.l2, n_ts);
    k_fin_b<<<dim3((unsigned)(g.K * g.K), (unsigned)n_ts), 256, 0, c->stream>>>(
        c->Zp, nparts, g.Spad, g.ldy, g.L, g.K, g.l, t_per, c->bpart);
    c->launches++;
  }
}

// M-step of Eqs. (x_EM), (rho_EM) from sums in the layout of launch_stats:
// rho, coverage, LL (from the lse-combine partials) and x.
void launch_mstep(srmra_ctx* c, const double* cfin, const float* bpart, int n_ts,
                  const double* llpart, int ll_blocks, double* rho1, double* rho2, double* Ar,
                  double* ll_out, float* x, int* status, cudaStream_t stream) {
  const Geom& g = c->g;
  k_fin_counts<<<(unsigned)(g.K * g.K + 1), 1024, 0, stream>>>(
      cfin, g.Spad, g.S, g.L, g.K, g.l, llpart, ll_blocks, rho1, rho2, Ar, ll_out, status);
  k_fin_x<<<(unsigned)ceil_div(8 * (int64_t)g.S, 256), 256, 0, stream>>>(bpart, n_ts, g.L, g.K,
                                                                         g.l, Ar, x, status);
  c->launches += 2;
}

void launch_finalize(srmra_ctx* c, int ll_index) {
  launch_stats(c);
  launch_mstep(c, c->cfin, c->bpart, stats_t_splits(c), c->llpart, c->plan.ll_blocks, c->rho1,
               c->rho2, c->Ar, c->ll_hist + ll_index, c->x, c->status, c->stream);
}

// The E-step statistics of launch_stats as one float64 vector (sums over the context's
// observations, so the vectors of disjoint shards of the data add):
//   [c_s (S) | zb_s (S) | b'_r[m] (K^2 l^2 = S, the partials summed in a fixed order) |
//    LL (1, the lse-combine partials summed in a fixed order)].
__global__ void k_pack_stats(const double* __restrict__ cfin, const float* __restrict__ bpart,
                             int n_ts, const double* __restrict__ llpart, int ll_blocks, int S,
                             int Spad, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < S) {
    out[j] = cfin[j];
    out[S + j] = cfin[Spad + j];
    double b = 0.0;
    for (int t = 0; t < n_ts; ++t) b += (double)bpart[(int64_t)t * S + j];
    out[2 * S + j] = b;
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {  // the same reduction tree as k_fin_counts
    const int lane = threadIdx.x;
    double ll = 0.0;
    for (int k = lane; k < ll_blocks; k += 32) ll += llpart[k];
    ll = warp_sum_f64(ll);
    if (lane == 0) out[3 * S] = ll;
  }
}

// The inverse layout for the M-step: c_s, zb_s into cfin; b' into partial 0 of bpart;
// LL into llpart[0].
__global__ void k_unpack_stats(const double* __restrict__ in, int S, int Spad,
                               double* __restrict__ cfin, float* __restrict__ bpart,
                               double* __restrict__ llpart) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < S) {
    cfin[j] = in[j];
    cfin[Spad + j] = in[S + j];
    bpart[j] = (float)in[2 * S + j];
  }
  if (j == 0) llpart[0] = in[3 * S];
}

void launch_pack_stats(srmra_ctx* c, double* out) {
  const Geom& g = c->g;
  k_pack_stats<<<(unsigned)ceil_div(g.S, 256), 256, 0, c->stream>>>(
      c->cfin, c->bpart, stats_t_splits(c), c->llpart, c->plan.ll_blocks, g.S, g.Spad, out);
  c->launches++;
}

void launch_unpack_stats(srmra_ctx* c, const double* in) {
  const Geom& g = c->g;
  k_unpack_stats<<<(unsigned)ceil_div(g.S, 256), 256, 0, c->stream>>>(in, g.S, g.Spad, c->cfin,
                                                                       c->bpart, c->llpart);
  c->launches++;
}

void launch_dct_sched(srmra_ctx* c, double thr) {
  const Geom& g = c->g;
  const unsigned nb = (unsigned)((g.L / 8) * (g.L / 8));
  if (g.L % 8 == 0) {
    if (c->dn_spin && c->dn_acc) {
      k_dct8_spin_sched<<<dim3(nb, 64), 64, 0, c->stream>>>(c->x, g.L, c->dn_thr, c->dn_mode,
                                                             c->d_sched, c->dn_acc);
      k_spin_mean_sched<<<(unsigned)ceil_div(g.S, 256), 256, 0, c->stream>>>(c->dn_acc, g.S,
                                                                              c->x, c->d_sched);
      c->launches += 2;
    } else {
      k_dct8_sched<<<nb, 64, 0, c->stream>>>(c->x, g.L, c->dn_thr, c->dn_mode, c->d_sched);
      c->launches++;
    }
  }
  (void)thr;
  k_sched_advance<<<1, 1, 0, c->stream>>>(c->d_sched);
  c->launches++;
}

void launch_dct_denoise(srmra_ctx* c, double sigma_bm, double thr) {
  const Geom& g = c->g;
  const unsigned nb = (unsigned)((g.L / 8) * (g.L / 8));
  (void)thr;
  if (c->dn_spin && c->dn_acc) {
    k_dct8_spin<<<dim3(nb, 64), 64, 0, c->stream>>>(c->x, g.L, c->dn_thr * sigma_bm,
                                                    c->dn_mode, c->dn_acc);
    k_spin_mean<<<(unsigned)ceil_div(g.S, 256), 256, 0, c->stream>>>(c->dn_acc, g.S, c->x);
    c->launches += 2;
  } else {
    k_dct8<<<nb, 64, 0, c->stream>>>(c->x, g.L, c->dn_thr * sigma_bm, c->dn_mode);
    c->launches++;
  }
}

}  // namespace srmra
