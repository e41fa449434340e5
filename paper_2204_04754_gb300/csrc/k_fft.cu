// Float32 polyphase-FFT form of the E-step and M-step contractions (SRMRA_FFT32).
//
// With the K^2 sub-images x_r[m] = x[r1 + m1 K, r2 + m2 K] (r in [0,K)^2, m in [0,l)^2),
// the template of shift s = t K - r (mod L, per axis) is the low-resolution circular
// translate of x_r by t: (P R_s x)[n] = x_r[n - t] (the polyphase structure behind
// Theorem 1 of Sec. 2).  Hence, with centred observations y'_i and sub-images x'_r,
//   <y'_i, T'_s> = corr_{i,r}[t] = IFFT2( FFT2(y'_i) . conj(FFT2(x'_r)) )[t] / l^2,
// and the M-step right-hand side of Eq. (x_EM) on sub-image r is the correlation
//   b'_r[m] = sum_i sum_t w^{i,(r,t)} y'_i[m + t] = IFFT2( sum_i conj(FFT2(w_{i,r})) .
//             FFT2(y'_i) )[m] / l^2,
// so neither the L^2 x l^2 templates nor the N x L^2 weights are ever formed.  The
// logits use the same centred expression as the dense forms,
//   logit2[i,s] = a2 <y'_i, T'_s> + colb[s] - c2 (ybar_i - m_r)^2     (Eq. weights_EM),
// and the partial outputs have the layouts the dense forms use (pass-1 (max, sum)
// partials per phase, c / zb partials per shift), so the combine and finalize kernels
// are shared; only b' comes from the frequency-domain sums.
//
// Accuracy: the float32 rounding of these correlations was measured against the float64
// oracle beside that of the dense float32 form on the same inputs; the two agree in
// size (tests/test_gpu_fft.py).
//
// Two observations per transform: the spectra Y^'_i . conj(X^'_r) of real images are
// Hermitian, so one inverse FFT2 of P_i + i P_{i+1} gives corr_i in its real part and
// corr_{i+1} in its imaginary part; likewise one forward FFT2 of the real weight maps
// w_i + i w_{i+1} gives F, and W^_i = (F[k] + conj F[-k]) / 2, W^_{i+1} =
// (F[k] - conj F[-k]) / (2i).  Both passes pair observations (2j, 2j + 1) the same way,
// so pass 2's logits round exactly like pass 1's.
//
// FFTs: l x l with l in {8, 16, 32}.  One warp transforms one tile: lane j holds one
// line (l complex values) in registers and runs a radix-2 decimation-in-time FFT on it;
// the other direction is reached through a padded shared-memory transpose (row stride
// l + 1, conflict-free).  Twiddles e^{-2 pi i m / 64} come from constant memory,
// computed on the host in double precision.
#include <cmath>
#include <mutex>

#include "srmra_internal.cuh"

namespace srmra {

namespace {

__constant__ float2 c_tw[32];  // e^{-2 pi i m / 64}, m < 32

constexpr int FFT_WARPS = 8;      // warps per CTA of pass 1
// warps per CTA of pass 2: each warp keeps the c and zb sums of its lag row in registers
// and its G sum in shared memory, so more warps fit than with all three in shared memory
template <int N>
constexpr int p2_warps() {
  return N == 32 ? 12 : 16;
}
constexpr int SPEC_WARPS = 4;     // warps per CTA of the spectra kernels

constexpr int brev(int i, int n) {
  int r = 0;
  for (int b = 1; b < n; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// In-register FFT of length N (natural order in and out): X[k] = sum_n v[n] W^{+-nk},
// W = e^{-2 pi i / N}; INV selects the + sign (no 1/N scaling).
template <int N, bool INV>
__device__ __forceinline__ void fft_reg(float2 (&v)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int j = brev(i, N);
    if (j > i) {
      const float2 t = v[i];
      v[i] = v[j];
      v[j] = t;
    }
  }
#pragma unroll
  for (int h = 1; h < N; h <<= 1) {
#pragma unroll
    for (int k = 0; k < N; k += 2 * h) {
#pragma unroll
      for (int j = 0; j < h; ++j) {
        const float2 a = v[k + j];
        float2 b = v[k + j + h];
        const int m = j * (32 / h);  // twiddle e^{-2 pi i m / 64} (conjugated when INV)
        if (m == 16) {  // -i (+i): an exchange of the parts
          b = INV ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
        } else if (m == 8 || m == 24) {  // (1 -+ i) c and (-1 -+ i) c, c = cos(pi / 4)
          const float c = c_tw[8].x;
          const float sp = c * (b.x + b.y), sm = c * (b.x - b.y);
          if (m == 8)
            b = INV ? make_float2(sm, sp) : make_float2(sp, -sm);
          else
            b = INV ? make_float2(-sp, sm) : make_float2(-sm, -sp);
        } else if (m != 0) {
          float2 w = c_tw[m];
          if (INV) w.y = -w.y;
          b = cmul(b, w);
        }
        v[k + j] = make_float2(a.x + b.x, a.y + b.y);
        v[k + j + h] = make_float2(a.x - b.x, a.y - b.y);
      }
    }
  }
}

// The line a lane holds goes through the warp's tile (row stride N + 1) and comes back
// as the crossing line: lane j writes line j as the j-th column (COLS_IN = true) or
// row, and reads the j-th row (or column).  Lanes >= N only join the barriers.
template <int N, bool COLS_IN>
__device__ __forceinline__ void transpose(float2 (&v)[N], float2* tile, int lane) {
  __syncwarp();
  if (lane < N) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (COLS_IN)
        tile[k * (N + 1) + lane] = v[k];
      else
        tile[lane * (N + 1) + k] = v[k];
    }
  }
  __syncwarp();
  if (lane < N) {
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = COLS_IN ? tile[lane * (N + 1) + k] : tile[k * (N + 1) + lane];
  }
  __syncwarp();
}

// 2D FFT of a real l x l image given by column (lane j: v[k] = img[k][j]), result stored
// in natural [k1][k2] order to `out` (coalesced, through the tile).
template <int N>
__device__ __forceinline__ void fft2_real_store(float2 (&v)[N], float2* tile, int lane,
                                                float2* __restrict__ out) {
  fft_reg<N, false>(v);            // along the first axis (column j)
  transpose<N, true>(v, tile, lane);
  fft_reg<N, false>(v);            // along the second axis (row j = k1)
  __syncwarp();
  if (lane < N) {
#pragma unroll
    for (int k = 0; k < N; ++k) tile[lane * (N + 1) + k] = v[k];
  }
  __syncwarp();
  for (int idx = lane; idx < N * N; idx += 32) out[idx] = tile[(idx / N) * (N + 1) + idx % N];
  __syncwarp();
}

// ---------------------------------------------------------------- spectra of the data
// Yf[i][k1 l + k2] = FFT2(y'_i) (once per context).  One warp per observation.
template <int N>
__global__ void __launch_bounds__(32 * SPEC_WARPS) k_fft_obs(const float* __restrict__ Yc, int ldy,
                                                             int64_t n_obs,
                                                             float2* __restrict__ Yf) {
  __shared__ float2 tiles[SPEC_WARPS][N * (N + 1)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * SPEC_WARPS + warp;
  if (i >= n_obs) return;  // whole warps only
  float2 v[N];
#pragma unroll
  for (int k = 0; k < N; ++k)
    v[k] = make_float2(lane < N ? Yc[i * ldy + k * N + lane] : 0.f, 0.f);
  fft2_real_store<N>(v, tiles[warp], lane, Yf + i * (N * N));
}

// Xf[r][k1 l + k2] = FFT2(x'_r), x'_r = x_r - m_r (each iteration).  One warp per phase.
template <int N>
__global__ void __launch_bounds__(32 * SPEC_WARPS) k_fft_templates(const float* __restrict__ x,
                                                                   const double* __restrict__ sub,
                                                                   int L, int K,
                                                                   float2* __restrict__ Xf) {
  __shared__ float2 tiles[SPEC_WARPS][N * (N + 1)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * SPEC_WARPS + warp;
  if (r >= K * K) return;
  const int r1 = r / K, r2 = r % K;
  const float m = (float)sub[r];
  float2 v[N];
#pragma unroll
  for (int k = 0; k < N; ++k)
    v[k] = make_float2(lane < N ? x[(r1 + k * K) * L + r2 + lane * K] - m : 0.f, 0.f);
  fft2_real_store<N>(v, tiles[warp], lane, Xf + (int64_t)r * (N * N));
}

// Shared by both passes: stage X^_r and the column terms of phase r, then for one
// observation produce corr_{i,r}[t1 = lane][t2 = k] * l^2 in v[k].x (lane < l).
struct FftPassArgs {
  const float2* Yf;
  const float2* Xf;
  const float* ybar;
  const float* colb;
  const float* colm;
  const float* lse2;
  int64_t N, Npad;
  int L, K, B;  // B: observations per block
  float a2n;    // a2 / l^2 (the inverse FFT is unscaled)
  float c2;
};

template <int N>
__device__ __forceinline__ void stage_phase(const FftPassArgs& a, int r, float2* sX, float* sCol,
                                            float& mr) {
  const int r1 = r / a.K, r2 = r % a.K;
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    sX[idx] = a.Xf[(int64_t)r * (N * N) + idx];
    const int t1 = idx / N, t2 = idx % N;
    const int s1 = ((t1 * a.K - r1) % a.L + a.L) % a.L, s2 = ((t2 * a.K - r2) % a.L + a.L) % a.L;
    sCol[t1 * (N + 1) + t2] = a.colb[s1 * a.L + s2];
  }
  const int s0 = ((a.L - r1) % a.L) * a.L + (a.L - r2) % a.L;  // s(r, t = 0)
  mr = a.colm[s0];
  __syncthreads();
}

// Observations i and i + 1 (`two`: whether i + 1 exists) against the staged phase:
// v[k] = l^2 (corr_i, corr_{i+1})[t1 = lane][t2 = k].
template <int N>
__device__ __forceinline__ void correlate2(const FftPassArgs& a, int64_t i, bool two,
                                           const float2* sX, float2* tile, int lane,
                                           float2 (&v)[N]) {
  // unconditional loads (the second spectrum weighted by 0 when absent), so that all
  // of a lane's loads can be in flight at once
  const float2* yf0 = a.Yf + i * (N * N);
  const float2* yf1 = two ? yf0 + N * N : yf0;
  const float s1 = two ? 1.f : 0.f;
  if (lane < N) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const float2 x = sX[k * N + lane];
      const float2 p0 = cmul_conj(yf0[k * N + lane], x);
      const float2 p1 = cmul_conj(yf1[k * N + lane], x);
      v[k] = make_float2(p0.x - s1 * p1.y, p0.y + s1 * p1.x);  // P_i + i P_{i+1}
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = make_float2(0.f, 0.f);
  }
  fft_reg<N, true>(v);  // column lane (over k1)
  transpose<N, true>(v, tile, lane);
  fft_reg<N, true>(v);  // row lane (over k2)
}

// v[k] = (logit2 of observation i, of observation i + 1) at lag (t1 = lane, t2 = k) of the
// staged phase; cst0, cst1 their -c2 (ybar - m_r)^2 terms.
template <int N>
__device__ __forceinline__ void phase_logits2(const FftPassArgs& a, int64_t i, bool two,
                                              const float2* sX, const float* sCol, float2* tile,
                                              int lane, float cst0, float cst1, float2 (&v)[N]) {
  correlate2<N>(a, i, two, sX, tile, lane, v);
  if (lane < N) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const float cb = sCol[lane * (N + 1) + k];
      v[k].x = fmaf(v[k].x, a.a2n, cb + cst0);
      v[k].y = fmaf(v[k].y, a.a2n, cb + cst1);
    }
  }
}

// ---------------------------------------------------------------------- pass 1
// Per (observation block, phase r): the running (max, sum of 2^(logit2 - max)) over the
// l^2 lags of phase r, written as the partial of group r.
template <int N>
__global__ void __launch_bounds__(32 * FFT_WARPS, 2) k_fft_p1(FftPassArgs a, float* __restrict__ pm,
                                                           float* __restrict__ ps) {
  extern __shared__ __align__(16) unsigned char fsm[];
  float2* sX = (float2*)fsm;                         // [N*N]
  float2* tiles = sX + N * N;                        // [W][N*(N+1)]
  float* sCol = (float*)(tiles + FFT_WARPS * N * (N + 1));  // [N*(N+1)]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.y;
  float mr;
  stage_phase<N>(a, r, sX, sCol, mr);
  const int64_t i0 = (int64_t)blockIdx.x * a.B;  // even: B is a multiple of FFT_WARPS
  const int64_t i1 = min(a.N, i0 + a.B);
  for (int64_t i = i0 + 2 * warp; i < i1; i += 2 * FFT_WARPS) {  // pairs (i, i + 1)
    const bool two = i + 1 < i1;
    float2 v[N];
    const float dd0 = a.ybar[i] - mr;
    const float dd1 = two ? a.ybar[i + 1] - mr : 0.f;
    phase_logits2<N>(a, i, two, sX, sCol, tiles + warp * N * (N + 1), lane, -a.c2 * dd0 * dd0,
                     -a.c2 * dd1 * dd1, v);
    float mx0 = -INFINITY, mx1 = -INFINITY;
    if (lane < N) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        mx0 = fmaxf(mx0, v[k].x);
        mx1 = fmaxf(mx1, v[k].y);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
      mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
    }
    const float base0 = (mx0 == -INFINITY) ? 0.f : mx0;
    const float base1 = (mx1 == -INFINITY) ? 0.f : mx1;
    float sm0 = 0.f, sm1 = 0.f;
    if (lane < N) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        sm0 += exp2f(v[k].x - base0);
        sm1 += exp2f(v[k].y - base1);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sm0 += __shfl_xor_sync(0xffffffffu, sm0, o);
      sm1 += __shfl_xor_sync(0xffffffffu, sm1, o);
    }
    if (lane == 0) {
      pm[(int64_t)r * a.Npad + i] = mx0;
      ps[(int64_t)r * a.Npad + i] = sm0;
      if (two) {
        pm[(int64_t)r * a.Npad + i + 1] = mx1;
        ps[(int64_t)r * a.Npad + i + 1] = sm1;
      }
    }
  }
}

// ---------------------------------------------------------------------- pass 2
// Per (observation block b, phase r): w = 2^(logit2 - lse2) over the lags of phase r;
// c and zb per shift of phase r, and G_r = sum_i conj(FFT2(w_{i,r})) . Y^'_i, summed
// over the block's observations in a fixed order (each warp over its observation pairs
// in increasing i, then the warps in order).
template <int N>
__global__ void __launch_bounds__(32 * p2_warps<N>(), 1) k_fft_p2(FftPassArgs a, float* __restrict__ cp,
                                                           float* __restrict__ zbp, int Spad,
                                                           float2* __restrict__ Gp) {
  extern __shared__ __align__(16) unsigned char fsm[];
  constexpr int W = p2_warps<N>();
  float2* sX = (float2*)fsm;                              // [N*N]
  float2* tiles = sX + N * N;                             // [W][N*(N+1)]
  float2* sG = tiles + W * N * (N + 1);                   // [W][N*N]
  float* sCol = (float*)(sG + W * N * N);                 // [N*(N+1)]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.y, b = blockIdx.x;
  float2* tile = tiles + warp * N * (N + 1);
  float2* g = sG + warp * N * N;
  float crow[N], zrow[N];  // c and zb of lag row t1 = lane, over this warp's observations
#pragma unroll
  for (int k = 0; k < N; ++k) crow[k] = zrow[k] = 0.f;
  for (int idx = lane; idx < N * N; idx += 32) g[idx] = make_float2(0.f, 0.f);
  float mr;
  stage_phase<N>(a, r, sX, sCol, mr);
  const int64_t i0 = (int64_t)b * a.B;
  const int64_t i1 = min(a.N, i0 + a.B);
  for (int64_t i = i0 + 2 * warp; i < i1; i += 2 * W) {  // pairs (i, i + 1), as in pass 1
    const bool two = i + 1 < i1;
    float2 v[N];
    const float yb0 = a.ybar[i], yb1 = two ? a.ybar[i + 1] : 0.f;
    const float dd0 = yb0 - mr, dd1 = yb1 - mr;
    phase_logits2<N>(a, i, two, sX, sCol, tile, lane, -a.c2 * dd0 * dd0, -a.c2 * dd1 * dd1, v);
    const float ls0 = a.lse2[i], ls1 = two ? a.lse2[i + 1] : 0.f;
    if (lane < N) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const float w0 = exp2f(v[k].x - ls0);
        const float w1 = two ? exp2f(v[k].y - ls1) : 0.f;
        crow[k] += w0;
        zrow[k] = fmaf(w0, yb0, zrow[k]);
        crow[k] += w1;
        zrow[k] = fmaf(w1, yb1, zrow[k]);
        v[k] = make_float2(w0, w1);
      }
    }
    // F = FFT2(w_i + i w_{i+1}) (row lane = t1 first): v[k] = F[k1 = k][k2 = lane]
    fft_reg<N, false>(v);
    transpose<N, false>(v, tile, lane);
    fft_reg<N, false>(v);
    // W^_i = (F[k] + conj F[-k]) / 2 and W^_{i+1} = (F[k] - conj F[-k]) / (2i); F[-k] is
    // element (N - k1) mod N of lane (N - k2) mod N.  Then G += conj(W^) . Y^' by column.
    const int src = (N - lane) & (N - 1);
    const float2* yf0 = a.Yf + i * (N * N);
    const float2* yf1 = two ? yf0 + N * N : yf0;  // unconditional loads, as in correlate2
    const float h1 = two ? 0.5f : 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int km = (N - k) & (N - 1);
      const float fmx = __shfl_sync(0xffffffffu, v[km].x, src);
      const float fmy = __shfl_sync(0xffffffffu, v[km].y, src);
      if (lane < N) {
        const float2 f = v[k];
        const float2 y0 = yf0[k * N + lane], y1 = yf1[k * N + lane];
        const float2 w0 = make_float2(0.5f * (f.x + fmx), 0.5f * (f.y - fmy));
        const float2 w1 = make_float2(h1 * (f.y + fmy), -h1 * (f.x - fmx));
        float2 acc = g[k * N + lane];
        const float2 p0 = cmul_conj(y0, w0);
        acc.x += p0.x;
        acc.y += p0.y;
        const float2 p1 = cmul_conj(y1, w1);
        acc.x += p1.x;
        acc.y += p1.y;
        g[k * N + lane] = acc;
      }
    }
  }
  // each warp's c and zb rows into its transpose tile (floats: c, then zb)
  if (lane < N) {
    float* cz = (float*)tile;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      cz[lane * (N + 1) + k] = crow[k];
      cz[N * (N + 1) + lane * (N + 1) + k] = zrow[k];
    }
  }
  __syncthreads();
  // the warps' sums in order; c and zb go to the dense forms' per-shift partial layout
  const int r1 = r / a.K, r2 = r % a.K;
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int t1 = idx / N, t2 = idx % N;
    float c = 0.f, z = 0.f;
    float2 gg = make_float2(0.f, 0.f);
    for (int w = 0; w < W; ++w) {
      const float* cz = (const float*)(tiles + w * N * (N + 1));
      c += cz[t1 * (N + 1) + t2];
      z += cz[N * (N + 1) + t1 * (N + 1) + t2];
      const float2 q = sG[w * N * N + idx];
      gg.x += q.x;
      gg.y += q.y;
    }
    const int s1 = ((t1 * a.K - r1) % a.L + a.L) % a.L, s2 = ((t2 * a.K - r2) % a.L + a.L) % a.L;
    cp[(int64_t)b * Spad + s1 * a.L + s2] = c;
    zbp[(int64_t)b * Spad + s1 * a.L + s2] = z;
    Gp[((int64_t)b * a.K * a.K + r) * (N * N) + idx] = gg;
  }
}

// b'_r = IFFT2(sum_b G_{b,r}) / l^2, written as the single lag-range partial of the
// dense finalize (bpart[r][m1 l + m2]).  One CTA per phase.
template <int N>
__global__ void __launch_bounds__(256) k_fft_fin_b(const float2* __restrict__ Gp, int nb, int KK,
                                                   float* __restrict__ bpart) {
  __shared__ float2 sG[N * N];
  __shared__ float2 tile[N * (N + 1)];
  const int r = blockIdx.x;
  for (int idx = threadIdx.x; idx < N * N; idx += 256) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8  // loads issued ahead; the additions keep their order
    for (int b = 0; b < nb; ++b) {
      const float2 q = Gp[((int64_t)b * KK + r) * (N * N) + idx];
      acc.x += q.x;
      acc.y += q.y;
    }
    sG[idx] = acc;
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  float2 v[N];
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = lane < N ? sG[k * N + lane] : make_float2(0.f, 0.f);
  fft_reg<N, true>(v);
  transpose<N, true>(v, tile, lane);
  fft_reg<N, true>(v);  // v[k] = l^2 b'_r[m1 = lane][m2 = k]
  if (lane < N) {
    const float inv = 1.f / (float)(N * N);
#pragma unroll
    for (int k = 0; k < N; ++k) bpart[(int64_t)r * (N * N) + lane * N + k] = v[k].x * inv;
  }
}

template <int N>
constexpr size_t p1_smem_bytes() {
  return sizeof(float2) * (N * N + FFT_WARPS * N * (N + 1)) + sizeof(float) * (N * (N + 1));
}

template <int N>
constexpr size_t p2_smem_bytes() {
  return sizeof(float2) * (N * N + p2_warps<N>() * N * (N + 1) + p2_warps<N>() * N * N) +
         sizeof(float) * (N * (N + 1));
}

cudaError_t upload_twiddles() {
  static std::mutex mu;
  static int done_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done_dev == dev) return cudaSuccess;
  float2 tw[32];
  const double pi = std::acos(-1.0);
  for (int m = 0; m < 32; ++m)
    tw[m] = make_float2((float)std::cos(2.0 * pi * m / 64.0), (float)-std::sin(2.0 * pi * m / 64.0));
  e = cudaMemcpyToSymbol(c_tw, tw, sizeof(tw));
  if (e == cudaSuccess) done_dev = dev;
  return e;
}

FftPassArgs pass_args(srmra_ctx* c) {
  const Geom& g = c->g;
  const LogitScalars ls = logit_scalars(g);
  FftPassArgs a;
  a.Yf = c->Yf;
  a.Xf = c->Xf;
  a.ybar = c->ybar;
  a.colb = c->colb;
  a.colm = c->colm;
  a.lse2 = c->lse2;
  a.N = g.N;
  a.Npad = g.Npad;
  a.L = g.L;
  a.K = g.K;
  a.B = c->plan.fft_obs_per_block;
  a.a2n = ls.a2 / (float)g.l2;
  a.c2 = ls.c2;
  return a;
}

template <int N>
cudaError_t set_smem_n() {
  cudaError_t e = cudaFuncSetAttribute(k_fft_p1<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)p1_smem_bytes<N>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft_p2<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)p2_smem_bytes<N>());
  return e;
}
static_assert(p2_smem_bytes<32>() <= 232448, "exceeds the shared memory of one CTA");

}  // namespace

bool fft_supported(int l) { return l == 8 || l == 16 || l == 32; }

void plan_fft(srmra_ctx* c) {
  const Geom& g = c->g;
  Plan& p = c->plan;
  const int KK = g.K * g.K;
  int nb = c->num_sms / KK;  // about one wave of (block, phase) CTAs
  if (nb < 1) nb = 1;
  int64_t B = ceil_div(g.N, nb);
  B = round_up(B, FFT_WARPS);
  p.fft_obs_per_block = (int)B;
  p.fft_blocks = (int)ceil_div(g.N, B);
  // pass 1 writes only per-observation results and fits two CTAs per SM: twice the CTAs
  // (pass 2 keeps one per SM, of 12 or 16 warps, and one partial per block)
  const int64_t B1 = round_up(ceil_div(g.N, 2 * (int64_t)nb), FFT_WARPS);
  p.fft_p1_obs_per_block = (int)B1;
  p.fft_p1_blocks = (int)ceil_div(g.N, B1);
  p.p1_groups = KK;
  p.p1_tiles_per_group = 1;
  p.nparts_c = p.fft_blocks;
  p.nparts_z = 0;
  p.ll_blocks = (int)ceil_div(g.Npad, 256);
}

cudaError_t fft_set_attributes() {
  cudaError_t e = upload_twiddles();
  if (e == cudaSuccess) e = set_smem_n<8>();
  if (e == cudaSuccess) e = set_smem_n<16>();
  if (e == cudaSuccess) e = set_smem_n<32>();
  return e;
}

cudaError_t prep_obs_fft(srmra_ctx* c) {
  cudaError_t e = fft_set_attributes();
  if (e != cudaSuccess) return e;
  const Geom& g = c->g;
  const unsigned grid = (unsigned)ceil_div(g.N, SPEC_WARPS);
  switch (g.l) {
    case 8: k_fft_obs<8><<<grid, 32 * SPEC_WARPS, 0, c->stream>>>(c->Yc, g.ldy, g.N, c->Yf); break;
    case 16: k_fft_obs<16><<<grid, 32 * SPEC_WARPS, 0, c->stream>>>(c->Yc, g.ldy, g.N, c->Yf); break;
    default: k_fft_obs<32><<<grid, 32 * SPEC_WARPS, 0, c->stream>>>(c->Yc, g.ldy, g.N, c->Yf); break;
  }
  c->launches++;
  return cudaGetLastError();
}

void launch_templates_fft(srmra_ctx* c) {
  const Geom& g = c->g;
  const unsigned grid = (unsigned)ceil_div(g.K * g.K, SPEC_WARPS);
  switch (g.l) {
    case 8: k_fft_templates<8><<<grid, 32 * SPEC_WARPS, 0, c->stream>>>(c->x, c->sub, g.L, g.K, c->Xf); break;
    case 16: k_fft_templates<16><<<grid, 32 * SPEC_WARPS, 0, c->stream>>>(c->x, c->sub, g.L, g.K, c->Xf); break;
    default: k_fft_templates<32><<<grid, 32 * SPEC_WARPS, 0, c->stream>>>(c->x, c->sub, g.L, g.K, c->Xf); break;
  }
  c->launches++;
}

void launch_pass1_fft(srmra_ctx* c) {
  const Geom& g = c->g;
  FftPassArgs a = pass_args(c);
  a.B = c->plan.fft_p1_obs_per_block;
  const dim3 grid((unsigned)c->plan.fft_p1_blocks, (unsigned)(g.K * g.K));
  switch (g.l) {
    case 8: k_fft_p1<8><<<grid, 32 * FFT_WARPS, p1_smem_bytes<8>(), c->stream>>>(a, c->pm, c->ps); break;
    case 16: k_fft_p1<16><<<grid, 32 * FFT_WARPS, p1_smem_bytes<16>(), c->stream>>>(a, c->pm, c->ps); break;
    default: k_fft_p1<32><<<grid, 32 * FFT_WARPS, p1_smem_bytes<32>(), c->stream>>>(a, c->pm, c->ps); break;
  }
  c->launches++;
}

cudaError_t launch_pass2_fft(srmra_ctx* c) {
  const Geom& g = c->g;
  const FftPassArgs a = pass_args(c);
  const dim3 grid((unsigned)c->plan.fft_blocks, (unsigned)(g.K * g.K));
  switch (g.l) {
    case 8:
      k_fft_p2<8><<<grid, 32 * p2_warps<8>(), p2_smem_bytes<8>(), c->stream>>>(a, c->cp, c->zbp, g.Spad, c->Gp);
      break;
    case 16:
      k_fft_p2<16><<<grid, 32 * p2_warps<16>(), p2_smem_bytes<16>(), c->stream>>>(a, c->cp, c->zbp, g.Spad, c->Gp);
      break;
    default:
      k_fft_p2<32><<<grid, 32 * p2_warps<32>(), p2_smem_bytes<32>(), c->stream>>>(a, c->cp, c->zbp, g.Spad, c->Gp);
      break;
  }
  c->launches++;
  return cudaGetLastError();
}

void launch_fin_b_fft(srmra_ctx* c) {
  const Geom& g = c->g;
  const int KK = g.K * g.K;
  switch (g.l) {
    case 8: k_fft_fin_b<8><<<KK, 256, 0, c->stream>>>(c->Gp, c->plan.fft_blocks, KK, c->bpart); break;
    case 16: k_fft_fin_b<16><<<KK, 256, 0, c->stream>>>(c->Gp, c->plan.fft_blocks, KK, c->bpart); break;
    default: k_fft_fin_b<32><<<KK, 256, 0, c->stream>>>(c->Gp, c->plan.fft_blocks, KK, c->bpart); break;
  }
  c->launches++;
}

}  // namespace srmra
