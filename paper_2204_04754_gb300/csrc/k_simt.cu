// Float32 form of the E-step / M-step contractions on CUDA cores (FFMA).
//
// Pass 1 (Eq. weights_EM, Eq. likelihood_EM): for an observation tile and a group of
// shift tiles, logit2[i,s] = a2 <y'_i, T'_s> + colb[s] - c2 (ybar_i - colm[s])^2 and the
// running (max, sum of 2^(logit2 - max)) per observation -> partials per shift group.
//
// Pass 2 (Eq. x_EM, Eq. rho_EM): w[i,s] = 2^(logit2[i,s] - lse2[i]) is recomputed from
// the same contraction, and the M-step sums
//   Z'[s][n] = sum_i w[i,s] y'_i[n],  c[s] = sum_i w[i,s],  zb[s] = sum_i w[i,s] ybar_i
// are accumulated.  The N x L^2 weight matrix is never stored: a cluster of gc CTAs
// (one per 256-pixel chunk of Z') works on one 64-shift tile; each CTA computes the
// weights of its own 64 observations per round and the others read them through
// distributed shared memory, so no CTA recomputes another's logits.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "srmra_internal.cuh"

namespace cg = cooperative_groups;

namespace srmra {

namespace {

__device__ __forceinline__ float4 ld4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ void st4(float* p, float4 v) {
  *reinterpret_cast<float4*>(p) = v;
}

// Packed pairs of float32 in one 64-bit register (element 0 in the low half, i.e. the
// memory order of a float2).  fma.rn.f32x2 rounds each half exactly like fmaf, so the
// packed loops give the same bits as scalar ones with half the issued instructions.
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
__device__ __forceinline__ ulonglong2 ld4p(const float* p) {
  return *reinterpret_cast<const ulonglong2*>(p);
}
__device__ __forceinline__ void st4p(float* p, f2 a, f2 b) {
  *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(a, b);
}

// ----------------------------------------------------------------------------- pass 1
// Tile 128 observations x 128 shifts, 256 threads, 8x8 outputs per thread, k-step 8.
// Operands are pixel-major: YcT[k][i], AxT[k][s].
__global__ void __launch_bounds__(256, 2)
    k_p1_f32(const float* __restrict__ YcT, int64_t Npad, const float* __restrict__ AxT,
             int Spad, int ldy, const float* __restrict__ ybar,
             const float* __restrict__ colb, const float* __restrict__ colm, float a2,
             float c2, int tiles_per_group, int n_tiles, int64_t N, float* __restrict__ pm,
             float* __restrict__ ps) {
  __shared__ __align__(16) float As[2][8][128];
  __shared__ __align__(16) float Bs[2][8][128];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * 128;
  const int grp = blockIdx.y;
  const int tb = grp * tiles_per_group;
  const int te = min(n_tiles, tb + tiles_per_group);
  const int lk = tid >> 5, lc = (tid & 31) * 4;

  // The 16 lanes with the same ty share the rows of their 8 observations; lane tx < 8
  // keeps row tx's ybar and running (max, sum), read by the others through shuffles.
  const int orow = (tx & 7) < 4 ? ty * 4 + (tx & 7) : 64 + ty * 4 + (tx & 7) - 4;
  const int lane = tid & 31, lgrp = lane & 16;
  const float my_yb = ybar[i0 + orow];
  float my_rm = -INFINITY, my_rs = 0.f;

  for (int tile = tb; tile < te; ++tile) {
    const int s0 = tile * 128;
    f2 acc2[8][4];  // acc2[j][c/2] holds the outputs (j, c) and (j, c + 1)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc2[j][c] = 0ull;

    float4 ra = ld4(YcT + (int64_t)lk * Npad + i0 + lc);
    float4 rb = ld4(AxT + (int64_t)lk * Spad + s0 + lc);
    st4(&As[0][lk][lc], ra);
    st4(&Bs[0][lk][lc], rb);
    __syncthreads();
    int cur = 0;
    for (int kc = 0; kc < ldy; kc += 8) {
      const bool more = kc + 8 < ldy;
      if (more) {
        ra = ld4(YcT + (int64_t)(kc + 8 + lk) * Npad + i0 + lc);
        rb = ld4(AxT + (int64_t)(kc + 8 + lk) * Spad + s0 + lc);
      }
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const float4 a0 = ld4(&As[cur][kk][ty * 4]);
        const float4 a1 = ld4(&As[cur][kk][64 + ty * 4]);
        const ulonglong2 b0 = ld4p(&Bs[cur][kk][tx * 4]);
        const ulonglong2 b1 = ld4p(&Bs[cur][kk][64 + tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const f2 b[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const f2 aj = dup2(a[j]);
#pragma unroll
          for (int c = 0; c < 4; ++c) ffma2(acc2[j][c], aj, b[c]);
        }
      }
      if (more) {
        st4(&As[cur ^ 1][lk][lc], ra);
        st4(&Bs[cur ^ 1][lk][lc], rb);
      }
      __syncthreads();
      cur ^= 1;
    }

    // online log-sum-exp over this tile's 128 shifts (16 lanes share a row)
    float cb[8], cm[8];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      cb[c] = colb[s0 + tx * 4 + c];
      cm[c] = colm[s0 + tx * 4 + c];
      cb[4 + c] = colb[s0 + 64 + tx * 4 + c];
      cm[4 + c] = colm[s0 + 64 + tx * 4 + c];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float ybj = __shfl_sync(0xffffffffu, my_yb, lgrp | j);
      const float rmj = __shfl_sync(0xffffffffu, my_rm, lgrp | j);
      const float rsj = __shfl_sync(0xffffffffu, my_rs, lgrp | j);
      float v[8];
      float mx = -INFINITY;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float d = ybj - cm[c];
        const float acc = (c & 1) ? hi2(acc2[j][c >> 1]) : lo2(acc2[j][c >> 1]);
        v[c] = fmaf(acc, a2, cb[c]) - c2 * d * d;
        mx = fmaxf(mx, v[c]);
      }
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float nm = fmaxf(rmj, mx);
      const float base = (nm == -INFINITY) ? 0.f : nm;
      float sm = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) sm += exp2f(v[c] - base);
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
      const float nrs = rsj * exp2f(rmj - base) + sm;
      if (tx == j) {
        my_rm = nm;
        my_rs = nrs;
      }
    }
  }
  if (tx < 8 && i0 + orow < N) {
    pm[grp * Npad + i0 + orow] = my_rm;
    ps[grp * Npad + i0 + orow] = my_rs;
  }
}

// ----------------------------------------------------------------------------- pass 2
// Work: for every 64-shift tile and group of gc 256-pixel chunks (a "unit"), the
// observation blocks of 64 are taken gc at a time ("rounds", R per unit); in a round,
// rank q of a cluster of gc CTAs computes the 64x64 weight tile of block q, and every
// rank accumulates Z' over its own pixel chunk for all gc blocks.  The launch is
// persistent, one cluster per co-resident slot.  The first U1 = ncl floor(U / ncl)
// units are dealt out whole (cluster c takes units c, c + ncl, ...), so all clusters
// sweep the observations in step and each block is read from DRAM about once.  The
// items (unit, round) of the remaining units are split into ncl contiguous ranges, one
// per cluster, so a remaining unit is shared by a few consecutive clusters.  Each
// cluster writes the partial sums of its part of a unit into its own segment (whole
// units: segment 0; shared units: the cluster's index minus that of the unit's first
// cluster); the cluster that finishes a unit zero-fills the segments after its own, so
// the finalize sums nseg segments for every shift.
//
// Every rank holds the weight tiles of all gc blocks of a round: the rank that computes
// a tile stores it into its own shared memory and into every other rank's (remote
// stores through distributed shared memory, which do not wait for a reply), so the
// M-step loop reads only local shared memory.
//
// The 512 threads of a CTA form two groups that work one round apart:
//   group A (threads 0-255): logits S[s][i] = <T'_s, y'_i> of the next round's block
//     (4x4 outputs per thread), then w = 2^(logit2 - lse2) into the weight buffers and
//     the partial sums c[s], zb[s];
//   group C (threads 256-511): Z'[s][p] += sum_i w[i][s] y'_i[p] for the current round
//     (8 shifts x 8 pixels per thread).
// Two weight buffers alternate between rounds.  One split-phase cluster barrier per
// round orders them: group A arrives after writing the weights of round p, group C
// after it has finished reading round p - 1 (whose buffer round p + 1 reuses); group A
// waits on it before writing a buffer, group C before reading one.  Each group stages
// its operands through a 2-deep cp.async ring synchronised by its own named barrier.
constexpr int P2_ATHREADS = 256;
constexpr int P2_THREADS = 512;
constexpr int P2_NST = 2;     // cp.async stages per group
constexpr int P2_MAX_GC = 4;  // cluster width (weight tiles held per round)
constexpr int P2_KS = 64;     // group A: pixels (k) per stage
constexpr int P2_SMEM_FLOATS = 2 * P2_MAX_GC * 64 * 64      // P[2][gc][64 obs][64 shifts]
                               + P2_NST * 2 * P2_KS * 64    // group A: As, Bs [stage][KS][64]
                               + P2_NST * 16 * 256;         // group C: Ys [stage][16][256]
static_assert(P2_SMEM_FLOATS * 4 <= 232448, "exceeds the shared memory of one CTA");
constexpr size_t P2_SMEM_BYTES = P2_SMEM_FLOATS * sizeof(float);

__device__ __forceinline__ void cp16(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void group_bar(int id) {
  asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory");
}
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(P2_THREADS, 1)
    k_p2_f32(const float* __restrict__ YcT, const float* __restrict__ Yc, int64_t Npad,
             const float* __restrict__ AxT, int Spad, int ldy,
             const float* __restrict__ ybar, const float* __restrict__ colb,
             const float* __restrict__ colm, const float* __restrict__ lse2, float a2,
             float c2, int64_t N, int S, int n_iblk, int gc, int n_cgroups, int R,
             int64_t U, int64_t U1, int ncl, int nseg, float* __restrict__ Zp,
             float* __restrict__ cp,
             float* __restrict__ zbp) {
  extern __shared__ __align__(16) float smem[];
  float* const Pbuf = smem;                              // [2][gc][64 obs][64 shifts]
  float* const As = smem + 2 * P2_MAX_GC * 4096;         // [P2_NST][KS][64] shifts
  float* const Bs = As + P2_NST * P2_KS * 64;            // [P2_NST][KS][64] observations
  float* const Ys = Bs + P2_NST * P2_KS * 64;            // [P2_NST][16][256] pixels
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cid = (int)(blockIdx.x / gc);
  const int64_t kw = U1 / ncl;  // whole units of this cluster
  const int64_t T2 = (U - U1) * R;  // items of the shared units
  const int64_t ncl2 = T2 < ncl ? T2 : ncl;  // clusters sharing them (non-empty ranges)
  const int64_t t2b = cid < ncl2 ? (int64_t)cid * T2 / ncl2 : 0;
  const int64_t t2e = cid < ncl2 ? (int64_t)(cid + 1) * T2 / ncl2 : 0;
  const int64_t n_loc = kw * R + (t2e - t2b);
  // j-th item of this cluster, as (unit) * R + (round)
  auto item = [&](int64_t j) -> int64_t {
    if (j < kw * R) return (cid + (j / R) * ncl) * R + j % R;
    return U1 * R + t2b + (j - kw * R);
  };
  const int nks = (ldy + P2_KS - 1) / P2_KS;  // rows past ldy are zero-filled
  // segment of unit u written by this cluster
  auto segment = [&](int64_t u) -> int {
    if (u < U1) return 0;
    const int64_t t0 = (u - U1) * R;
    int64_t c = t0 * ncl2 / T2;
    while (c + 1 < ncl2 && (c + 1) * T2 / ncl2 <= t0) ++c;
    return cid - (int)c;
  };

  if (threadIdx.x < P2_ATHREADS) {
    // ------------------------------------------------------------------ group A
    const int tid = threadIdx.x;
    const int ts = tid & 15, ti = tid >> 4;  // 4 shifts x 4 observations
    const int lk = tid >> 4, lc = (tid & 15) * 4;
    float cacc[4], zacc[4], cbA[4], cmA[4];
    int64_t cur_u = -1;
    for (int64_t tl = 0; tl < n_loc; ++tl) {
      const int64_t t = item(tl), u = t / R;
      const int r = (int)(t % R);
      const int cgrp = (int)(u % n_cgroups);
      const int s0 = (int)(u / n_cgroups) * 64;
      if (u != cur_u) {
        cur_u = u;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          cacc[a] = zacc[a] = 0.f;
          cbA[a] = colb[s0 + ts * 4 + a];
          cmA[a] = colm[s0 + ts * 4 + a];
        }
      }
      const int myb = r * gc + rank;
      const bool mine = myb < n_iblk;
      const int64_t ib = (int64_t)myb * 64;
      f2 acc2[4][2];  // acc2[a][b/2] holds S entries (a, b) and (a, b + 1)
#pragma unroll
      for (int a = 0; a < 4; ++a) acc2[a][0] = acc2[a][1] = 0ull;
      if (mine) {
        auto issue = [&](int ks) {
          const int st = ks % P2_NST;
          if (ks < nks) {
#pragma unroll
            for (int h = 0; h < P2_KS / 16; ++h) {
              const int kr = lk + 16 * h, k = ks * P2_KS + kr;
              const bool v = k < ldy;
              const int64_t kc = v ? k : 0;
              cp16(As + (st * P2_KS + kr) * 64 + lc, AxT + kc * Spad + s0 + lc, v);
              cp16(Bs + (st * P2_KS + kr) * 64 + lc, YcT + kc * Npad + ib + lc, v);
            }
          }
          cp_commit();
        };
        group_bar(1);  // the stage buffers (and the reduction area) are no longer read
        issue(0);
        for (int ks = 0; ks < nks; ++ks) {
          cp_wait0();
          group_bar(1);
          issue(ks + 1);  // into the buffer of stage ks - 1, free after the barrier
          const float* Ac = As + (ks % P2_NST) * P2_KS * 64;
          const float* Bc = Bs + (ks % P2_NST) * P2_KS * 64;
#pragma unroll
          for (int kk = 0; kk < P2_KS; ++kk) {
            const float4 a4 = ld4(Ac + kk * 64 + ts * 4);
            const ulonglong2 b4 = ld4p(Bc + kk * 64 + ti * 4);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              const f2 aa = dup2(av[a]);
              ffma2(acc2[a][0], aa, b4.x);
              ffma2(acc2[a][1], aa, b4.y);
            }
          }
        }
      }
      if (tl >= 1) cluster_wait();  // every rank has finished reading round tl - 2
      if (mine) {
        float* const P = Pbuf + ((tl & 1) * P2_MAX_GC + rank) * 4096;  // this block's tile
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int64_t i = ib + ti * 4 + b;
          const float yb = ybar[i];
          const float ls = lse2[i];
          const bool iv = i < N;
          float w[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const float d = yb - cmA[a];
            const float acc = (b & 1) ? hi2(acc2[a][b >> 1]) : lo2(acc2[a][b >> 1]);
            const float v = fmaf(acc, a2, cbA[a]) - c2 * d * d - ls;
            w[a] = (iv && (s0 + ts * 4 + a) < S) ? exp2f(v) : 0.f;
            cacc[a] += w[a];
            zacc[a] = fmaf(w[a], yb, zacc[a]);
          }
          const float4 w4 = make_float4(w[0], w[1], w[2], w[3]);
          for (int q = 0; q < gc; ++q)  // own copy and every other rank's
            st4(cluster.map_shared_rank(P, q) + (ti * 4 + b) * 64 + ts * 4, w4);
        }
      }
      cluster_arrive();  // the weights of round tl are in place
      if (cgrp == 0 && (r == R - 1 || tl == n_loc - 1)) {
        // this cluster's part of the unit ends here: its partial c and zb
        float* red = As;  // [16][64] c, then [16][64] zb
        group_bar(1);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          red[ti * 64 + ts * 4 + a] = cacc[a];
          red[1024 + ti * 64 + ts * 4 + a] = zacc[a];
        }
        group_bar(1);
        if (tid < 64) {
          float c = 0.f, zb = 0.f;
          for (int k = 0; k < 16; ++k) {
            c += red[k * 64 + tid];
            zb += red[1024 + k * 64 + tid];
          }
          const int seg = segment(u);
          cp[((int64_t)seg * gc + rank) * Spad + s0 + tid] = c;
          zbp[((int64_t)seg * gc + rank) * Spad + s0 + tid] = zb;
          if (r == R - 1)  // the unit is complete: no later segment exists
            for (int sg2 = seg + 1; sg2 < nseg; ++sg2) {
              cp[((int64_t)sg2 * gc + rank) * Spad + s0 + tid] = 0.f;
              zbp[((int64_t)sg2 * gc + rank) * Spad + s0 + tid] = 0.f;
            }
        }
      }
    }
    cluster_wait();
    cluster_arrive();
    cluster_wait();  // no rank leaves while another may still access its shared memory
  } else {
    // ------------------------------------------------------------------ group C
    const int tid = threadIdx.x - P2_ATHREADS;
    const int sg = tid >> 5, pg = tid & 31;  // 8 shifts x 8 pixels
    f2 z2[8][4];  // z2[a][b/2] holds Z' entries (a, b) and (a, b + 1)
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) z2[a][b] = 0ull;
    for (int64_t tl = 0; tl <= n_loc; ++tl) {
      cluster_arrive();  // finished reading round tl - 1
      cluster_wait();    // the weights of round tl are in place
      if (tl == n_loc) break;
      const int64_t t = item(tl), u = t / R;
      const int r = (int)(t % R);
      const int s0 = (int)(u / n_cgroups) * 64;
      const int p0 = ((int)(u % n_cgroups) * gc + rank) * 256;
      const float* const P = Pbuf + (tl & 1) * P2_MAX_GC * 4096;
      const int nq = min(gc, n_iblk - r * gc);
      const int nchunks = nq * 4;  // 16-observation chunks
      auto issue = [&](int cidx) {
        const int st = cidx % P2_NST;
        if (cidx < nchunks) {
          const int q = cidx >> 2, ic = (cidx & 3) * 16;
          const int64_t ib = (int64_t)(r * gc + q) * 64 + ic;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int row = (tid >> 6) + 4 * j, col = (tid & 63) * 4;
            const int p = p0 + col;
            const bool v = p < ldy;
            cp16(Ys + st * 4096 + row * 256 + col, Yc + (ib + row) * ldy + (v ? p : 0), v);
          }
        }
        cp_commit();
      };
      group_bar(2);  // the stage buffers of the previous round are no longer read
      issue(0);
      for (int cidx = 0; cidx < nchunks; ++cidx) {
        cp_wait0();
        group_bar(2);
        issue(cidx + 1);  // into the buffer of stage cidx - 1, free after the barrier
        const int q = cidx >> 2, ic = (cidx & 3) * 16;
        const float* Pq = P + q * 4096 + ic * 64 + sg * 8;
        const float* Yb = Ys + (cidx % P2_NST) * 4096;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float4 w0 = ld4(Pq + k * 64);
          const float4 w1 = ld4(Pq + k * 64 + 4);
          const ulonglong2 y0 = ld4p(Yb + k * 256 + pg * 4);
          const ulonglong2 y1 = ld4p(Yb + k * 256 + 128 + pg * 4);
          const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
          const f2 yv[4] = {y0.x, y0.y, y1.x, y1.y};
#pragma unroll
          for (int a = 0; a < 8; ++a) {
            const f2 wa = dup2(wv[a]);
#pragma unroll
            for (int b = 0; b < 4; ++b) ffma2(z2[a][b], wa, yv[b]);
          }
        }
      }
      if (r == R - 1 || tl == n_loc - 1) {
        // this cluster's part of the unit ends here: its partial Z' over the chunk
        const int seg = segment(u);
        const int pa = p0 + pg * 4, pb = p0 + 128 + pg * 4;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int s = s0 + sg * 8 + a;
          float* zr = Zp + ((int64_t)seg * Spad + s) * ldy;
          if (pa < ldy) st4p(zr + pa, z2[a][0], z2[a][1]);
          if (pb < ldy) st4p(zr + pb, z2[a][2], z2[a][3]);
#pragma unroll
          for (int b = 0; b < 4; ++b) z2[a][b] = 0ull;
          if (r == R - 1)  // the unit is complete: no later segment exists
            for (int sg2 = seg + 1; sg2 < nseg; ++sg2) {
              float* zz = Zp + ((int64_t)sg2 * Spad + s) * ldy;
              if (pa < ldy) st4(zz + pa, make_float4(0.f, 0.f, 0.f, 0.f));
              if (pb < ldy) st4(zz + pb, make_float4(0.f, 0.f, 0.f, 0.f));
            }
        }
      }
    }
  }
}

}  // namespace

int p2_clusters(int gc, int num_sms);

void plan_simt(srmra_ctx* c) {
  const Geom& g = c->g;
  Plan& p = c->plan;
  const int slots = c->num_sms * 2;  // pass 1: two 256-thread CTAs per SM (128 registers)
  const int n_tiles = g.Spad / P1_BN;
  const int iblk1 = (int)(g.Npad / P1_BM);
  // CTAs of equal work run in waves of `slots`: pick the shift tiles per CTA that
  // minimise waves x (tiles + a quarter tile of per-CTA overhead), so that the last wave
  // is not mostly empty
  int tpg_best = 1;
  double best = 0.0;
  for (int tpg = n_tiles; tpg >= 1; --tpg) {
    const int G = (int)ceil_div(n_tiles, tpg);
    if (ceil_div(n_tiles, G) != tpg) continue;
    const int64_t waves = ceil_div((int64_t)G * iblk1, slots);
    const double cost = (double)waves * (tpg + 0.25);
    if (best == 0.0 || cost < best) {
      best = cost;
      tpg_best = tpg;
    }
  }
  p.p1_tiles_per_group = tpg_best;
  p.p1_groups = (int)ceil_div(n_tiles, p.p1_tiles_per_group);

  const int chunks = (int)ceil_div(g.l2, P2_BP);
  p.p2_chunk_groups = (int)ceil_div(chunks, P2_MAX_GC);
  p.p2_gc = (int)ceil_div(chunks, p.p2_chunk_groups);
  const int n_iblk2 = (int)(g.Npad / P2_BI);
  const int R = (int)ceil_div(n_iblk2, p.p2_gc);
  const int64_t U = (int64_t)(g.Spad / P2_BS) * p.p2_chunk_groups;
  const int64_t T = U * R;
  const int ncl = (int)std::min<int64_t>(p2_clusters(p.p2_gc, c->num_sms), T);
  const int64_t U1 = (U / ncl) * ncl, T2 = (U - U1) * R;
  const int64_t ncl2 = std::min<int64_t>(ncl, T2);
  auto first_cluster = [&](int64_t t0) {
    int64_t cl = t0 * ncl2 / T2;
    while (cl + 1 < ncl2 && (cl + 1) * T2 / ncl2 <= t0) ++cl;
    return cl;
  };
  int nseg = 1;
  for (int64_t u = U1; u < U; ++u) {
    const int64_t t0 = (u - U1) * R;
    nseg = std::max(nseg, (int)(first_cluster(t0 + R - 1) - first_cluster(t0) + 1));
  }
  p.p2_rounds = R;
  p.p2_units = U;
  p.p2_units_whole = U1;
  p.p2_ncl = ncl;
  p.p2_nseg = nseg;
  p.p2_iblk_per_split = R * p.p2_gc;
  p.p2_nsplit = nseg;
  p.nparts_z = nseg;
  p.nparts_c = nseg * p.p2_gc;
  p.ll_blocks = (int)ceil_div(g.Npad, 256);
}

void launch_pass1_f32(srmra_ctx* c) {
  const Geom& g = c->g;
  const Plan& p = c->plan;
  const LogitScalars ls = logit_scalars(g);
  dim3 grid((unsigned)(g.Npad / P1_BM), (unsigned)p.p1_groups);
  k_p1_f32<<<grid, 256, 0, c->stream>>>(c->YcT, g.Npad, c->AxT, g.Spad, g.ldy, c->ybar,
                                         c->colb, c->colm, ls.a2, ls.c2, p.p1_tiles_per_group,
                                         g.Spad / P1_BN, g.N, c->pm, c->ps);
  c->launches++;
}

cudaError_t simt_set_attributes() {
  return cudaFuncSetAttribute(k_p2_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)P2_SMEM_BYTES);
}

// Clusters of gc pass-2 CTAs that are resident at once on the current device (one CTA
// per SM; clusters must fit within a GPU processing cluster, so this can be below
// num_sms / gc).  Without a device, num_sms / gc, which is an upper bound: more clusters
// only ever split a unit into more segments.
int p2_clusters(int gc, int num_sms) {
  const int bound = std::max(1, num_sms / gc);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return bound;
  }
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({dev, gc});
  if (it != cache.end()) return it->second;
  int n = 0;
  if (simt_set_attributes() == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(gc * bound), 1, 1);
    cfg.blockDim = dim3(P2_THREADS, 1, 1);
    cfg.dynamicSmemBytes = P2_SMEM_BYTES;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)gc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&n, k_p2_f32, &cfg) != cudaSuccess) n = 0;
  }
  cudaGetLastError();
  if (n < 1 || n > bound) n = bound;
  cache[{dev, gc}] = n;
  return n;
}

cudaError_t launch_pass2_f32(srmra_ctx* c) {
  {
    cudaError_t e = once_per_device(ATTR_SIMT_P2, simt_set_attributes);
    if (e != cudaSuccess) return e;
  }
  const Geom& g = c->g;
  const Plan& p = c->plan;
  const LogitScalars ls = logit_scalars(g);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(p.p2_gc * p.p2_ncl), 1, 1);
  cfg.blockDim = dim3(P2_THREADS, 1, 1);
  cfg.dynamicSmemBytes = P2_SMEM_BYTES;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)p.p2_gc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int n_iblk2 = (int)(g.Npad / P2_BI);
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_p2_f32, (const float*)c->YcT, (const float*)c->Yc,
                                     g.Npad, (const float*)c->AxT, g.Spad, g.ldy,
                                     (const float*)c->ybar, (const float*)c->colb,
                                     (const float*)c->colm, (const float*)c->lse2, ls.a2, ls.c2,
                                     g.N, g.S, n_iblk2, p.p2_gc, p.p2_chunk_groups, p.p2_rounds,
                                     p.p2_units, p.p2_units_whole, p.p2_ncl, p.p2_nseg, c->Zp,
                                     c->cp, c->zbp);
  c->launches++;
  return e;
}

}  // namespace srmra
