// Tensor-core (tcgen05 / TMA) form of the E-step and M-step contractions on sm_103a.
//
// Operands are bf16 (SRMRA_BF16) or split bf16 hi + lo (SRMRA_BF16X3, the product
// y * x = yh*xh + yh*xl + yl*xh accumulated in f32 on the tensor cores).  The logit of
// pass 1 and pass 2 is the same expression as in the float32 form:
//   logit2[i,s] = a2 <y'_i, T'_s> + colb[s] - c2 (ybar_i - colm[s])^2      (Eq. weights_EM)
//
// Pass 1: D[i, s] = Y'[i, :] . T'[s, :] for a 128-observation x 256-shift tile in TMEM,
//   the epilogue warps keep the running (max, sum) of 2^logit2 per observation.
// Pass 2: D[s, i] = T'[s, :] . Y'[i, :] for 128 shifts x 128 observations, the epilogue
//   turns it into weights w = 2^(logit2 - lse2[i]), written to shared memory in the
//   layout tcgen05 reads, and a second MMA accumulates Z'[s, p] += sum_i w[s,i]
//   Y'^T[p, i] for a 256-pixel chunk in TMEM (Eq. x_EM); c[s] = sum_i w[s,i] and
//   zb[s] = sum_i w[s,i] ybar_i use the same rounded weights (Eq. rho_EM).  This second
//   contraction runs on fp16 operands (same instruction kind and rate as bf16, 8x finer
//   rounding): the weights are scaled by 2^12 before rounding, which keeps weights down
//   to ~1e-8 out of the fp16 subnormal range, and the scale is removed exactly
//   afterwards.
//
// Every CTA has three roles: warp 0 issues TMA loads into a ring of 32 KB shared-memory
// slots, warp 1 issues tcgen05.mma (one thread) and owns the TMEM allocation, warps 2-5
// (128 threads, one TMEM lane each) run the epilogue.  All waits are bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "ptx_sm103.cuh"
#include "srmra_internal.cuh"

namespace srmra {

namespace {

using namespace ptx;

constexpr int SLOT = 32768;
constexpr int P1_SLOTS = 6;
constexpr int P2_SLOTS = 5;
constexpr int TC_THREADS = 192;
constexpr float W_SCALE = 4096.f;        // 2^12, weights scaled before fp16 rounding
constexpr float W_UNSCALE = 1.f / 4096.f;

struct TcP1Args {
  int nk;         // 64-wide k-blocks of the contraction over pixels
  int n_stiles;   // 256-shift tiles
  int groups;     // shift groups per observation tile
  int tpg;        // tiles per group
  int64_t n_units;
  int64_t N, Npad;
  const float* ybar;
  const float* colb;
  const float* colm;
  float a2, c2;
  float* pm;
  float* ps;
  int* status;
};

struct TcP2Args {
  int nk;           // 64-wide k-blocks of the logit contraction
  int n_stiles;     // 128-shift tiles
  int n_chunks;     // 256-pixel chunks of Z'
  int n_iblk;       // 128-observation blocks
  int iblk_per_split;
  int64_t n_units;
  int64_t N;
  int Spad, ldy;
  const float* ybar;
  const float* colb;
  const float* colm;
  const float* lse2;
  float a2, c2;
  float* Zp;
  float* cp;
  float* zbp;
  int* status;
};

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return (uint8_t*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ void raise_timeout(volatile int* abort, int* status) {
  *abort = 1;
  atomicOr(status, STATUS_TIMEOUT);
}

// ------------------------------------------------------------------------------ pass 1
template <int NPROD>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_p1_tc(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmYl,
            const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAl,
            const TcP1Args a) {
  constexpr int SPK = (NPROD == 3) ? 3 : 2;  // ring slots per k-block
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = (uint64_t*)(smem + P1_SLOTS * SLOT);
  uint64_t* empty = full + P1_SLOTS;
  uint64_t* tfull = empty + P1_SLOTS;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tptr = (uint32_t*)(drain + 1);
  volatile int* abort = (volatile int*)(tptr + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int k = 0; k < P1_SLOTS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128);
    }
    mbar_init(drain, 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tptr, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tptr;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tmY);
      prefetch_tmap(&tmA);
      uint32_t it = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; ok && u < a.n_units; u += gridDim.x) {
        const int iblk = (int)(u / a.groups), grp = (int)(u % a.groups);
        const int tb = grp * a.tpg, te = min(a.n_stiles, tb + a.tpg);
        for (int tile = tb; ok && tile < te; ++tile)
          for (int kb = 0; ok && kb < a.nk; ++kb)
            for (int sl = 0; sl < SPK; ++sl) {
              const int st = it % P1_SLOTS;
              const uint32_t ph = (it / P1_SLOTS) & 1;
              if (!mbar_wait(&empty[st], ph ^ 1, abort)) {
                ok = false;
                break;
              }
              uint8_t* dst = smem + st * SLOT;
              if (sl == 0) {
                mbar_expect_tx(&full[st], NPROD == 3 ? 32768 : 16384);
                tma_load_2d(dst, &tmY, &full[st], kb * 64, iblk * 128);
                if (NPROD == 3) tma_load_2d(dst + 16384, &tmYl, &full[st], kb * 64, iblk * 128);
              } else {
                mbar_expect_tx(&full[st], 32768);
                tma_load_2d(dst, sl == 1 ? &tmA : &tmAl, &full[st], kb * 64, tile * 256);
              }
              ++it;
            }
      }
      if (!ok) {
        raise_timeout(abort, a.status);
        // let the loads already issued land before the CTA exits
        const uint32_t lo = it > P1_SLOTS ? it - P1_SLOTS : 0;
        int zero = 0;
        for (uint32_t k = lo; k < it; ++k)
          mbar_wait(&full[k % P1_SLOTS], (k / P1_SLOTS) & 1, (volatile int*)&zero);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(128, 256);
      uint32_t it = 0, tcount = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; ok && u < a.n_units; u += gridDim.x) {
        const int grp = (int)(u % a.groups);
        const int tb = grp * a.tpg, te = min(a.n_stiles, tb + a.tpg);
        for (int tile = tb; ok && tile < te; ++tile) {
          const int b = tcount & 1;
          const uint32_t tph = (tcount >> 1) & 1;
          if (!mbar_wait(&tempty[b], tph ^ 1, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tbase + (uint32_t)(b * 256);
          for (int kb = 0; ok && kb < a.nk; ++kb) {
            int st[SPK];
            for (int sl = 0; sl < SPK; ++sl) {
              st[sl] = (it + sl) % P1_SLOTS;
              if (!mbar_wait(&full[st[sl]], ((it + sl) / P1_SLOTS) & 1, abort)) ok = false;
            }
            if (!ok) break;
            tc_fence_after();
            const uint64_t dY = desc_sw128(smem + st[0] * SLOT);
            const uint64_t dA = desc_sw128(smem + st[1] * SLOT);
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
              mma_bf16(d, desc_advance(dY, k4), desc_advance(dA, k4), idesc,
                       (kb > 0 || k4 > 0) ? 1u : 0u);
              if (NPROD == 3) {
                const uint64_t dYl = desc_sw128(smem + st[0] * SLOT + 16384);
                const uint64_t dAl = desc_sw128(smem + st[SPK - 1] * SLOT);
                mma_bf16(d, desc_advance(dY, k4), desc_advance(dAl, k4), idesc, 1u);
                mma_bf16(d, desc_advance(dYl, k4), desc_advance(dA, k4), idesc, 1u);
              }
            }
            for (int sl = 0; sl < SPK; ++sl) mma_commit(&empty[st[sl]]);
            it += SPK;
          }
          if (!ok) break;
          mma_commit(&tfull[b]);
          ++tcount;
        }
      }
      if (!ok) {
        raise_timeout(abort, a.status);
        mma_commit(drain);  // all issued MMAs complete before TMEM is released
        int zero = 0;
        mbar_wait(drain, 0, (volatile int*)&zero);
      }
    }
  } else {
    const int q = warp & 3;  // TMEM lane quadrant of this warp
    const int row = q * 32 + lane;
    const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
    uint32_t tcount = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; ok && u < a.n_units; u += gridDim.x) {
      const int iblk = (int)(u / a.groups), grp = (int)(u % a.groups);
      const int tb = grp * a.tpg, te = min(a.n_stiles, tb + a.tpg);
      const int64_t i = (int64_t)iblk * 128 + row;
      const float yb = a.ybar[i];
      float rm = -INFINITY, rs = 0.f;
      for (int tile = tb; tile < te; ++tile) {
        const int b = tcount & 1;
        const uint32_t tph = (tcount >> 1) & 1;
        ok = __all_sync(0xffffffffu, mbar_wait(&tfull[b], tph, abort));
        if (!ok) break;
        tc_fence_after();
#pragma unroll 1
        for (int c = 0; c < 8; ++c) {
          float v[32];
          tmem_ld32(lane_addr + (uint32_t)(b * 256 + c * 32), v);
          tmem_ld_wait();
          const int sb = tile * 256 + c * 32;
          float mx = -INFINITY;
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const float dd = yb - a.colm[sb + e];
            v[e] = fmaf(v[e], a.a2, a.colb[sb + e]) - a.c2 * dd * dd;
            mx = fmaxf(mx, v[e]);
          }
          const float nm = fmaxf(rm, mx);
          const float base = (nm == -INFINITY) ? 0.f : nm;
          float sm = 0.f;
#pragma unroll
          for (int e = 0; e < 32; ++e) sm += exp2f(v[e] - base);
          rs = rs * exp2f(rm - base) + sm;
          rm = nm;
        }
        tc_fence_before();
        mbar_arrive(&tempty[b]);
        ++tcount;
      }
      if (ok && i < a.N) {
        a.pm[grp * a.Npad + i] = rm;
        a.ps[grp * a.Npad + i] = rs;
      }
    }
    if (!ok) raise_timeout(abort, a.status);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// ------------------------------------------------------------------------------ pass 2
template <int NPROD>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_p2_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAl,
            const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmYl,
            const __grid_constant__ CUtensorMap tmYT, const TcP2Args a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* pbuf = smem + P2_SLOTS * SLOT;  // 2 x 32 KB weight tiles (K-major, SW128)
  uint64_t* full = (uint64_t*)(pbuf + 2 * SLOT);
  uint64_t* empty = full + P2_SLOTS;
  uint64_t* sfull = empty + P2_SLOTS;
  uint64_t* sempty = sfull + 2;
  uint64_t* pfull = sempty + 2;
  uint64_t* pempty = pfull + 2;
  uint64_t* zfull = pempty + 2;
  uint64_t* zempty = zfull + 1;
  uint64_t* drain = zempty + 1;
  uint32_t* tptr = (uint32_t*)(drain + 1);
  volatile int* abort = (volatile int*)(tptr + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_split = a.n_stiles * a.n_chunks;

  if (threadIdx.x == 0) {
    for (int k = 0; k < P2_SLOTS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sfull[b], 1);
      mbar_init(&sempty[b], 128);
      mbar_init(&pfull[b], 128);
      mbar_init(&pempty[b], 1);
    }
    mbar_init(zfull, 1);
    mbar_init(zempty, 128);
    mbar_init(drain, 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tptr, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tptr;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tmA);
      prefetch_tmap(&tmY);
      prefetch_tmap(&tmYT);
      uint32_t it = 0;
      bool ok = true;
      auto next_slot = [&](uint32_t bytes) -> uint8_t* {
        const int st = it % P2_SLOTS;
        if (!mbar_wait(&empty[st], ((it / P2_SLOTS) & 1) ^ 1, abort)) {
          ok = false;
          return nullptr;
        }
        mbar_expect_tx(&full[st], bytes);
        return smem + st * SLOT;
      };
      for (int64_t u = blockIdx.x; ok && u < a.n_units; u += gridDim.x) {
        const int split = (int)(u / per_split), rem = (int)(u % per_split);
        const int stile = rem / a.n_chunks, chunk = rem % a.n_chunks;
        const int jb0 = split * a.iblk_per_split;
        const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
        for (int j = 0; ok && j <= nb; ++j) {
          if (j < nb) {
            const int ib = (jb0 + j) * 128;
            for (int kb = 0; ok && kb < a.nk; ++kb) {
              if (NPROD == 3) {
                uint8_t* s0 = next_slot(32768);
                if (!ok) break;
                tma_load_2d(s0, &tmA, &full[it % P2_SLOTS], kb * 64, stile * 128);
                tma_load_2d(s0 + 16384, &tmAl, &full[it % P2_SLOTS], kb * 64, stile * 128);
                ++it;
                uint8_t* s1 = next_slot(32768);
                if (!ok) break;
                tma_load_2d(s1, &tmY, &full[it % P2_SLOTS], kb * 64, ib);
                tma_load_2d(s1 + 16384, &tmYl, &full[it % P2_SLOTS], kb * 64, ib);
                ++it;
              } else {
                uint8_t* s0 = next_slot(32768);
                if (!ok) break;
                tma_load_2d(s0, &tmA, &full[it % P2_SLOTS], kb * 64, stile * 128);
                tma_load_2d(s0 + 16384, &tmY, &full[it % P2_SLOTS], kb * 64, ib);
                ++it;
              }
            }
          }
          if (ok && j >= 1) {
            const int ib = (jb0 + j - 1) * 128;
            for (int h = 0; ok && h < 2; ++h) {
              uint8_t* s0 = next_slot(32768);
              if (!ok) break;
              tma_load_2d(s0, &tmYT, &full[it % P2_SLOTS], ib + h * 64, chunk * 256);
              ++it;
            }
          }
        }
      }
      if (!ok) {
        raise_timeout(abort, a.status);
        const uint32_t lo = it > P2_SLOTS ? it - P2_SLOTS : 0;
        int zero = 0;
        for (uint32_t k = lo; k < it; ++k)
          mbar_wait(&full[k % P2_SLOTS], (k / P2_SLOTS) & 1, (volatile int*)&zero);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16_f32(128, 128);
      constexpr uint32_t idZ = idesc_f16_f32(128, 256);
      uint32_t it = 0, sc = 0, pz = 0, uc = 0;
      bool ok = true;
      auto wait_slot = [&]() -> uint8_t* {
        const int st = it % P2_SLOTS;
        if (!mbar_wait(&full[st], (it / P2_SLOTS) & 1, abort)) {
          ok = false;
          return nullptr;
        }
        return smem + st * SLOT;
      };
      for (int64_t u = blockIdx.x; ok && u < a.n_units; u += gridDim.x) {
        const int split = (int)(u / per_split);
        const int jb0 = split * a.iblk_per_split;
        const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
        for (int j = 0; ok && j <= nb; ++j) {
          if (j < nb) {  // logits S_j into TMEM buffer sc & 1
            const int b = sc & 1;
            if (!mbar_wait(&sempty[b], ((sc >> 1) & 1) ^ 1, abort)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tbase + (uint32_t)(b * 128);
            for (int kb = 0; ok && kb < a.nk; ++kb) {
              uint8_t* sA = wait_slot();
              if (!ok) break;
              const int stA = it % P2_SLOTS;
              uint8_t* sY = sA + 16384;
              int stY = stA;
              if (NPROD == 3) {
                ++it;
                sY = wait_slot();
                if (!ok) break;
                stY = it % P2_SLOTS;
              }
              tc_fence_after();
              const uint64_t dA = desc_sw128(sA), dY = desc_sw128(sY);
#pragma unroll
              for (int k4 = 0; k4 < 4; ++k4) {
                mma_bf16(d, desc_advance(dA, k4), desc_advance(dY, k4), idS,
                         (kb > 0 || k4 > 0) ? 1u : 0u);
                if (NPROD == 3) {
                  const uint64_t dAl = desc_sw128(sA + 16384), dYl = desc_sw128(sY + 16384);
                  mma_bf16(d, desc_advance(dA, k4), desc_advance(dYl, k4), idS, 1u);
                  mma_bf16(d, desc_advance(dAl, k4), desc_advance(dY, k4), idS, 1u);
                }
              }
              mma_commit(&empty[stA]);
              if (NPROD == 3) mma_commit(&empty[stY]);
              ++it;
            }
            if (!ok) break;
            mma_commit(&sfull[b]);
            ++sc;
          }
          if (j >= 1) {  // Z' += W_{j-1} . Y'^T
            const int jj = j - 1;
            const int pb = pz & 1;
            if (jj == 0 && !mbar_wait(zempty, (uc & 1) ^ 1, abort)) {
              ok = false;
              break;
            }
            if (!mbar_wait(&pfull[pb], (pz >> 1) & 1, abort)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t dZ = tbase + 256u;
            for (int h = 0; ok && h < 2; ++h) {
              uint8_t* sT = wait_slot();
              if (!ok) break;
              tc_fence_after();
              const uint64_t dP = desc_sw128(pbuf + pb * SLOT + h * 16384);
              const uint64_t dT = desc_sw128(sT);
#pragma unroll
              for (int k4 = 0; k4 < 4; ++k4)
                mma_bf16(dZ, desc_advance(dP, k4), desc_advance(dT, k4), idZ,
                         (jj > 0 || h > 0 || k4 > 0) ? 1u : 0u);
              mma_commit(&empty[it % P2_SLOTS]);
              ++it;
            }
            if (!ok) break;
            mma_commit(&pempty[pb]);
            ++pz;
          }
        }
        if (!ok) break;
        mma_commit(zfull);
        ++uc;
      }
      if (!ok) {
        raise_timeout(abort, a.status);
        mma_commit(drain);
        int zero = 0;
        mbar_wait(drain, 0, (volatile int*)&zero);
      }
    }
  } else {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
    uint32_t sc = 0, pz = 0, uc = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; ok && u < a.n_units; u += gridDim.x) {
      const int split = (int)(u / per_split), rem = (int)(u % per_split);
      const int stile = rem / a.n_chunks, chunk = rem % a.n_chunks;
      const int jb0 = split * a.iblk_per_split;
      const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
      const int s = stile * 128 + row;
      const float cb = a.colb[s], cm = a.colm[s];
      float cacc = 0.f, zacc = 0.f;
      for (int j = 0; j < nb; ++j) {
        const int64_t ib = (int64_t)(jb0 + j) * 128;
        const int b = sc & 1, pb = pz & 1;
        ok = __all_sync(0xffffffffu, mbar_wait(&sfull[b], (sc >> 1) & 1, abort));
        if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&pempty[pb], ((pz >> 1) & 1) ^ 1, abort));
        if (!ok) break;
        tc_fence_after();
        uint8_t* prow = pbuf + pb * SLOT + row * 128;
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          float v[32];
          tmem_ld32(lane_addr + (uint32_t)(b * 128 + c * 32), v);
          tmem_ld_wait();
          uint32_t packed[16];
#pragma unroll
          for (int e = 0; e < 32; e += 2) {
            float w2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int64_t i = ib + c * 32 + e + h;
              const float ybi = a.ybar[i];
              const float dd = ybi - cm;
              const float val = fmaf(v[e + h], a.a2, cb - a.lse2[i]) - a.c2 * dd * dd;
              const float w = (i < a.N) ? exp2f(val) * W_SCALE : 0.f;
              w2[h] = __half2float(__float2half_rn(w));
              cacc += w2[h];
              zacc = fmaf(w2[h], ybi, zacc);
            }
            const __half2 pr = __floats2half2_rn(w2[0], w2[1]);
            packed[e >> 1] = *reinterpret_cast<const uint32_t*>(&pr);
          }
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const int col16 = c * 4 + g;           // 16-byte unit along the observations
            const int kb2 = col16 >> 3, cc = col16 & 7;
            uint4 val = make_uint4(packed[4 * g], packed[4 * g + 1], packed[4 * g + 2],
                                   packed[4 * g + 3]);
            *reinterpret_cast<uint4*>(prow + kb2 * 16384 + ((cc ^ (row & 7)) << 4)) = val;
          }
        }
        tc_fence_before();
        mbar_arrive(&sempty[b]);
        fence_proxy_async_smem();
        mbar_arrive(&pfull[pb]);
        ++sc;
        ++pz;
      }
      if (!ok) break;
      ok = __all_sync(0xffffffffu, mbar_wait(zfull, uc & 1, abort));
      if (!ok) break;
      tc_fence_after();
      float* zrow = a.Zp + ((int64_t)split * a.Spad + s) * a.ldy;
#pragma unroll 1
      for (int c = 0; c < 8; ++c) {
        float v[32];
        tmem_ld32(lane_addr + (uint32_t)(256 + c * 32), v);
        tmem_ld_wait();
        const int p0 = chunk * 256 + c * 32;
        if (p0 < a.ldy) {
#pragma unroll
          for (int e = 0; e < 32; e += 4)
            if (p0 + e < a.ldy)
              *reinterpret_cast<float4*>(zrow + p0 + e) =
                  make_float4(v[e] * W_UNSCALE, v[e + 1] * W_UNSCALE, v[e + 2] * W_UNSCALE,
                              v[e + 3] * W_UNSCALE);
        }
      }
      tc_fence_before();
      mbar_arrive(zempty);
      if (chunk == 0) {
        a.cp[(int64_t)split * a.Spad + s] = cacc * W_UNSCALE;
        a.zbp[(int64_t)split * a.Spad + s] = zacc * W_UNSCALE;
      }
      ++uc;
    }
    if (!ok) raise_timeout(abort, a.status);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

constexpr size_t P1_SMEM = 1024 + P1_SLOTS * SLOT + 256;
constexpr size_t P2_SMEM = 1024 + P2_SLOTS * SLOT + 2 * SLOT + 256;

// ------------------------------------------------------------------------------ operands
// y' -> bf16 hi / lo rows [Npad][ldk] (zero padding beyond l2).
__global__ void k_split_obs(const float* __restrict__ Yc, int ldy, int l2, int64_t Npad,
                            int ldk, __nv_bfloat16* __restrict__ Yh,
                            __nv_bfloat16* __restrict__ Yl) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Npad * ldk) return;
  const int64_t i = idx / ldk;
  const int k = (int)(idx % ldk);
  const float v = (k < l2) ? Yc[i * ldy + k] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  Yh[idx] = h;
  if (Yl) Yl[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// YT[p][i] = fp16(y'_i[p]) for p < l2 (32x32 tiles): the M-step operand.
__global__ void k_transpose_f16(const float* __restrict__ in, int64_t R, int ld_in, int C,
                                __half* __restrict__ out) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32;
  const int c0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int64_t r = r0 + k;
    const int c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < R && c < C) ? in[r * ld_in + c] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int c = c0 + k;
    const int64_t r = r0 + threadIdx.x;
    if (c < C && r < R) out[(int64_t)c * R + r] = __float2half_rn(tile[threadIdx.x][k]);
  }
}

__device__ __forceinline__ int mod_pos(int a, int m) {
  const int r = a % m;
  return r < 0 ? r + m : r;
}

// Centred templates, shift-major bf16 hi / lo: T[s][n] = x'_r(s)[n - t(s)].
__global__ void k_templates_bf16(const float* __restrict__ x, const double* __restrict__ sub,
                                 int L, int K, int l, int S, int Spad, int l2, int ldk,
                                 __nv_bfloat16* __restrict__ Ah,
                                 __nv_bfloat16* __restrict__ Al) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)Spad * ldk) return;
  const int s = (int)(idx / ldk), n = (int)(idx % ldk);
  float v = 0.f;
  if (s < S && n < l2) {
    const int s1 = s / L, s2 = s % L;
    const int r1 = mod_pos(-s1, K), r2 = mod_pos(-s2, K);
    const int t1 = ((s1 + r1) / K) % l, t2 = ((s2 + r2) / K) % l;
    const int m1 = mod_pos(n / l - t1, l), m2 = mod_pos(n % l - t2, l);
    v = (float)((double)x[(r1 + m1 * K) * L + r2 + m2 * K] - sub[r1 * K + r2]);
  }
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  Ah[idx] = h;
  if (Al) Al[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2D 16-bit (bf16 or fp16) tensor map with 128-byte swizzle: `rows` rows of `inner` elements, row pitch
// `pitch` elements, box of 64 x box_rows.
bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint64_t pitch,
              uint32_t box_rows,
              CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {pitch * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, dt, 2, const_cast<void*>(base), dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

void plan_tc(srmra_ctx* c) {
  const Geom& g = c->g;
  Plan& p = c->plan;
  const int sms = c->num_sms;
  const int n_st1 = g.Spad / 256;
  const int iblk1 = (int)(g.Npad / 128);
  int G = (int)ceil_div(4 * (int64_t)sms, iblk1);
  G = G < 1 ? 1 : (G > n_st1 ? n_st1 : G);
  p.p1_tiles_per_group = (int)ceil_div(n_st1, G);
  p.p1_groups = (int)ceil_div(n_st1, p.p1_tiles_per_group);

  const int n_st2 = g.Spad / 128;
  const int chunks = (int)ceil_div(g.l2, 256);
  const int n_iblk = (int)(g.Npad / 128);
  const int64_t per_split = (int64_t)n_st2 * chunks;
  int ns = (int)((4 * (int64_t)sms + per_split / 2) / per_split);
  ns = ns < 1 ? 1 : (ns > n_iblk ? n_iblk : ns);
  if (ns > 32) ns = 32;
  p.p2_iblk_per_split = (int)ceil_div(n_iblk, ns);
  p.p2_nsplit = (int)ceil_div(n_iblk, p.p2_iblk_per_split);
  p.p2_gc = 1;
  p.p2_chunk_groups = chunks;
  p.nparts_z = p.p2_nsplit;
  p.nparts_c = p.p2_nsplit;
  p.ll_blocks = (int)ceil_div(g.Npad, 256);
}

cudaError_t prep_obs_tc(srmra_ctx* c) {
  const Geom& g = c->g;
  const int64_t n = g.Npad * g.ldk;
  k_split_obs<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(
      c->Yc, g.ldy, g.l2, g.Npad, g.ldk, c->Yh, c->prec == SRMRA_BF16X3 ? c->Yl : nullptr);
  dim3 grid((unsigned)ceil_div(g.l2, 32), (unsigned)ceil_div(g.Npad, 32));
  k_transpose_f16<<<grid, dim3(32, 8), 0, c->stream>>>(c->Yc, g.Npad, g.ldy, g.l2, c->YTf);
  c->launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // tensor maps over the fixed operands
  bool ok = make_map(&c->tmY128, c->Yh, g.ldk, g.Npad, g.ldk, 128) &&
            make_map(&c->tmYT, c->YTf, g.Npad, g.l2, g.Npad, 256,
                     CU_TENSOR_MAP_DATA_TYPE_FLOAT16) &&
            make_map(&c->tmA128, c->Ah, g.ldk, g.Spad, g.ldk, 128) &&
            make_map(&c->tmA256, c->Ah, g.ldk, g.Spad, g.ldk, 256);
  if (ok && c->prec == SRMRA_BF16X3)
    ok = make_map(&c->tmYl128, c->Yl, g.ldk, g.Npad, g.ldk, 128) &&
         make_map(&c->tmAl128, c->Al, g.ldk, g.Spad, g.ldk, 128) &&
         make_map(&c->tmAl256, c->Al, g.ldk, g.Spad, g.ldk, 256);
  if (!ok) return cudaErrorInvalidValue;
  return cudaSuccess;
}

void launch_templates_tc(srmra_ctx* c) {
  const Geom& g = c->g;
  const int64_t n = (int64_t)g.Spad * g.ldk;
  k_templates_bf16<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(
      c->x, c->sub, g.L, g.K, g.l, g.S, g.Spad, g.l2, g.ldk, c->Ah,
      c->prec == SRMRA_BF16X3 ? c->Al : nullptr);
  c->launches++;
}

cudaError_t launch_pass1_tc(srmra_ctx* c) {
  const Geom& g = c->g;
  const Plan& p = c->plan;
  const LogitScalars ls = logit_scalars(g);
  TcP1Args a;
  a.nk = (int)ceil_div(g.l2, 64);
  a.n_stiles = g.Spad / 256;
  a.groups = p.p1_groups;
  a.tpg = p.p1_tiles_per_group;
  a.n_units = (g.Npad / 128) * p.p1_groups;
  a.N = g.N;
  a.Npad = g.Npad;
  a.ybar = c->ybar;
  a.colb = c->colb;
  a.colm = c->colm;
  a.a2 = ls.a2;
  a.c2 = ls.c2;
  a.pm = c->pm;
  a.ps = c->ps;
  a.status = c->status;
  const unsigned grid = (unsigned)(a.n_units < c->num_sms ? a.n_units : c->num_sms);
  cudaError_t e;
  if (c->prec == SRMRA_BF16X3) {
    static bool once = false;
    if (!once) {
      e = set_smem(k_p1_tc<3>, P1_SMEM);
      if (e != cudaSuccess) return e;
      once = true;
    }
    k_p1_tc<3><<<grid, TC_THREADS, P1_SMEM, c->stream>>>(c->tmY128, c->tmYl128, c->tmA256,
                                                         c->tmAl256, a);
  } else {
    static bool once = false;
    if (!once) {
      e = set_smem(k_p1_tc<1>, P1_SMEM);
      if (e != cudaSuccess) return e;
      once = true;
    }
    k_p1_tc<1><<<grid, TC_THREADS, P1_SMEM, c->stream>>>(c->tmY128, c->tmY128, c->tmA256,
                                                         c->tmA256, a);
  }
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_pass2_tc(srmra_ctx* c) {
  const Geom& g = c->g;
  const Plan& p = c->plan;
  const LogitScalars ls = logit_scalars(g);
  TcP2Args a;
  a.nk = (int)ceil_div(g.l2, 64);
  a.n_stiles = g.Spad / 128;
  a.n_chunks = (int)ceil_div(g.l2, 256);
  a.n_iblk = (int)(g.Npad / 128);
  a.iblk_per_split = p.p2_iblk_per_split;
  a.n_units = (int64_t)a.n_stiles * a.n_chunks * p.p2_nsplit;
  a.N = g.N;
  a.Spad = g.Spad;
  a.ldy = g.ldy;
  a.ybar = c->ybar;
  a.colb = c->colb;
  a.colm = c->colm;
  a.lse2 = c->lse2;
  a.a2 = ls.a2;
  a.c2 = ls.c2;
  a.Zp = c->Zp;
  a.cp = c->cp;
  a.zbp = c->zbp;
  a.status = c->status;
  const unsigned grid = (unsigned)(a.n_units < c->num_sms ? a.n_units : c->num_sms);
  cudaError_t e;
  if (c->prec == SRMRA_BF16X3) {
    static bool once = false;
    if (!once) {
      e = set_smem(k_p2_tc<3>, P2_SMEM);
      if (e != cudaSuccess) return e;
      once = true;
    }
    k_p2_tc<3><<<grid, TC_THREADS, P2_SMEM, c->stream>>>(c->tmA128, c->tmAl128, c->tmY128,
                                                         c->tmYl128, c->tmYT, a);
  } else {
    static bool once = false;
    if (!once) {
      e = set_smem(k_p2_tc<1>, P2_SMEM);
      if (e != cudaSuccess) return e;
      once = true;
    }
    k_p2_tc<1><<<grid, TC_THREADS, P2_SMEM, c->stream>>>(c->tmA128, c->tmA128, c->tmY128,
                                                         c->tmY128, c->tmYT, a);
  }
  c->launches++;
  return cudaGetLastError();
}

}  // namespace srmra
