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

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "ptx_sm103.cuh"
#include "srmra_internal.cuh"

namespace srmra {

namespace {

using namespace ptx;

constexpr int SLOT = 32768;
constexpr int P1_SLOTS = 6;
constexpr int P2_SLOTS_PLAIN = 5;  // per-chunk pass 2: operand ring slots
constexpr int P2_SLOTS_COMP = 3;   // the same with the compensated M-step
constexpr int P2_MAX_ACC = 512;    // MMAs added into one Z' accumulator (see plan_tc)
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
  uint64_t wait_ns;  // limit of every bounded wait of the launch (instance 0's is used)
  int hook;          // test hook (srmra_set_wait_limit): 1 = a wait in pass 1 that never ends
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
  uint64_t wait_ns;  // limit of every bounded wait of the launch (instance 0's is used)
  int hook;          // test hook (srmra_set_wait_limit): 2 = a wait in pass 2 that never ends
};

// One problem instance of a (possibly grouped) launch: the tensor maps of its operands
// and the arguments of both passes.  Kept in device memory; TMA reads the maps there.
struct TcInst {
  CUtensorMap tmY, tmYl, tmA256, tmAl256, tmA128, tmAl128, tmYT, tmYTl;
  // pair form: 64-observation boxes of Y' (hi, lo) and 128-pixel boxes of Y'^T
  CUtensorMap tmY64, tmYl64, tmYT128;
  TcP1Args p1;
  TcP2Args p2;
};

// Instance of global work unit u: the largest k with ustart[k] <= u (ustart ascending,
// ustart[n] = total units).
__device__ __forceinline__ int find_inst(const int64_t* __restrict__ ustart, int n, int64_t u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ustart[mid] <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return (uint8_t*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ void raise_timeout(volatile int* abort, int* status) {
  *abort = 1;
  atomicOr(status, STATUS_TIMEOUT);
}

// ------------------------------------------------------------------------------ pass 1
// BN is the shift width of a tile: 256 (two TMEM accumulators of 256 columns) or 128
// (four of 128, so that the MMAs can run further ahead of the epilogue; the template
// tile of a k-block, hi and lo, then shares one ring slot).  Every instance of a
// launch has the same BN (its p1 arguments are counted in BN-wide tiles).
template <int NPROD, int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_p1_tc(const TcInst* __restrict__ insts, const int64_t* __restrict__ ustart, int n_inst,
            int* status) {
  static_assert(BN == 256 || BN == 128, "pass-1 tiles are 128 or 256 shifts wide");
  constexpr int SPK = (NPROD == 3 && BN == 256) ? 3 : 2;  // ring slots per k-block
  constexpr int NB = 512 / BN;                             // TMEM accumulators
  constexpr uint32_t A_BYTES = BN * 128;                   // one template part, one k-block
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = (uint64_t*)(smem + P1_SLOTS * SLOT);
  uint64_t* empty = full + P1_SLOTS;
  uint64_t* tfull = empty + P1_SLOTS;
  uint64_t* tempty = tfull + NB;
  uint64_t* drain = tempty + NB;
  uint64_t* never = drain + 1;  // nothing arrives on it (test hook)
  uint32_t* tptr = (uint32_t*)(never + 1);
  volatile int* abort = (volatile int*)(tptr + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t wlim = insts[0].p1.wait_ns;
  const int hook = insts[0].p1.hook;

  if (threadIdx.x == 0) {
    for (int k = 0; k < P1_SLOTS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128);
    }
    mbar_init(drain, 1);
    mbar_init(never, 1);
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
  const int64_t total = ustart[n_inst];

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; ok && u < total; u += gridDim.x) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP1Args& a = I->p1;
        const int64_t lu = u - ustart[ki];
        const int iblk = (int)(lu / a.groups), grp = (int)(lu % a.groups);
        const int tb = grp * a.tpg, te = min(a.n_stiles, tb + a.tpg);
        for (int tile = tb; ok && tile < te; ++tile)
          for (int kb = 0; ok && kb < a.nk; ++kb)
            for (int sl = 0; sl < SPK; ++sl) {
              const int st = it % P1_SLOTS;
              const uint32_t ph = (it / P1_SLOTS) & 1;
              if (!mbar_wait(&empty[st], ph ^ 1, abort, wlim)) {
                ok = false;
                break;
              }
              uint8_t* dst = smem + st * SLOT;
              if (sl == 0) {
                mbar_expect_tx(&full[st], NPROD == 3 ? 32768 : 16384);
                tma_load_2d(dst, &I->tmY, &full[st], kb * 64, iblk * 128);
                if (NPROD == 3) tma_load_2d(dst + 16384, &I->tmYl, &full[st], kb * 64, iblk * 128);
              } else if (BN == 256) {
                mbar_expect_tx(&full[st], 32768);
                tma_load_2d(dst, sl == 1 ? &I->tmA256 : &I->tmAl256, &full[st], kb * 64, tile * 256);
              } else {  // 128-row template parts, hi then lo, in one slot
                mbar_expect_tx(&full[st], NPROD == 3 ? 2 * A_BYTES : A_BYTES);
                tma_load_2d(dst, &I->tmA128, &full[st], kb * 64, tile * 128);
                if (NPROD == 3)
                  tma_load_2d(dst + A_BYTES, &I->tmAl128, &full[st], kb * 64, tile * 128);
              }
              ++it;
            }
      }
      if (!ok) raise_timeout(abort, status);
      {
        // the fills already issued land before the CTA exits, also when another role
        // gave up and stopped consuming them (in a normal run they are all consumed and
        // these waits return at once)
        const uint32_t lo = it > P1_SLOTS ? it - P1_SLOTS : 0;
        int zero = 0;
        for (uint32_t k = lo; k < it; ++k)
          mbar_wait(&full[k % P1_SLOTS], (k / P1_SLOTS) & 1, (volatile int*)&zero);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(128, BN);
      uint32_t it = 0, tcount = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; ok && u < total; u += gridDim.x) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP1Args& a = I->p1;
        const int64_t lu = u - ustart[ki];
        const int grp = (int)(lu % a.groups);
        const int tb = grp * a.tpg, te = min(a.n_stiles, tb + a.tpg);
        for (int tile = tb; ok && tile < te; ++tile) {
          const int b = tcount % NB;
          const uint32_t tph = (tcount / NB) & 1;
          if (!mbar_wait(&tempty[b], tph ^ 1, abort, wlim)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tbase + (uint32_t)(b * BN);
          for (int kb = 0; ok && kb < a.nk; ++kb) {
            int st[SPK];
            for (int sl = 0; sl < SPK; ++sl) {
              st[sl] = (it + sl) % P1_SLOTS;
              if (!mbar_wait(&full[st[sl]], ((it + sl) / P1_SLOTS) & 1, abort, wlim)) ok = false;
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
                const uint64_t dAl = desc_sw128(BN == 256 ? smem + st[SPK - 1] * SLOT
                                                          : smem + st[1] * SLOT + A_BYTES);
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
      if (!ok) raise_timeout(abort, status);
      // every issued MMA completes before TMEM is released, also when another role
      // gave up and left accumulators unread
      mma_commit(drain);
      int zero = 0;
      mbar_wait(drain, 0, (volatile int*)&zero);
    }
  } else {
    const int q = warp & 3;  // TMEM lane quadrant of this warp
    const int row = q * 32 + lane;
    const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
    float2* wcol = (float2*)(smem + P1_SLOTS * SLOT + 256) + q * 32;  // this warp's staging
    uint32_t tcount = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; ok && u < total; u += gridDim.x) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP1Args& a = I->p1;
        const int64_t lu = u - ustart[ki];
      const int iblk = (int)(lu / a.groups), grp = (int)(lu % a.groups);
      const int tb = grp * a.tpg, te = min(a.n_stiles, tb + a.tpg);
      const int64_t i = (int64_t)iblk * 128 + row;
      const float yb = a.ybar[i];
      const float a2 = a.a2, c2 = a.c2;
      const float* __restrict__ colb = a.colb;
      const float* __restrict__ colm = a.colm;
      float rm = -INFINITY, rs = 0.f;
      // (colb, colm) of the next 32-column chunk, loaded one chunk ahead of its use
      float nb_ = colb[tb * BN + lane], nm_ = colm[tb * BN + lane];
      for (int tile = tb; tile < te; ++tile) {
        const int b = tcount % NB;
        const uint32_t tph = (tcount / NB) & 1;
        // test hook: the first CTA's epilogue first waits on a barrier that nothing
        // completes, so that the wait runs out after the limit and the launch reports a
        // timeout through the ordinary abort path
        const bool held = hook == 1 && blockIdx.x == 0 && tcount == 0;
        ok = __all_sync(0xffffffffu, (!held || mbar_wait(never, 0, abort, wlim)) &&
                                         mbar_wait(&tfull[b], tph, abort, wlim));
        if (!ok) break;
        tc_fence_after();
        constexpr int NCH = BN / 32;  // 32-column chunks of a tile
#pragma unroll 1
        for (int c = 0; c < NCH; ++c) {
          __syncwarp();  // the warp is done with the previous chunk's terms
          wcol[lane] = make_float2(nb_, nm_);
          __syncwarp();
          const int nx = (c < NCH - 1) ? tile * BN + (c + 1) * 32 : (tile + 1) * BN;
          if (c < NCH - 1 || tile + 1 < te) {
            nb_ = colb[nx + lane];
            nm_ = colm[nx + lane];
          }
          float v[32];
          tmem_ld32(lane_addr + (uint32_t)(b * BN + c * 32), v);
          tmem_ld_wait();
          float mx = -INFINITY;
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const float2 cbm = wcol[e];
            const float dd = yb - cbm.y;
            v[e] = fmaf(v[e], a2, cbm.x) - c2 * dd * dd;
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
    if (!ok) raise_timeout(abort, status);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// ------------------------------------------------------------------------------ pass 2
// Per pixel chunk.  COMP selects the compensated M-step: the weights and Y' are each
// split into fp16 hi + lo parts and Z' accumulates Wh Yh' + Wh Yl' + Wl Yh' (the
// dropped Wl Yl' is below 2^-22 relative), so the rounding of the 16-bit operands no
// longer needs many observations to average out (Eq. x_EM); c and zb take Wh + Wl.
// The two weight tiles of a block take 64 KB, so the operand ring has 3 slots.
template <int NPROD, bool COMP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_p2_tc(const TcInst* __restrict__ insts, const int64_t* __restrict__ ustart, int n_inst,
            int* status) {
  constexpr int P2_SLOTS = COMP ? P2_SLOTS_COMP : P2_SLOTS_PLAIN;
  constexpr int WB = COMP ? 2 * SLOT : SLOT;  // one weight buffer: hi tile [+ lo tile]
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* pbuf = smem + P2_SLOTS * SLOT;  // 2 weight buffers (K-major, SW128)
  uint64_t* full = (uint64_t*)(pbuf + 2 * WB);
  uint64_t* empty = full + P2_SLOTS;
  uint64_t* sfull = empty + P2_SLOTS;
  uint64_t* sempty = sfull + 2;
  uint64_t* pfull = sempty + 2;
  uint64_t* pempty = pfull + 2;
  uint64_t* zfull = pempty + 2;
  uint64_t* zempty = zfull + 1;
  uint64_t* drain = zempty + 1;
  uint64_t* never = drain + 1;  // nothing arrives on it (test hook)
  uint32_t* tptr = (uint32_t*)(never + 1);
  volatile int* abort = (volatile int*)(tptr + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t wlim = insts[0].p2.wait_ns;
  const int hook = insts[0].p2.hook;

  if (threadIdx.x == 0) {
    mbar_init(never, 1);
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
  const int64_t total = ustart[n_inst];

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      auto next_slot = [&](uint32_t bytes) -> uint8_t* {
        const int st = it % P2_SLOTS;
        if (!mbar_wait(&empty[st], ((it / P2_SLOTS) & 1) ^ 1, abort, wlim)) {
          ok = false;
          return nullptr;
        }
        mbar_expect_tx(&full[st], bytes);
        return smem + st * SLOT;
      };
      for (int64_t u = blockIdx.x; ok && u < total; u += gridDim.x) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP2Args& a = I->p2;
        const int64_t lu = u - ustart[ki];
        const int per_split = a.n_stiles * a.n_chunks;
        const int split = (int)(lu / per_split), rem = (int)(lu % per_split);
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
                tma_load_2d(s0, &I->tmA128, &full[it % P2_SLOTS], kb * 64, stile * 128);
                tma_load_2d(s0 + 16384, &I->tmAl128, &full[it % P2_SLOTS], kb * 64, stile * 128);
                ++it;
                uint8_t* s1 = next_slot(32768);
                if (!ok) break;
                tma_load_2d(s1, &I->tmY, &full[it % P2_SLOTS], kb * 64, ib);
                tma_load_2d(s1 + 16384, &I->tmYl, &full[it % P2_SLOTS], kb * 64, ib);
                ++it;
              } else {
                uint8_t* s0 = next_slot(32768);
                if (!ok) break;
                tma_load_2d(s0, &I->tmA128, &full[it % P2_SLOTS], kb * 64, stile * 128);
                tma_load_2d(s0 + 16384, &I->tmY, &full[it % P2_SLOTS], kb * 64, ib);
                ++it;
              }
            }
          }
          if (ok && j >= 1) {
            const int ib = (jb0 + j - 1) * 128;
            for (int h = 0; ok && h < 2; ++h) {
              uint8_t* s0 = next_slot(32768);
              if (!ok) break;
              tma_load_2d(s0, &I->tmYT, &full[it % P2_SLOTS], ib + h * 64, chunk * 256);
              ++it;
              if (COMP) {  // the lo part of the same Y'^T tile
                uint8_t* s1 = next_slot(32768);
                if (!ok) break;
                tma_load_2d(s1, &I->tmYTl, &full[it % P2_SLOTS], ib + h * 64, chunk * 256);
                ++it;
              }
            }
          }
        }
      }
      if (!ok) raise_timeout(abort, status);
      {
        // the fills already issued land before the CTA exits, also when another role
        // gave up and stopped consuming them (in a normal run they are all consumed and
        // these waits return at once)
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
        if (!mbar_wait(&full[st], (it / P2_SLOTS) & 1, abort, wlim)) {
          ok = false;
          return nullptr;
        }
        return smem + st * SLOT;
      };
      for (int64_t u = blockIdx.x; ok && u < total; u += gridDim.x) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP2Args& a = I->p2;
        const int64_t lu = u - ustart[ki];
        const int per_split = a.n_stiles * a.n_chunks;
        const int split = (int)(lu / per_split);
        const int jb0 = split * a.iblk_per_split;
        const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
        for (int j = 0; ok && j <= nb; ++j) {
          if (j < nb) {  // logits S_j into TMEM buffer sc & 1
            const int b = sc & 1;
            if (!mbar_wait(&sempty[b], ((sc >> 1) & 1) ^ 1, abort, wlim)) {
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
            if (jj == 0 && !mbar_wait(zempty, (uc & 1) ^ 1, abort, wlim)) {
              ok = false;
              break;
            }
            if (!mbar_wait(&pfull[pb], (pz >> 1) & 1, abort, wlim)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t dZ = tbase + 256u;
            for (int h = 0; ok && h < 2; ++h) {
              uint8_t* sT = wait_slot();
              if (!ok) break;
              const int stT = it % P2_SLOTS;
              uint8_t* sTl = sT;
              int stTl = stT;
              if (COMP) {
                ++it;
                sTl = wait_slot();
                if (!ok) break;
                stTl = it % P2_SLOTS;
              }
              tc_fence_after();
              const uint64_t dP = desc_sw128(pbuf + pb * WB + h * 16384);
              const uint64_t dT = desc_sw128(sT);
#pragma unroll
              for (int k4 = 0; k4 < 4; ++k4) {
                mma_bf16(dZ, desc_advance(dP, k4), desc_advance(dT, k4), idZ,
                         (jj > 0 || h > 0 || k4 > 0) ? 1u : 0u);
                if (COMP) {
                  const uint64_t dPl = desc_sw128(pbuf + pb * WB + SLOT + h * 16384);
                  const uint64_t dTl = desc_sw128(sTl);
                  mma_bf16(dZ, desc_advance(dP, k4), desc_advance(dTl, k4), idZ, 1u);
                  mma_bf16(dZ, desc_advance(dPl, k4), desc_advance(dT, k4), idZ, 1u);
                }
              }
              mma_commit(&empty[stT]);
              if (COMP) mma_commit(&empty[stTl]);
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
      if (!ok) raise_timeout(abort, status);
      // every issued MMA completes before TMEM is released, also when another role
      // gave up and left accumulators unread
      mma_commit(drain);
      int zero = 0;
      mbar_wait(drain, 0, (volatile int*)&zero);
    }
  } else {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
    float2* wobs = (float2*)(pbuf + 2 * WB + 256) + q * 32;  // this warp's staging
    uint32_t sc = 0, pz = 0, uc = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; ok && u < total; u += gridDim.x) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP2Args& a = I->p2;
        const int64_t lu = u - ustart[ki];
        const int per_split = a.n_stiles * a.n_chunks;
      const int split = (int)(lu / per_split), rem = (int)(lu % per_split);
      const int stile = rem / a.n_chunks, chunk = rem % a.n_chunks;
      const int jb0 = split * a.iblk_per_split;
      const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
      const int s = stile * 128 + row;
      const float cb = a.colb[s], cm = a.colm[s];
      const float a2 = a.a2, c2 = a.c2;
      // per-block float32 sums of the rounded weights, added to float64 totals once a
      // block (a float32 total over thousands of observations would drop the small
      // weights of a shift against its large running sum)
      float cacc = 0.f, zacc = 0.f;
      double cacc_d = 0.0, zacc_d = 0.0;
      for (int j = 0; j < nb; ++j) {
        const int64_t ib = (int64_t)(jb0 + j) * 128;
        const int b = sc & 1, pb = pz & 1;
        // (ybar, lse2) of the next 32-observation chunk, loaded one chunk ahead of its
        // use; lse2 = +inf past N gives weight 0
        float ny = a.ybar[ib + lane];
        float nl = (ib + lane < a.N) ? a.lse2[ib + lane] : INFINITY;
        // test hook: see pass 1
        const bool held = hook == 2 && blockIdx.x == 0 && sc == 0;
        ok = __all_sync(0xffffffffu, (!held || mbar_wait(never, 0, abort, wlim)) &&
                                         mbar_wait(&sfull[b], (sc >> 1) & 1, abort, wlim));
        if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&pempty[pb], ((pz >> 1) & 1) ^ 1, abort, wlim));
        if (!ok) break;
        tc_fence_after();
        uint8_t* prow = pbuf + pb * WB + row * 128;
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          __syncwarp();  // the warp is done with the previous chunk's terms
          wobs[lane] = make_float2(ny, nl);
          __syncwarp();
          if (c < 3) {
            const int64_t io = ib + (c + 1) * 32 + lane;
            ny = a.ybar[io];
            nl = (io < a.N) ? a.lse2[io] : INFINITY;
          }
          float v[32];
          tmem_ld32(lane_addr + (uint32_t)(b * 128 + c * 32), v);
          tmem_ld_wait();
          uint32_t packed[16], packed_lo[16];
#pragma unroll
          for (int e = 0; e < 32; e += 2) {
            float w2[2], wl2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float2 yl = wobs[e + h];
              const float ybi = yl.x;
              const float dd = ybi - cm;
              const float val = fmaf(v[e + h], a2, cb - yl.y) - c2 * dd * dd;
              const float w = exp2f(val) * W_SCALE;
              w2[h] = __half2float(__float2half_rn(w));
              wl2[h] = COMP ? __half2float(__float2half_rn(w - w2[h])) : 0.f;
              const float wsum = COMP ? w2[h] + wl2[h] : w2[h];
              cacc += wsum;
              zacc = fmaf(wsum, ybi, zacc);
            }
            const __half2 pr = __floats2half2_rn(w2[0], w2[1]);
            packed[e >> 1] = *reinterpret_cast<const uint32_t*>(&pr);
            if (COMP) {
              const __half2 pl = __floats2half2_rn(wl2[0], wl2[1]);
              packed_lo[e >> 1] = *reinterpret_cast<const uint32_t*>(&pl);
            }
          }
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const int col16 = c * 4 + g;           // 16-byte unit along the observations
            const int kb2 = col16 >> 3, cc = col16 & 7;
            uint4 val = make_uint4(packed[4 * g], packed[4 * g + 1], packed[4 * g + 2],
                                   packed[4 * g + 3]);
            *reinterpret_cast<uint4*>(prow + kb2 * 16384 + ((cc ^ (row & 7)) << 4)) = val;
            if (COMP)
              *reinterpret_cast<uint4*>(prow + SLOT + kb2 * 16384 + ((cc ^ (row & 7)) << 4)) =
                  make_uint4(packed_lo[4 * g], packed_lo[4 * g + 1], packed_lo[4 * g + 2],
                             packed_lo[4 * g + 3]);
          }
        }
        tc_fence_before();
        mbar_arrive(&sempty[b]);
        fence_proxy_async_smem();
        mbar_arrive(&pfull[pb]);
        cacc_d += (double)cacc;
        zacc_d += (double)zacc;
        cacc = zacc = 0.f;
        ++sc;
        ++pz;
      }
      if (!ok) break;
      ok = __all_sync(0xffffffffu, mbar_wait(zfull, uc & 1, abort, wlim));
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
        a.cp[(int64_t)split * a.Spad + s] = (float)(cacc_d * W_UNSCALE);
        a.zbp[(int64_t)split * a.Spad + s] = (float)(zacc_d * W_UNSCALE);
      }
      ++uc;
    }
    if (!ok) raise_timeout(abort, status);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// ------------------------------------------------------------------------------ pass 2,
// cluster forms.  A cluster of G CTAs shares one 128-shift tile and one range of
// observation blocks; CTA `rank` owns pixel chunk cg*G + rank of Z'.  In each round every
// CTA computes the logits of ITS OWN 128-observation block (no CTA recomputes another's),
// turns them into an fp16 weight tile, and the tile reaches the other CTAs through
// distributed shared memory; each CTA then accumulates Z'[s, its chunk] over the blocks
// of the round.  The weights of one (shift tile, observation block) are thus computed
// once per group of G chunks instead of once per pixel chunk.  Two forms:
// - ring form (G <= 4): every weight tile, the own one included, goes through the
//   7-slot operand ring.  Each CTA's producer reserves a slot for every tile of the
//   round and mails the slot index to the tile's owner; once all G reservations are in,
//   the owner writes its tile into its own slot and bulk-copies it into the others'.
// - interleaved form (G >= 5): the own tile is written to a staging slot, a sender warp
//   copies it to each peer as soon as that peer's reservation arrives (the CTAs no
//   longer wait for the slowest reservation of each tile), the peers' tiles land in a
//   weight ring of their own, and the Z' blocks of a round are interleaved with the
//   logit k-blocks of the next one.
// The deeper operand ring is worth more to small clusters (their logits dominate a
// round); the early per-peer hand-off to large ones (one weight tile per member per
// round).
// largest cluster; clusters above 8 CTAs (the portable limit) need the non-portable
// cluster-size attribute and fit only where a GPC has the free SMs
constexpr int P2C_MAX_G = 16;
constexpr int P2C_PORTABLE_G = 8;
constexpr int P2R_MAX_G = 4;  // ring form: clusters up to 4
// Mailbox rows, one per use of a tile.  In the ring form a producer can announce at most
// one use per ring slot it holds for a peer (the slot is freed only after the peer has
// read the announcement and sent its tile), so more rows than ring slots keep a row from
// being reused before it is read, whatever the cluster's chunk ownership.
constexpr int MBOX_DEPTH = 8;

// ---- ring form
constexpr int P2R_SLOTS = 7;
static_assert(MBOX_DEPTH > P2R_SLOTS, "a mailbox row could be reused before it is read");
// barriers: full, empty (ring), sfull, sempty, zfull, zempty, mfull (rows), drain, wready,
// never;
// then the mailbox, the TMEM address and the abort flag, in P2R_BOOK bytes after the ring
constexpr int P2R_BOOK = 512;
static_assert((2 * P2R_SLOTS + 2 + 2 + 1 + 1 + MBOX_DEPTH + 1 + 1 + 1) * 8 +
                      MBOX_DEPTH * P2R_MAX_G * 4 + 4 + 4 <= P2R_BOOK,
              "ring-form bookkeeping exceeds its P2R_BOOK bytes");

template <int NPROD>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_p2c_tc(const TcInst* __restrict__ insts, const int64_t* __restrict__ ustart, int n_inst,
             int G, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = (uint64_t*)(smem + P2R_SLOTS * SLOT);
  uint64_t* empty = full + P2R_SLOTS;
  uint64_t* sfull = empty + P2R_SLOTS;
  uint64_t* sempty = sfull + 2;
  uint64_t* zfull = sempty + 2;
  uint64_t* zempty = zfull + 1;
  uint64_t* mfull = zempty + 1;  // [MBOX_DEPTH]: one barrier per mailbox row
  uint64_t* drain = mfull + MBOX_DEPTH;
  uint64_t* wready = drain + 1;  // the 128 epilogue threads have written the weight tile
  uint64_t* never = wready + 1;  // nothing arrives on it (test hook)
  uint32_t* mbox = (uint32_t*)(never + 1);  // [MBOX_DEPTH][P2R_MAX_G] reserved slots
  uint32_t* tptr = mbox + MBOX_DEPTH * P2R_MAX_G;
  volatile int* abort = (volatile int*)(tptr + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t wlim = insts[0].p2.wait_ns;
  const int hook = insts[0].p2.hook;
  const uint32_t rank = cluster_rank();
  const int64_t cid = blockIdx.x / G, ncl = gridDim.x / G;

  if (threadIdx.x == 0) {
    for (int k = 0; k < P2R_SLOTS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sfull[b], 1);
      mbar_init(&sempty[b], 128);
    }
    mbar_init(zfull, 1);
    mbar_init(zempty, 128);
    for (int k = 0; k < MBOX_DEPTH; ++k) mbar_init(&mfull[k], G);
    mbar_init(drain, 1);
    mbar_init(wready, 128);
    mbar_init(never, 1);
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
  cluster_sync_all();  // every CTA's barriers exist before any peer arrives on them
  const uint32_t tbase = *tptr;
  const int64_t total = ustart[n_inst];

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0, sent[P2R_MAX_G] = {};
      bool ok = true;
      auto reserve = [&](bool expect_copy) -> int {
        const int st = it % P2R_SLOTS;
        if (!mbar_wait(&empty[st], ((it / P2R_SLOTS) & 1) ^ 1, abort, wlim)) {
          ok = false;
          return -1;
        }
        if (expect_copy) mbar_expect_tx(&full[st], 32768);
        return st;
      };
      for (int64_t u = cid; ok && u < total; u += ncl) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP2Args& a = I->p2;
        const int64_t lu = u - ustart[ki];
        const int ncg = (a.n_chunks + G - 1) / G;
        const int per_split = a.n_stiles * ncg;
        const int split = (int)(lu / per_split), rem = (int)(lu % per_split);
        const int stile = rem / ncg, chunk = (rem % ncg) * G + (int)rank;
        const bool cvalid = chunk < a.n_chunks;
        const int jb0 = split * a.iblk_per_split;
        const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
        const int rounds = (nb + G - 1) / G;
        // software-pipelined order: logits of round j, then the weights of round j - 1
        for (int j = 0; ok && j <= rounds; ++j) {
          const int r0 = j * G, nq = j < rounds ? min(G, nb - r0) : 0;
          if ((int)rank < nq) {  // logits of this CTA's own block
            const int ib = (jb0 + r0 + (int)rank) * 128;
            for (int kb = 0; ok && kb < a.nk; ++kb) {
              if (NPROD == 3) {
                int st = reserve(true);
                if (!ok) break;
                tma_load_2d(smem + st * SLOT, &I->tmA128, &full[st], kb * 64, stile * 128);
                tma_load_2d(smem + st * SLOT + 16384, &I->tmAl128, &full[st], kb * 64,
                            stile * 128);
                ++it;
                st = reserve(true);
                if (!ok) break;
                tma_load_2d(smem + st * SLOT, &I->tmY, &full[st], kb * 64, ib);
                tma_load_2d(smem + st * SLOT + 16384, &I->tmYl, &full[st], kb * 64, ib);
                ++it;
              } else {
                const int st = reserve(true);
                if (!ok) break;
                tma_load_2d(smem + st * SLOT, &I->tmA128, &full[st], kb * 64, stile * 128);
                tma_load_2d(smem + st * SLOT + 16384, &I->tmY, &full[st], kb * 64, ib);
                ++it;
              }
            }
          }
          // the slots of round j - 1: the weight tile of block rp + kq (filled by CTA kq)
          // is reserved one block ahead of the two Y'^T tiles it multiplies, i.e. in the
          // order W0 W1 T0 T0 W2 T1 T1 W3 T2 T2 T3 T3.  Every Y'^T tile then lies within
          // P2R_SLOTS - 1 places of its weight slot, so no fill waits for a slot that is
          // only freed by the products that need that fill, while the tiles of the other
          // CTAs can still be sent early.
          const int rp = (j - 1) * G, nqp = j >= 1 ? min(G, nb - rp) : 0;
          auto reserve_w = [&](int kq) {
            const int st = reserve(kq != (int)rank);
            if (!ok) return;
            // row sent % DEPTH of peer kq's mailbox, and that row's own barrier, so the
            // arrivals of different rounds can never complete each other's phases
            const uint32_t row = sent[kq] % MBOX_DEPTH;
            st_cluster_u32(mapa(smem_u32(mbox + row * P2R_MAX_G + rank), kq), (uint32_t)st);
            mbar_arrive_cluster(mapa(smem_u32(&mfull[row]), kq));
            ++sent[kq];
            ++it;
          };
          if (nqp > 0) reserve_w(0);
          for (int kq = 0; ok && kq < nqp; ++kq) {
            if (kq + 1 < nqp) reserve_w(kq + 1);
            const int ib = (jb0 + rp + kq) * 128;
            for (int h = 0; ok && cvalid && h < 2; ++h) {
              const int s2 = reserve(false);
              if (!ok) break;
              mbar_expect_tx(&full[s2], 32768);
              tma_load_2d(smem + s2 * SLOT, &I->tmYT, &full[s2], ib + h * 64, chunk * 256);
              ++it;
            }
          }
        }
      }
      if (!ok) raise_timeout(abort, status);
      {
        // the fills already issued land before the CTA exits, also when another role
        // gave up and stopped consuming them (in a normal run they are all consumed and
        // these waits return at once)
        const uint32_t lo = it > P2R_SLOTS ? it - P2R_SLOTS : 0;
        int zero = 0;
        for (uint32_t k = lo; k < it; ++k)
          mbar_wait(&full[k % P2R_SLOTS], (k / P2R_SLOTS) & 1, (volatile int*)&zero);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16_f32(128, 128);
      constexpr uint32_t idZ = idesc_f16_f32(128, 256);
      uint32_t it = 0, sc = 0, uc = 0;
      bool ok = true;
      auto wait_slot = [&]() -> int {
        const int st = it % P2R_SLOTS;
        if (!mbar_wait(&full[st], (it / P2R_SLOTS) & 1, abort, wlim)) {
          ok = false;
          return -1;
        }
        return st;
      };
      for (int64_t u = cid; ok && u < total; u += ncl) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP2Args& a = I->p2;
        const int64_t lu = u - ustart[ki];
        const int ncg = (a.n_chunks + G - 1) / G;
        const int per_split = a.n_stiles * ncg;
        const int rem = (int)(lu % per_split);
        const int chunk = (rem % ncg) * G + (int)rank;
        const bool cvalid = chunk < a.n_chunks;
        const int split = (int)(lu / per_split);
        const int jb0 = split * a.iblk_per_split;
        const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
        bool first_z = true;
        const int rounds = (nb + G - 1) / G;
        for (int j = 0; ok && j <= rounds; ++j) {
          const int r0 = j * G, nq = j < rounds ? min(G, nb - r0) : 0;
          if ((int)rank < nq) {
            const int b = sc & 1;
            if (!mbar_wait(&sempty[b], ((sc >> 1) & 1) ^ 1, abort, wlim)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tbase + (uint32_t)(b * 128);
            for (int kb = 0; ok && kb < a.nk; ++kb) {
              const int stA = wait_slot();
              if (!ok) break;
              uint8_t* sA = smem + stA * SLOT;
              uint8_t* sY = sA + 16384;
              int stY = stA;
              if (NPROD == 3) {
                ++it;
                stY = wait_slot();
                if (!ok) break;
                sY = smem + stY * SLOT;
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
          const int nqp = j >= 1 ? min(G, nb - (j - 1) * G) : 0;
          // same slot order as the producer: W0 W1 T0 T0 W2 T1 T1 W3 T2 T2 T3 T3
          int stPs[P2R_MAX_G] = {};
          if (nqp > 0) {
            stPs[0] = wait_slot();
            ++it;
          }
          for (int kq = 0; ok && kq < nqp; ++kq) {
            if (kq + 1 < nqp) {
              stPs[kq + 1] = wait_slot();
              ++it;
              if (!ok) break;
            }
            const int stP = stPs[kq];
            if (cvalid) {
              if (first_z && !mbar_wait(zempty, (uc & 1) ^ 1, abort, wlim)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t dZ = tbase + 256u;
              for (int h = 0; ok && h < 2; ++h) {
                const int stT = wait_slot();
                if (!ok) break;
                tc_fence_after();
                const uint64_t dP = desc_sw128(smem + stP * SLOT + h * 16384);
                const uint64_t dT = desc_sw128(smem + stT * SLOT);
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4)
                  mma_bf16(dZ, desc_advance(dP, k4), desc_advance(dT, k4), idZ,
                           (!first_z || h > 0 || k4 > 0) ? 1u : 0u);
                mma_commit(&empty[stT]);
                ++it;
              }
              first_z = false;
            }
            mma_commit(&empty[stP]);
          }
        }
        if (!ok) break;
        if (cvalid) {
          mma_commit(zfull);
          ++uc;
        }
      }
      if (!ok) raise_timeout(abort, status);
      // every issued MMA completes before TMEM is released, also when another role
      // gave up and left accumulators unread
      mma_commit(drain);
      int zero = 0;
      mbar_wait(drain, 0, (volatile int*)&zero);
    }
  } else {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
    float2* wobs = (float2*)(smem + P2R_SLOTS * SLOT + P2R_BOOK) + q * 32;  // warp's staging
    uint32_t sc = 0, mr = 0, uc = 0;
    bool ok = true;
    for (int64_t u = cid; ok && u < total; u += ncl) {
      const int ki = find_inst(ustart, n_inst, u);
      const TcInst* I = insts + ki;
      const TcP2Args& a = I->p2;
      const int64_t lu = u - ustart[ki];
      const int ncg = (a.n_chunks + G - 1) / G;
      const int per_split = a.n_stiles * ncg;
      const int split = (int)(lu / per_split), rem = (int)(lu % per_split);
      const int stile = rem / ncg, cgrp = rem % ncg;
      const int chunk = cgrp * G + (int)rank;
      const bool cvalid = chunk < a.n_chunks;
      const int jb0 = split * a.iblk_per_split;
      const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
      const int s = stile * 128 + row;
      const float cb = a.colb[s], cm = a.colm[s];
      const float a2 = a.a2, c2 = a.c2;
      // per-block float32 sums of the rounded weights, added to float64 totals once a
      // block (a float32 total over thousands of observations would drop the small
      // weights of a shift against its large running sum)
      float cacc = 0.f, zacc = 0.f;
      double cacc_d = 0.0, zacc_d = 0.0;
      for (int r0 = 0; ok && r0 < nb; r0 += G) {
        const int nq = min(G, nb - r0);
        if ((int)rank >= nq) continue;
        const int64_t ib = (int64_t)(jb0 + r0 + (int)rank) * 128;
        const int b = sc & 1;
        // (ybar, lse2) of the next 32-observation chunk, loaded one chunk ahead of its
        // use; lse2 = +inf past N gives weight 0
        float ny = a.ybar[ib + lane];
        float nl = (ib + lane < a.N) ? a.lse2[ib + lane] : INFINITY;
        // test hook: see pass 1 (the first cluster's rank 0 never builds its first tile,
        // so its peers' waits for that tile run out as well)
        const bool held = hook == 2 && blockIdx.x == 0 && sc == 0;
        ok = __all_sync(0xffffffffu, (!held || mbar_wait(never, 0, abort, wlim)) &&
                                         mbar_wait(&sfull[b], (sc >> 1) & 1, abort, wlim));
        if (!ok) break;
        tc_fence_after();
        // the weights of this row, as fp16 pairs in the order of the tile's columns; they
        // are computed as soon as the logits are in TMEM, before the slot they go to has
        // been granted, so that the logit buffer is released early
        uint32_t packed[64];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          __syncwarp();  // the warp is done with the previous chunk's terms
          wobs[lane] = make_float2(ny, nl);
          __syncwarp();
          if (c < 3) {
            const int64_t io = ib + (c + 1) * 32 + lane;
            ny = a.ybar[io];
            nl = (io < a.N) ? a.lse2[io] : INFINITY;
          }
          float v[32];
          tmem_ld32(lane_addr + (uint32_t)(b * 128 + c * 32), v);
          tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < 32; e += 2) {
            float w2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float2 yl = wobs[e + h];
              const float ybi = yl.x;
              const float dd = ybi - cm;
              const float val = fmaf(v[e + h], a2, cb - yl.y) - c2 * dd * dd;
              const float w = exp2f(val) * W_SCALE;
              w2[h] = __half2float(__float2half_rn(w));
              cacc += w2[h];
              zacc = fmaf(w2[h], ybi, zacc);
            }
            const __half2 pr = __floats2half2_rn(w2[0], w2[1]);
            packed[c * 16 + (e >> 1)] = *reinterpret_cast<const uint32_t*>(&pr);
          }
        }
        tc_fence_before();
        mbar_arrive(&sempty[b]);  // the logits are no longer needed
        ok = __all_sync(0xffffffffu,
                        mbar_wait_cluster(&mfull[mr % MBOX_DEPTH], (mr / MBOX_DEPTH) & 1, abort, wlim));
        if (!ok) break;
        const uint32_t* mrow = mbox + (mr % MBOX_DEPTH) * P2R_MAX_G;
        const int own = (int)mrow[rank];
        uint8_t* prow = smem + own * SLOT + row * 128;
#pragma unroll
        for (int col16 = 0; col16 < 16; ++col16) {  // 16-byte units along the observations
          const int kb2 = col16 >> 3, cc = col16 & 7;
          *reinterpret_cast<uint4*>(prow + kb2 * 16384 + ((cc ^ (row & 7)) << 4)) =
              make_uint4(packed[4 * col16], packed[4 * col16 + 1], packed[4 * col16 + 2],
                         packed[4 * col16 + 3]);
        }
        fence_proxy_async_smem();
        mbar_arrive(wready);
        bool sent_ok = true;
        if (row == 0) {  // all 128 rows written: send the tile to the other CTAs
          sent_ok = mbar_wait(wready, mr & 1, abort, wlim);
          if (sent_ok) {
            const uint8_t* src = smem + own * SLOT;
            for (int j = 0; j < G; ++j) {
              if (j == (int)rank) continue;
              const int dst = (int)mrow[j];
              bulk_copy_to_peer(mapa(smem_u32(smem + dst * SLOT), j), src, 32768,
                                mapa(smem_u32(&full[dst]), j));
            }
            bulk_commit();
            bulk_wait_read0();
            mbar_arrive(&full[own]);
          }
        }
        ok = __all_sync(0xffffffffu, sent_ok);
        if (!ok) break;
        cacc_d += (double)cacc;
        zacc_d += (double)zacc;
        cacc = zacc = 0.f;
        ++sc;
        ++mr;
      }
      if (!ok) break;
      if (cvalid) {
        ok = __all_sync(0xffffffffu, mbar_wait(zfull, uc & 1, abort, wlim));
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
        ++uc;
      }
      if (cgrp == 0) {
        const int64_t part = (int64_t)split * G + rank;
        a.cp[part * a.Spad + s] = (float)(cacc_d * W_UNSCALE);
        a.zbp[part * a.Spad + s] = (float)(zacc_d * W_UNSCALE);
      }
    }
    if (!ok) raise_timeout(abort, status);
    if (row == 0) bulk_wait0();  // the tiles sent to the peers have landed
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
  cluster_sync_all();  // no CTA leaves while a peer may still copy into it
}

// ring + bookkeeping (30 mbarriers, 8 x 4 mailbox, TMEM address, abort flag: 376 of the
// 512 bytes) +
// per-warp staging of one 32-observation chunk's (ybar, lse2) (4 x 256 bytes)
constexpr size_t P2R_SMEM = 1024 + P2R_SLOTS * SLOT + P2R_BOOK + 1024;
static_assert(P2R_SMEM <= 232448, "exceeds the shared memory of one CTA");

// ---- pair form
// The CTAs of a cluster form pairs (cluster ranks 2p, 2p + 1) that issue 2-CTA tcgen05
// MMAs (cta_group::2): the even CTA of a pair issues every MMA of the pair; each CTA
// holds its own rows of the A operand and half of the columns of the B operand, and
// its own rows of the accumulator in its Tensor Memory.  A pair works on two 128-shift
// tiles at once, one per CTA:
// - the logits of a 128-observation block are a 256 x 128 product per k-step, each CTA
//   loading its own templates and 64 of the block's observations;
// - Z' of a 256-pixel chunk is a 256 x 256 product per k-step, each CTA loading 128 of
//   the chunk's pixels of Y'^T;
// so each SM reads a quarter fewer operand bytes from shared memory per flop than with
// one CTA's 128 x 128 and 128 x 256 products.  (Measured on GB300 this did not make the
// tensor pipe busier per SM, and clusters of 8 CTAs fit on fewer SMs than clusters of
// 4: the form is slower than the ring form and is used only on request,
// SRMRA_FLAG_P2_PAIR.)  The G pairs of a cluster share their weight tiles as in the ring
// form, among the CTAs of the same parity (the same shift tile): every weight tile and
// Y'^T tile goes through the 7-slot ring, the slots of a round's weight tiles are
// reserved first (each tile's Y'^T fill lies nqp <= 4 places after its slot, so no fill
// waits for a slot that only its own products release), and the owner sends its tile
// once all G reservations are in.  Both CTAs of a pair run the same sequence of fills,
// so a fill has the same slot in both.  The odd CTA's TMA loads complete on the even
// CTA's barrier (cta_group::2 loads), which expects the bytes of both; a weight tile
// copied into a CTA completes on that CTA's barrier, and the odd CTA's MMA warp relays
// each of its weight fills to the even CTA (pfull), whose MMA thread waits on both
// before it reads the slot of both CTAs.  Each MMA completion is committed to the
// barriers of both CTAs, and the odd CTA's epilogue warps report a drained accumulator
// to the even CTA (one arrival per warp).
constexpr int P2P_MAX_G = 4;  // pairs per cluster (clusters of up to 8 CTAs)
constexpr int P2_KEY_PAIR = 32;  // pass-2 launch keys above it: the pair form
// barriers: full, pfull, empty (ring), sfull, sempty, zfull, zempty, mfull (rows), drain,
// wready, never; then the mailbox, the TMEM address and the abort flag
static_assert((3 * P2R_SLOTS + 2 + 2 + 1 + 1 + MBOX_DEPTH + 1 + 1 + 1) * 8 +
                      MBOX_DEPTH * P2P_MAX_G * 4 + 4 + 4 <= P2R_BOOK,
              "pair-form bookkeeping exceeds its P2R_BOOK bytes");

template <int NPROD>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_p2p_tc(const TcInst* __restrict__ insts, const int64_t* __restrict__ ustart, int n_inst,
             int G, int* status) {
  static_assert(NPROD == 3, "the pair form is built for split-bf16 logits");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = (uint64_t*)(smem + P2R_SLOTS * SLOT);
  uint64_t* pfull = full + P2R_SLOTS;  // even CTA: the odd CTA's fill of the slot is in
  uint64_t* empty = pfull + P2R_SLOTS;
  uint64_t* sfull = empty + P2R_SLOTS;
  uint64_t* sempty = sfull + 2;
  uint64_t* zfull = sempty + 2;
  uint64_t* zempty = zfull + 1;
  uint64_t* mfull = zempty + 1;  // [MBOX_DEPTH]: one barrier per mailbox row
  uint64_t* drain = mfull + MBOX_DEPTH;
  uint64_t* wready = drain + 1;  // the 128 epilogue threads have written the weight tile
  uint64_t* never = wready + 1;  // nothing arrives on it (test hook)
  uint32_t* mbox = (uint32_t*)(never + 1);  // [MBOX_DEPTH][P2P_MAX_G] reserved slots
  uint32_t* tptr = mbox + MBOX_DEPTH * P2P_MAX_G;
  volatile int* abort = (volatile int*)(tptr + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t wlim = insts[0].p2.wait_ns;
  const int hook = insts[0].p2.hook;
  const uint32_t rank = cluster_rank();
  const uint32_t peer = rank ^ 1u;  // the other CTA of the pair
  const int h = (int)(rank & 1u), pr = (int)(rank >> 1);
  const int64_t cid = blockIdx.x / (2 * G), ncl = gridDim.x / (2 * G);

  if (threadIdx.x == 0) {
    for (int k = 0; k < P2R_SLOTS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&pfull[k], 1);
      mbar_init(&empty[k], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sfull[b], 1);
      mbar_init(&sempty[b], 128 + 4);  // even CTA: its 128 threads + the odd CTA's 4 warps
    }
    mbar_init(zfull, 1);
    mbar_init(zempty, 128 + 4);
    for (int k = 0; k < MBOX_DEPTH; ++k) mbar_init(&mfull[k], G);
    mbar_init(drain, 1);
    mbar_init(wready, 128);
    mbar_init(never, 1);
    *abort = 0;
    fence_mbar_init();
  }
  // every CTA's barriers exist before any peer arrives on them, and both CTAs of a pair
  // are running before they allocate Tensor Memory together
  cluster_sync_all();
  if (warp == 1) {
    tmem_alloc_pair(tptr, 512);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  cluster_sync_all();  // the pair's allocation is complete in both CTAs
  const uint32_t tbase = *tptr;
  const int64_t total = ustart[n_inst];

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0, sent[P2P_MAX_G] = {};
      bool wfill[P2R_SLOTS] = {};  // the slot's last fill is a weight tile (lands locally)
      uint32_t wcnt[P2R_SLOTS] = {};  // weight-tile fills of each slot so far
      bool ok = true;
      auto reserve = [&](uint32_t tx) -> int {
        const int st = it % P2R_SLOTS;
        if (!mbar_wait(&empty[st], ((it / P2R_SLOTS) & 1) ^ 1, abort, wlim)) {
          ok = false;
          return -1;
        }
        if (tx) mbar_expect_tx(&full[st], tx);
        return st;
      };
      // a TMA fill of the pair: the even CTA expects the bytes of both CTAs on its
      // barrier, the odd CTA's loads complete there too
      auto reserve_tma = [&](uint32_t bytes) -> int {
        const int st = reserve(h == 0 ? 2u * bytes : 0u);
        if (st >= 0) wfill[st] = false;
        return st;
      };
      const uint32_t lead_full = mapa(smem_u32(full), peer);  // odd CTA: the even CTA's full[0]
      auto load = [&](int st, int off, const CUtensorMap* map, int c0, int c1) {
        if (h == 0)
          tma_load_2d(smem + st * SLOT + off, map, &full[st], c0, c1);
        else
          tma_load_2d_pair(smem + st * SLOT + off, map, lead_full + 8u * (uint32_t)st, c0, c1);
      };
      for (int64_t u = cid; ok && u < total; u += ncl) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP2Args& a = I->p2;
        const int64_t lu = u - ustart[ki];
        const int ncg = (a.n_chunks + G - 1) / G;
        const int per_split = (a.n_stiles / 2) * ncg;
        const int split = (int)(lu / per_split), rem = (int)(lu % per_split);
        const int stile = (rem / ncg) * 2 + h, chunk = (rem % ncg) * G + pr;
        const bool cvalid = chunk < a.n_chunks;
        const int jb0 = split * a.iblk_per_split;
        const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
        const int rounds = (nb + G - 1) / G;
        for (int j = 0; ok && j <= rounds; ++j) {
          const int r0 = j * G, nq = j < rounds ? min(G, nb - r0) : 0;
          if (pr < nq) {  // logits of the pair's block: this CTA's 64 observations of it
            const int ib = (jb0 + r0 + pr) * 128 + h * 64;
            for (int kb = 0; ok && kb < a.nk; kb += 2) {
              const int nkk = min(2, a.nk - kb);
              for (int t = 0; ok && t < nkk; ++t) {  // templates of k-blocks kb, kb + 1
                const int st = reserve_tma(32768);
                if (!ok) break;
                load(st, 0, &I->tmA128, (kb + t) * 64, stile * 128);
                load(st, 16384, &I->tmAl128, (kb + t) * 64, stile * 128);
                ++it;
              }
              if (!ok) break;
              const int st = reserve_tma(16384u * (uint32_t)nkk);  // observations: hi, lo
              if (!ok) break;
              for (int t = 0; t < nkk; ++t) {
                load(st, t * 16384, &I->tmY64, (kb + t) * 64, ib);
                load(st, t * 16384 + 8192, &I->tmYl64, (kb + t) * 64, ib);
              }
              ++it;
            }
          }
          // round j - 1: a slot for the weight tile of every block, announced to the
          // tile's owner (the CTA of the same parity in the block's pair), then this
          // CTA's 128 pixels of the Y'^T tile of every block
          const int rp = (j - 1) * G, nqp = j >= 1 ? min(G, nb - rp) : 0;
          for (int i = 0; ok && i < nqp; ++i) {
            const int st = reserve(i != pr ? 32768u : 0u);
            if (!ok) break;
            wfill[st] = true;
            ++wcnt[st];
            const uint32_t owner = 2u * (uint32_t)i + (uint32_t)h;
            // row sent % DEPTH of the owner's mailbox, and that row's own barrier
            const uint32_t row = sent[i] % MBOX_DEPTH;
            st_cluster_u32(mapa(smem_u32(mbox + row * P2P_MAX_G + pr), owner), (uint32_t)st);
            mbar_arrive_cluster(mapa(smem_u32(&mfull[row]), owner));
            ++sent[i];
            ++it;
          }
          for (int i = 0; ok && cvalid && i < nqp; ++i) {
            const int st = reserve_tma(32768);
            if (!ok) break;
            const int ibq = (jb0 + rp + i) * 128;
            for (int hh = 0; hh < 2; ++hh)
              load(st, hh * 16384, &I->tmYT128, ibq + hh * 64, chunk * 256 + h * 128);
            ++it;
          }
        }
      }
      if (!ok) raise_timeout(abort, status);
      {
        // the fills already issued land before the CTA exits, also when another role
        // gave up and stopped consuming them.  The odd CTA's TMA fills complete on the
        // even CTA's barriers, whose producer waits for them (the final cluster barrier
        // keeps the odd CTA until then); the odd CTA's own barriers see only its weight
        // fills, so their phases count those.
        const uint32_t lo = it > P2R_SLOTS ? it - P2R_SLOTS : 0;
        int zero = 0;
        for (uint32_t k = lo; k < it; ++k) {
          const int st = k % P2R_SLOTS;
          if (h == 0)
            mbar_wait(&full[st], (k / P2R_SLOTS) & 1, (volatile int*)&zero);
          else if (wfill[st])
            mbar_wait(&full[st], (wcnt[st] - 1) & 1, (volatile int*)&zero);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // even CTA: the pair's MMAs; odd CTA: relays its completed weight-tile fills to the
      // even CTA, in the order in which the even CTA's MMA thread waits for them
      const bool issuer = h == 0;
      constexpr uint32_t idS = idesc_bf16_f32(256, 128);
      constexpr uint32_t idZ = idesc_f16_f32(256, 256);
      uint32_t it = 0, sc = 0, uc = 0;
      bool ok = true;
      // TMA fill k has landed in both CTAs (issuer; the odd CTA skips it)
      auto take = [&](uint32_t k) -> int {
        const int st = k % P2R_SLOTS;
        if (issuer && !mbar_wait_cluster(&full[st], (k / P2R_SLOTS) & 1, abort, wlim)) {
          ok = false;
          return -1;
        }
        return st;
      };
      // weight-tile fill k has landed in both CTAs (issuer) / relay it (odd CTA).  The
      // odd CTA's barrier of the slot and the even CTA's pfull of it see only weight
      // fills: their phases count those (wc), the even CTA's full counts every fill.
      uint32_t wc[P2R_SLOTS] = {};
      auto take_w = [&](uint32_t k) -> int {
        const int st = k % P2R_SLOTS;
        const uint32_t wpar = wc[st] & 1;
        ++wc[st];
        if (!mbar_wait(&full[st], issuer ? (k / P2R_SLOTS) & 1 : wpar, abort, wlim)) {
          ok = false;
          return -1;
        }
        if (issuer) {
          if (!mbar_wait_cluster(&pfull[st], wpar, abort, wlim)) {
            ok = false;
            return -1;
          }
        } else {
          mbar_arrive_cluster(mapa(smem_u32(&pfull[st]), peer));
        }
        return st;
      };
      // the products that read a slot are done: free it in both CTAs
      auto release = [&](uint64_t* bar) {
        mma_commit_pair(smem_u32(bar));
        mma_commit_pair(mapa(smem_u32(bar), peer));
      };
      for (int64_t u = cid; ok && u < total; u += ncl) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP2Args& a = I->p2;
        const int64_t lu = u - ustart[ki];
        const int ncg = (a.n_chunks + G - 1) / G;
        const int per_split = (a.n_stiles / 2) * ncg;
        const int rem = (int)(lu % per_split);
        const int chunk = (rem % ncg) * G + pr;
        const bool cvalid = chunk < a.n_chunks;
        const int split = (int)(lu / per_split);
        const int jb0 = split * a.iblk_per_split;
        const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
        bool first_z = true;
        const int rounds = (nb + G - 1) / G;
        for (int j = 0; ok && j <= rounds; ++j) {
          const int r0 = j * G, nq = j < rounds ? min(G, nb - r0) : 0;
          if (pr < nq) {
            const int b = sc & 1;
            if (issuer && !mbar_wait_cluster(&sempty[b], ((sc >> 1) & 1) ^ 1, abort, wlim)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tbase + (uint32_t)(b * 128);
            for (int kb = 0; ok && kb < a.nk; kb += 2) {
              const int nkk = min(2, a.nk - kb);
              int stA[2] = {0, 0};
              for (int t = 0; ok && t < nkk; ++t) stA[t] = take(it++);
              if (!ok) break;
              const int stY = take(it++);
              if (!ok || !issuer) continue;
              tc_fence_after();
              for (int t = 0; t < nkk; ++t) {
                const uint8_t* sA = smem + stA[t] * SLOT;
                const uint8_t* sY = smem + stY * SLOT + t * 16384;
                const uint64_t dA = desc_sw128(sA), dAl = desc_sw128(sA + 16384);
                const uint64_t dY = desc_sw128(sY), dYl = desc_sw128(sY + 8192);
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                  mma_f16_pair(d, desc_advance(dA, k4), desc_advance(dY, k4), idS,
                               (kb + t > 0 || k4 > 0) ? 1u : 0u);
                  mma_f16_pair(d, desc_advance(dA, k4), desc_advance(dYl, k4), idS, 1u);
                  mma_f16_pair(d, desc_advance(dAl, k4), desc_advance(dY, k4), idS, 1u);
                }
                release(&empty[stA[t]]);
              }
              release(&empty[stY]);
            }
            if (!ok) break;
            if (issuer) release(&sfull[b]);
            ++sc;
          }
          // Z' of round j - 1: weight tile i (slot it + i) times this pair's Y'^T tile i
          // (slot it + nqp + i)
          const int nqp = j >= 1 ? min(G, nb - (j - 1) * G) : 0;
          const uint32_t base = it;
          it += (uint32_t)(cvalid ? 2 * nqp : nqp);
          for (int i = 0; ok && i < nqp; ++i) {
            const int stW = take_w(base + (uint32_t)i);
            if (!ok) break;
            if (cvalid) {
              if (issuer && first_z && !mbar_wait_cluster(zempty, (uc & 1) ^ 1, abort, wlim)) {
                ok = false;
                break;
              }
              const int stT = take(base + (uint32_t)(nqp + i));
              if (!ok) break;
              if (issuer) {
                tc_fence_after();
                const uint32_t dZ = tbase + 256u;
                for (int hh = 0; hh < 2; ++hh) {
                  const uint64_t dP = desc_sw128(smem + stW * SLOT + hh * 16384);
                  const uint64_t dT = desc_sw128(smem + stT * SLOT + hh * 16384);
#pragma unroll
                  for (int k4 = 0; k4 < 4; ++k4)
                    mma_f16_pair(dZ, desc_advance(dP, k4), desc_advance(dT, k4), idZ,
                                 (!first_z || hh > 0 || k4 > 0) ? 1u : 0u);
                }
                release(&empty[stT]);
              }
              first_z = false;
            }
            if (issuer) release(&empty[stW]);
          }
        }
        if (!ok) break;
        if (cvalid) {
          if (issuer) release(zfull);
          ++uc;
        }
      }
      if (!ok) raise_timeout(abort, status);
      if (issuer) {
        // every issued MMA completes before the Tensor Memory is released, also when
        // another role gave up and left accumulators unread
        mma_commit_pair(smem_u32(drain));
        int zero = 0;
        mbar_wait(drain, 0, (volatile int*)&zero);
      }
    }
  } else {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
    float2* wobs = (float2*)(smem + P2R_SLOTS * SLOT + P2R_BOOK) + q * 32;  // warp's staging
    uint32_t sc = 0, mr = 0, uc = 0;
    bool ok = true;
    // an accumulator of the pair has been read: the even CTA counts its own 128 threads,
    // the odd CTA reports once per warp
    auto drained = [&](uint64_t* bar) {
      tc_fence_before();
      if (h == 0) {
        mbar_arrive(bar);
      } else {
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(mapa(smem_u32(bar), peer));
      }
    };
    for (int64_t u = cid; ok && u < total; u += ncl) {
      const int ki = find_inst(ustart, n_inst, u);
      const TcInst* I = insts + ki;
      const TcP2Args& a = I->p2;
      const int64_t lu = u - ustart[ki];
      const int ncg = (a.n_chunks + G - 1) / G;
      const int per_split = (a.n_stiles / 2) * ncg;
      const int split = (int)(lu / per_split), rem = (int)(lu % per_split);
      const int stile = (rem / ncg) * 2 + h, cgrp = rem % ncg;
      const int chunk = cgrp * G + pr;
      const bool cvalid = chunk < a.n_chunks;
      const int jb0 = split * a.iblk_per_split;
      const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
      const int s = stile * 128 + row;
      const float cb = a.colb[s], cm = a.colm[s];
      const float a2 = a.a2, c2 = a.c2;
      // per-block float32 sums of the rounded weights, added to float64 totals once a
      // block
      float cacc = 0.f, zacc = 0.f;
      double cacc_d = 0.0, zacc_d = 0.0;
      for (int r0 = 0; ok && r0 < nb; r0 += G) {
        const int nq = min(G, nb - r0);
        if (pr >= nq) continue;
        const int64_t ib = (int64_t)(jb0 + r0 + pr) * 128;
        const int b = sc & 1;
        // (ybar, lse2) of the next 32-observation chunk, loaded one chunk ahead of its
        // use; lse2 = +inf past N gives weight 0
        float ny = a.ybar[ib + lane];
        float nl = (ib + lane < a.N) ? a.lse2[ib + lane] : INFINITY;
        // test hook: the first cluster's rank 0 never builds its first tile, so the waits
        // of the CTAs of its parity for that tile run out as well
        const bool held = hook == 2 && blockIdx.x == 0 && sc == 0;
        ok = __all_sync(0xffffffffu,
                        (!held || mbar_wait(never, 0, abort, wlim)) &&
                            mbar_wait_cluster(&sfull[b], (sc >> 1) & 1, abort, wlim));
        if (!ok) break;
        tc_fence_after();
        // the weights of this row, as fp16 pairs in the order of the tile's columns
        uint32_t packed[64];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          __syncwarp();  // the warp is done with the previous chunk's terms
          wobs[lane] = make_float2(ny, nl);
          __syncwarp();
          if (c < 3) {
            const int64_t io = ib + (c + 1) * 32 + lane;
            ny = a.ybar[io];
            nl = (io < a.N) ? a.lse2[io] : INFINITY;
          }
          float v[32];
          tmem_ld32(lane_addr + (uint32_t)(b * 128 + c * 32), v);
          tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < 32; e += 2) {
            float w2[2];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const float2 yl = wobs[e + hh];
              const float ybi = yl.x;
              const float dd = ybi - cm;
              const float val = fmaf(v[e + hh], a2, cb - yl.y) - c2 * dd * dd;
              const float w = exp2f(val) * W_SCALE;
              w2[hh] = __half2float(__float2half_rn(w));
              cacc += w2[hh];
              zacc = fmaf(w2[hh], ybi, zacc);
            }
            const __half2 pv = __floats2half2_rn(w2[0], w2[1]);
            packed[c * 16 + (e >> 1)] = *reinterpret_cast<const uint32_t*>(&pv);
          }
        }
        drained(&sempty[b]);  // the logits are no longer needed
        ok = __all_sync(0xffffffffu, mbar_wait_cluster(&mfull[mr % MBOX_DEPTH],
                                                       (mr / MBOX_DEPTH) & 1, abort, wlim));
        if (!ok) break;
        const uint32_t* mrow = mbox + (mr % MBOX_DEPTH) * P2P_MAX_G;
        const int own = (int)mrow[pr];
        uint8_t* prow = smem + own * SLOT + row * 128;
#pragma unroll
        for (int col16 = 0; col16 < 16; ++col16) {  // 16-byte units along the observations
          const int kb2 = col16 >> 3, cc = col16 & 7;
          *reinterpret_cast<uint4*>(prow + kb2 * 16384 + ((cc ^ (row & 7)) << 4)) =
              make_uint4(packed[4 * col16], packed[4 * col16 + 1], packed[4 * col16 + 2],
                         packed[4 * col16 + 3]);
        }
        fence_proxy_async_smem();
        mbar_arrive(wready);
        bool sent_ok = true;
        if (row == 0) {  // all 128 rows written: send the tile to the CTAs of this parity
          sent_ok = mbar_wait(wready, mr & 1, abort, wlim);
          if (sent_ok) {
            const uint8_t* src = smem + own * SLOT;
            for (int jq = 0; jq < G; ++jq) {
              if (jq == pr) continue;
              const uint32_t dcta = 2u * (uint32_t)jq + (uint32_t)h;
              const int dst = (int)mrow[jq];
              bulk_copy_to_peer(mapa(smem_u32(smem + dst * SLOT), dcta), src, 32768,
                                mapa(smem_u32(&full[dst]), dcta));
            }
            bulk_commit();
            bulk_wait_read0();
            mbar_arrive(&full[own]);
          }
        }
        ok = __all_sync(0xffffffffu, sent_ok);
        if (!ok) break;
        cacc_d += (double)cacc;
        zacc_d += (double)zacc;
        cacc = zacc = 0.f;
        ++sc;
        ++mr;
      }
      if (!ok) break;
      if (cvalid) {
        ok = __all_sync(0xffffffffu, mbar_wait_cluster(zfull, uc & 1, abort, wlim));
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
        drained(zempty);
        ++uc;
      }
      if (cgrp == 0) {
        const int64_t part = (int64_t)split * G + pr;
        a.cp[part * a.Spad + s] = (float)(cacc_d * W_UNSCALE);
        a.zbp[part * a.Spad + s] = (float)(zacc_d * W_UNSCALE);
      }
    }
    if (!ok) raise_timeout(abort, status);
    if (row == 0) bulk_wait0();  // the tiles sent to the peers have landed
  }
  __syncthreads();
  // neither CTA of a pair releases the pair's Tensor Memory before the even CTA's MMAs
  // are done and both CTAs' epilogues have left it
  cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tbase, 512);
  }
  cluster_sync_all();  // no CTA leaves while a peer may still copy into it
}

constexpr size_t P2P_SMEM = P2R_SMEM;

// ---- interleaved form
constexpr uint32_t MBOX_TAG_MASK = 0x0FFFFFFFu;  // entry = tag << 4 | slot, tag = use + 1

// The blocks of a round in this CTA's order: its own block first (rank < nq), then the
// next ranks cyclically; a CTA without a block of the round starts at rank mod nq.
__device__ __forceinline__ int p2c_block(int rank, int nq, int i) {
  return (rank % nq + i) % nq;
}

// Each CTA's own weight tile is written to a staging slot, from which its MMAs read it
// first in the round and a sender warp bulk-copies it to each peer with a pixel chunk as
// soon as that peer's slot is announced (a tagged entry in the sender's mailbox).  The
// peers' tiles land in a 2-slot weight ring of their own, whose slots a weight-producer
// thread announces as soon as they are free, at most about a round ahead of the main
// producer.  The Z' blocks of round j - 1 are interleaved with the logit k-blocks of
// round j, so that a tile is needed several k-blocks after its slot was announced.  The
// main ring (logit operands and Y'^T tiles) has 4 slots.
constexpr int P2I_SLOTS = 4;
constexpr int P2I_WSLOTS = 2;
constexpr int P2I_THREADS = 256;  // producer, MMA, 4 epilogue warps, sender, weight producer
// barriers: full, empty (main ring), wrfull, wrempty (weight ring), sfull, sempty, zfull,
// zempty, wfull, wfree, cdone, drain, never; then the mailbox, the TMEM address, the abort flag
// and the round counter, in P2I_BOOK bytes
constexpr int P2I_BOOK = 768;
static_assert((2 * P2I_SLOTS + 2 * P2I_WSLOTS + 2 + 2 + 1 + 1 + 1 + 1 + 1 + 1 + 1) * 8 +
                      MBOX_DEPTH * P2C_MAX_G * 4 + 4 + 4 + 4 <= P2I_BOOK,
              "interleaved-form bookkeeping exceeds its P2I_BOOK bytes");
static_assert(MBOX_DEPTH >= 4, "the weight producer's lead needs 4 mailbox rows");

// k-block of round j after which Z' block i of round j - 1 is issued (nqp blocks spread
// over the nk k-blocks; all after the last one when there are too few k-blocks)
__device__ __forceinline__ int p2i_zpos(int i, int nqp, int nk) {
  return nk >= nqp + 1 ? ((i + 1) * nk) / (nqp + 1) - 1 : nk - 1;
}

template <int NPROD>
__global__ void __launch_bounds__(P2I_THREADS, 1)
    k_p2i_tc(const TcInst* __restrict__ insts, const int64_t* __restrict__ ustart, int n_inst,
             int G, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* wring = smem + P2I_SLOTS * SLOT;     // the peers' weight tiles
  uint8_t* stage = wring + P2I_WSLOTS * SLOT;   // this CTA's weight tile
  uint64_t* full = (uint64_t*)(stage + SLOT);
  uint64_t* empty = full + P2I_SLOTS;
  uint64_t* wrfull = empty + P2I_SLOTS;     // weight ring: a peer's tile has landed
  uint64_t* wrempty = wrfull + P2I_WSLOTS;  // weight ring: its products are done
  uint64_t* sfull = wrempty + P2I_WSLOTS;
  uint64_t* sempty = sfull + 2;
  uint64_t* zfull = sempty + 2;
  uint64_t* zempty = zfull + 1;
  uint64_t* wfull = zempty + 1;  // the 128 epilogue threads have written the staged tile
  uint64_t* wfree = wfull + 1;   // the MMAs that read the staged tile have completed
  uint64_t* cdone = wfree + 1;   // the copies of the staged tile have read it
  uint64_t* drain = cdone + 1;
  uint64_t* never = drain + 1;  // nothing arrives on it (test hook)
  uint32_t* mbox = (uint32_t*)(never + 1);  // [MBOX_DEPTH][P2C_MAX_G]
  uint32_t* tptr = mbox + MBOX_DEPTH * P2C_MAX_G;
  volatile int* abort = (volatile int*)(tptr + 1);
  volatile uint32_t* rstart = (volatile uint32_t*)(tptr + 2);  // rounds the producer began
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t wlim = insts[0].p2.wait_ns;
  const int hook = insts[0].p2.hook;
  const uint32_t rank = cluster_rank();
  const int64_t cid = blockIdx.x / G, ncl = gridDim.x / G;

  if (threadIdx.x == 0) {
    for (int k = 0; k < P2I_SLOTS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    for (int k = 0; k < P2I_WSLOTS; ++k) {
      mbar_init(&wrfull[k], 1);
      mbar_init(&wrempty[k], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sfull[b], 1);
      mbar_init(&sempty[b], 128);
    }
    mbar_init(zfull, 1);
    mbar_init(zempty, 128);
    mbar_init(wfull, 128);
    mbar_init(wfree, 1);
    mbar_init(cdone, 1);
    mbar_init(drain, 1);
    mbar_init(never, 1);
    for (int k = 0; k < MBOX_DEPTH * P2C_MAX_G; ++k) mbox[k] = 0u;  // tag 0: no use yet
    *abort = 0;
    *rstart = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tptr, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  cluster_sync_all();  // every CTA's barriers and mailbox exist before any peer uses them
  const uint32_t tbase = *tptr;
  const int64_t total = ustart[n_inst];

  if (warp == 0) {
    if (lane == 0) {
      // main ring: logit operands of this CTA's block and the Y'^T tiles of its chunk, in
      // the MMA's order (Z' blocks of round j - 1 between the k-blocks of round j)
      uint32_t it = 0, g = 0;
      bool ok = true;
      auto reserve = [&]() -> int {
        const int st = it % P2I_SLOTS;
        if (!mbar_wait(&empty[st], ((it / P2I_SLOTS) & 1) ^ 1, abort, wlim)) {
          ok = false;
          return -1;
        }
        mbar_expect_tx(&full[st], 32768);
        return st;
      };
      for (int64_t u = cid; ok && u < total; u += ncl) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP2Args& a = I->p2;
        const int64_t lu = u - ustart[ki];
        const int ncg = (a.n_chunks + G - 1) / G;
        const int per_split = a.n_stiles * ncg;
        const int split = (int)(lu / per_split), rem = (int)(lu % per_split);
        const int stile = rem / ncg, chunk = (rem % ncg) * G + (int)rank;
        const bool cvalid = chunk < a.n_chunks;
        const int jb0 = split * a.iblk_per_split;
        const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
        const int rounds = (nb + G - 1) / G;
        for (int j = 0; ok && j <= rounds; ++j) {
          const int r0 = j * G, nq = j < rounds ? min(G, nb - r0) : 0;
          const int rp = (j - 1) * G, nqp = j >= 1 ? min(G, nb - rp) : 0;
          *rstart = ++g;  // the weight producer may announce the slots of round j - 1
          auto z_fills = [&](int i) {
            if (!cvalid) return;
            const int ib = (jb0 + rp + p2c_block((int)rank, nqp, i)) * 128;
            for (int h = 0; ok && h < 2; ++h) {
              const int s2 = reserve();
              if (!ok) break;
              tma_load_2d(smem + s2 * SLOT, &I->tmYT, &full[s2], ib + h * 64, chunk * 256);
              ++it;
            }
          };
          int zi = 0;
          if ((int)rank < nq) {  // logits of this CTA's own block
            const int ib = (jb0 + r0 + (int)rank) * 128;
            for (int kb = 0; ok && kb < a.nk; ++kb) {
              if (NPROD == 3) {
                int st = reserve();
                if (!ok) break;
                tma_load_2d(smem + st * SLOT, &I->tmA128, &full[st], kb * 64, stile * 128);
                tma_load_2d(smem + st * SLOT + 16384, &I->tmAl128, &full[st], kb * 64,
                            stile * 128);
                ++it;
                st = reserve();
                if (!ok) break;
                tma_load_2d(smem + st * SLOT, &I->tmY, &full[st], kb * 64, ib);
                tma_load_2d(smem + st * SLOT + 16384, &I->tmYl, &full[st], kb * 64, ib);
                ++it;
              } else {
                const int st = reserve();
                if (!ok) break;
                tma_load_2d(smem + st * SLOT, &I->tmA128, &full[st], kb * 64, stile * 128);
                tma_load_2d(smem + st * SLOT + 16384, &I->tmY, &full[st], kb * 64, ib);
                ++it;
              }
              for (; ok && zi < nqp && p2i_zpos(zi, nqp, a.nk) == kb; ++zi) z_fills(zi);
            }
          }
          for (; ok && zi < nqp; ++zi) z_fills(zi);
        }
      }
      if (!ok) raise_timeout(abort, status);
      {
        // the fills already issued land before the CTA exits, also when another role
        // gave up and stopped consuming them (in a normal run they are all consumed and
        // these waits return at once)
        const uint32_t lo = it > P2I_SLOTS ? it - P2I_SLOTS : 0;
        int zero = 0;
        for (uint32_t k = lo; k < it; ++k)
          mbar_wait(&full[k % P2I_SLOTS], (k / P2I_SLOTS) & 1, (volatile int*)&zero);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16_f32(128, 128);
      constexpr uint32_t idZ = idesc_f16_f32(128, 256);
      uint32_t it = 0, itw = 0, sc = 0, uc = 0, ow = 0;
      bool ok = true;
      auto wait_slot = [&]() -> int {
        const int st = it % P2I_SLOTS;
        if (!mbar_wait(&full[st], (it / P2I_SLOTS) & 1, abort, wlim)) {
          ok = false;
          return -1;
        }
        return st;
      };
      for (int64_t u = cid; ok && u < total; u += ncl) {
        const int ki = find_inst(ustart, n_inst, u);
        const TcInst* I = insts + ki;
        const TcP2Args& a = I->p2;
        const int64_t lu = u - ustart[ki];
        const int ncg = (a.n_chunks + G - 1) / G;
        const int per_split = a.n_stiles * ncg;
        const int rem = (int)(lu % per_split);
        const int chunk = (rem % ncg) * G + (int)rank;
        const bool cvalid = chunk < a.n_chunks;
        const int split = (int)(lu / per_split);
        const int jb0 = split * a.iblk_per_split;
        const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
        bool first_z = true;
        const int rounds = (nb + G - 1) / G;
        for (int j = 0; ok && j <= rounds; ++j) {
          const int r0 = j * G, nq = j < rounds ? min(G, nb - r0) : 0;
          const int nqp = j >= 1 ? min(G, nb - (j - 1) * G) : 0;
          // Z' block i of round j - 1: the own tile from the staging slot, the others'
          // from the weight ring, in this CTA's block order
          auto z_block = [&](int i) {
            const bool own = p2c_block((int)rank, nqp, i) == (int)rank;
            int sw = -1;
            if (own) {
              // the staged tile of this round is written (tiles without a chunk are
              // still consumed, so that the staging slot is released in order)
              if (!mbar_wait(wfull, ow & 1, abort, wlim)) {
                ok = false;
                return;
              }
            } else if (cvalid) {
              sw = itw % P2I_WSLOTS;
              if (!mbar_wait(&wrfull[sw], (itw / P2I_WSLOTS) & 1, abort, wlim)) {
                ok = false;
                return;
              }
              ++itw;
            }
            tc_fence_after();
            if (cvalid) {
              if (first_z && !mbar_wait(zempty, (uc & 1) ^ 1, abort, wlim)) {
                ok = false;
                return;
              }
              tc_fence_after();
              const uint32_t dZ = tbase + 256u;
              const uint8_t* wt = own ? stage : wring + sw * SLOT;
              for (int h = 0; ok && h < 2; ++h) {
                const int stT = wait_slot();
                if (!ok) break;
                tc_fence_after();
                const uint64_t dP = desc_sw128(wt + h * 16384);
                const uint64_t dT = desc_sw128(smem + stT * SLOT);
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4)
                  mma_bf16(dZ, desc_advance(dP, k4), desc_advance(dT, k4), idZ,
                           (!first_z || h > 0 || k4 > 0) ? 1u : 0u);
                mma_commit(&empty[stT]);
                ++it;
              }
              if (!ok) return;
              first_z = false;
            }
            if (own) {
              mma_commit(wfree);
              ++ow;
            } else if (cvalid) {
              mma_commit(&wrempty[sw]);
            }
          };
          int zi = 0;
          if ((int)rank < nq) {
            const int b = sc & 1;
            if (!mbar_wait(&sempty[b], ((sc >> 1) & 1) ^ 1, abort, wlim)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tbase + (uint32_t)(b * 128);
            for (int kb = 0; ok && kb < a.nk; ++kb) {
              const int stA = wait_slot();
              if (!ok) break;
              uint8_t* sA = smem + stA * SLOT;
              uint8_t* sY = sA + 16384;
              int stY = stA;
              if (NPROD == 3) {
                ++it;
                stY = wait_slot();
                if (!ok) break;
                sY = smem + stY * SLOT;
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
              if (kb == a.nk - 1) {
                mma_commit(&sfull[b]);  // the logits of round j are complete
                ++sc;
              }
              for (; ok && zi < nqp && p2i_zpos(zi, nqp, a.nk) == kb; ++zi) z_block(zi);
            }
            if (!ok) break;
          }
          for (; ok && zi < nqp; ++zi) z_block(zi);
        }
        if (!ok) break;
        if (cvalid) {
          mma_commit(zfull);
          ++uc;
        }
      }
      if (!ok) raise_timeout(abort, status);
      // every issued MMA completes before TMEM is released, also when another role
      // gave up and left accumulators unread
      mma_commit(drain);
      int zero = 0;
      mbar_wait(drain, 0, (volatile int*)&zero);
    }
  } else if (warp < 6) {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
    float2* wobs = (float2*)(stage + SLOT + P2I_BOOK) + q * 32;  // this warp's staging
    uint32_t sc = 0, m = 0, uc = 0;
    bool ok = true;
    for (int64_t u = cid; ok && u < total; u += ncl) {
      const int ki = find_inst(ustart, n_inst, u);
      const TcInst* I = insts + ki;
      const TcP2Args& a = I->p2;
      const int64_t lu = u - ustart[ki];
      const int ncg = (a.n_chunks + G - 1) / G;
      const int per_split = a.n_stiles * ncg;
      const int split = (int)(lu / per_split), rem = (int)(lu % per_split);
      const int stile = rem / ncg, cgrp = rem % ncg;
      const int chunk = cgrp * G + (int)rank;
      const bool cvalid = chunk < a.n_chunks;
      const int jb0 = split * a.iblk_per_split;
      const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
      const int s = stile * 128 + row;
      const float cb = a.colb[s], cm = a.colm[s];
      const float a2 = a.a2, c2 = a.c2;
      // per-block float32 sums of the rounded weights, added to float64 totals once a
      // block (a float32 total over thousands of observations would drop the small
      // weights of a shift against its large running sum)
      float cacc = 0.f, zacc = 0.f;
      double cacc_d = 0.0, zacc_d = 0.0;
      for (int r0 = 0; ok && r0 < nb; r0 += G) {
        const int nq = min(G, nb - r0);
        if ((int)rank >= nq) continue;
        const int64_t ib = (int64_t)(jb0 + r0 + (int)rank) * 128;
        const int b = sc & 1;
        // (ybar, lse2) of the next 32-observation chunk, loaded one chunk ahead of its
        // use; lse2 = +inf past N gives weight 0
        float ny = a.ybar[ib + lane];
        float nl = (ib + lane < a.N) ? a.lse2[ib + lane] : INFINITY;
        // test hook: see pass 1 (the first cluster's rank 0 never builds its first tile,
        // so its peers' waits for that tile run out as well)
        const bool held = hook == 2 && blockIdx.x == 0 && sc == 0;
        ok = __all_sync(0xffffffffu, (!held || mbar_wait(never, 0, abort, wlim)) &&
                                         mbar_wait(&sfull[b], (sc >> 1) & 1, abort, wlim));
        if (!ok) break;
        tc_fence_after();
        // the weights of this row, as fp16 pairs in the order of the tile's columns; they
        // are computed before the staging slot is free, so that the logit buffer is
        // released early
        uint32_t packed[64];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          __syncwarp();  // the warp is done with the previous chunk's terms
          wobs[lane] = make_float2(ny, nl);
          __syncwarp();
          if (c < 3) {
            const int64_t io = ib + (c + 1) * 32 + lane;
            ny = a.ybar[io];
            nl = (io < a.N) ? a.lse2[io] : INFINITY;
          }
          float v[32];
          tmem_ld32(lane_addr + (uint32_t)(b * 128 + c * 32), v);
          tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < 32; e += 2) {
            float w2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float2 yl = wobs[e + h];
              const float ybi = yl.x;
              const float dd = ybi - cm;
              const float val = fmaf(v[e + h], a2, cb - yl.y) - c2 * dd * dd;
              const float w = exp2f(val) * W_SCALE;
              w2[h] = __half2float(__float2half_rn(w));
              cacc += w2[h];
              zacc = fmaf(w2[h], ybi, zacc);
            }
            const __half2 pr = __floats2half2_rn(w2[0], w2[1]);
            packed[c * 16 + (e >> 1)] = *reinterpret_cast<const uint32_t*>(&pr);
          }
        }
        tc_fence_before();
        mbar_arrive(&sempty[b]);  // the logits are no longer needed
        // the staging slot is free once the MMAs and the copies of the previous tile
        // have read it
        ok = __all_sync(0xffffffffu, mbar_wait(wfree, (m & 1) ^ 1, abort, wlim) &&
                                         mbar_wait(cdone, (m & 1) ^ 1, abort, wlim));
        if (!ok) break;
        uint8_t* prow = stage + row * 128;
#pragma unroll
        for (int col16 = 0; col16 < 16; ++col16) {  // 16-byte units along the observations
          const int kb2 = col16 >> 3, cc = col16 & 7;
          *reinterpret_cast<uint4*>(prow + kb2 * 16384 + ((cc ^ (row & 7)) << 4)) =
              make_uint4(packed[4 * col16], packed[4 * col16 + 1], packed[4 * col16 + 2],
                         packed[4 * col16 + 3]);
        }
        fence_proxy_async_smem();
        mbar_arrive(wfull);
        cacc_d += (double)cacc;
        zacc_d += (double)zacc;
        cacc = zacc = 0.f;
        ++sc;
        ++m;
      }
      if (!ok) break;
      if (cvalid) {
        ok = __all_sync(0xffffffffu, mbar_wait(zfull, uc & 1, abort, wlim));
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
        ++uc;
      }
      if (cgrp == 0) {
        const int64_t part = (int64_t)split * G + rank;
        a.cp[part * a.Spad + s] = (float)(cacc_d * W_UNSCALE);
        a.zbp[part * a.Spad + s] = (float)(zacc_d * W_UNSCALE);
      }
    }
    if (!ok) raise_timeout(abort, status);
  } else if (warp == 6 && lane == 0) {
    // sender: each staged tile goes to every peer that owns a pixel chunk, into the
    // weight-ring slot that peer announced for this use of the tile, in the order the
    // announcements arrive
    uint32_t m = 0;
    bool ok = true;
    for (int64_t u = cid; ok && u < total; u += ncl) {
      const int ki = find_inst(ustart, n_inst, u);
      const TcP2Args& a = insts[ki].p2;
      const int64_t lu = u - ustart[ki];
      const int ncg = (a.n_chunks + G - 1) / G;
      const int per_split = a.n_stiles * ncg;
      const int split = (int)(lu / per_split), rem = (int)(lu % per_split);
      const int cgrp = rem % ncg;
      const int jb0 = split * a.iblk_per_split;
      const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
      uint32_t peers = 0;  // peers with a pixel chunk in this chunk group
      for (int k = 0; k < G; ++k)
        if (k != (int)rank && cgrp * G + k < a.n_chunks) peers |= 1u << k;
      for (int r0 = 0; ok && r0 < nb; r0 += G) {
        if ((int)rank >= min(G, nb - r0)) continue;
        if (!mbar_wait(wfull, m & 1, abort, wlim)) {
          ok = false;
          break;
        }
        const uint32_t* mrow = mbox + (m % MBOX_DEPTH) * P2C_MAX_G;
        const uint32_t expect = (m + 1u) & MBOX_TAG_MASK;
        uint32_t pending = peers;
        const uint64_t t0 = globaltimer();
        while (pending) {
          const uint32_t before = pending;
          for (uint32_t pm = pending; pm; pm &= pm - 1) {
            const int k = __ffs(pm) - 1;
            const uint32_t v = ld_acquire_cluster_u32(mrow + k);
            if ((v >> 4) == expect) {
              const uint32_t slot = v & 15u;
              bulk_copy_to_peer(mapa(smem_u32(wring + slot * SLOT), k), stage, 32768,
                                mapa(smem_u32(&wrfull[slot]), k));
              pending &= ~(1u << k);
            }
          }
          if (pending && (*abort || globaltimer() - t0 > wlim)) {
            ok = false;
            break;
          }
          // nothing announced: back off, so that the polling does not take shared-memory
          // bandwidth from the MMAs
          if (pending == before) __nanosleep(128);
        }
        bulk_commit();
        bulk_wait_read0();
        if (!ok) break;
        mbar_arrive(cdone);
        ++m;
      }
    }
    bulk_wait0();  // no copy is still landing in a peer when the cluster leaves
    if (!ok) raise_timeout(abort, status);
  } else if (warp == 7 && lane == 0) {
    // weight producer: a weight-ring slot for each peer's tile of round j - 1, announced
    // in that peer's mailbox once the main producer has begun round j (so that it runs at
    // most about a round ahead, also through units where this CTA owns no pixel chunk)
    uint32_t itw = 0, g = 0, sent[P2C_MAX_G] = {};
    bool ok = true;
    for (int64_t u = cid; ok && u < total; u += ncl) {
      const int ki = find_inst(ustart, n_inst, u);
      const TcP2Args& a = insts[ki].p2;
      const int64_t lu = u - ustart[ki];
      const int ncg = (a.n_chunks + G - 1) / G;
      const int per_split = a.n_stiles * ncg;
      const int split = (int)(lu / per_split), rem = (int)(lu % per_split);
      const int chunk = (rem % ncg) * G + (int)rank;
      const bool cvalid = chunk < a.n_chunks;
      const int jb0 = split * a.iblk_per_split;
      const int nb = min(a.n_iblk, jb0 + a.iblk_per_split) - jb0;
      const int rounds = (nb + G - 1) / G;
      ++g;  // round 0 of the unit multiplies no weight tiles
      for (int j = 1; ok && j <= rounds; ++j) {
        ++g;
        const uint64_t t0 = globaltimer();
        while (*rstart < g) {
          if (*abort || globaltimer() - t0 > wlim) {
            ok = false;
            break;
          }
          __nanosleep(64);
        }
        if (!ok) break;
        const int nqp = min(G, nb - (j - 1) * G);
        for (int i = 0; ok && i < nqp; ++i) {
          const int kq = p2c_block((int)rank, nqp, i);
          if (kq == (int)rank) continue;
          if (!cvalid) {  // not taken, but counted: later tags stay in step
            ++sent[kq];
            continue;
          }
          const int sw = itw % P2I_WSLOTS;
          if (!mbar_wait(&wrempty[sw], ((itw / P2I_WSLOTS) & 1) ^ 1, abort, wlim)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&wrfull[sw], 32768);
          const uint32_t row = sent[kq] % MBOX_DEPTH;
          const uint32_t tag = (sent[kq] + 1u) & MBOX_TAG_MASK;
          st_release_cluster_u32(mapa(smem_u32(mbox + row * P2C_MAX_G + rank), kq),
                                 (tag << 4) | (uint32_t)sw);
          ++sent[kq];
          ++itw;
        }
      }
    }
    if (!ok) {
      raise_timeout(abort, status);
      const uint32_t lo = itw > P2I_WSLOTS ? itw - P2I_WSLOTS : 0;
      int zero = 0;
      for (uint32_t q = lo; q < itw; ++q)
        mbar_wait(&wrfull[q % P2I_WSLOTS], (q / P2I_WSLOTS) & 1, (volatile int*)&zero);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
  cluster_sync_all();  // no CTA leaves while a peer may still copy into it
}

// ring + staging slot + bookkeeping (22 mbarriers, 8 x 16 mailbox, TMEM address, abort
// flag: 696 of the 768 bytes) + per-warp staging of one 32-observation chunk's
// (ybar, lse2) (4 x 256 bytes)
// main ring + weight ring + staging slot + bookkeeping + per-warp (ybar, lse2) staging
constexpr size_t P2I_SMEM = 1024 + (P2I_SLOTS + P2I_WSLOTS + 1) * SLOT + P2I_BOOK + 1024;
static_assert(P2I_SMEM <= 232448, "exceeds the shared memory of one CTA");

constexpr size_t P1_SMEM = 1024 + P1_SLOTS * SLOT + 256 + 1024;
constexpr size_t P2_SMEM = 1024 + P2_SLOTS_PLAIN * SLOT + 2 * SLOT + 256 + 1024;
constexpr size_t P2_SMEM_COMP = 1024 + P2_SLOTS_COMP * SLOT + 4 * SLOT + 256 + 1024;
static_assert(P2_SMEM <= 232448, "exceeds the shared memory of one CTA");
static_assert(P2_SMEM_COMP <= 232448, "exceeds the shared memory of one CTA");

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

// YT[p][i] = fp16(y'_i[p]) for p < l2 (32x32 tiles): the M-step operand; with out_lo,
// also its rounding residual fp16(y' - YT) (the compensated M-step's lo part).
__global__ void k_transpose_f16(const float* __restrict__ in, int64_t R, int ld_in, int C,
                                __half* __restrict__ out, __half* __restrict__ out_lo) {
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
    if (c < C && r < R) {
      const float v = tile[threadIdx.x][k];
      const __half h = __float2half_rn(v);
      out[(int64_t)c * R + r] = h;
      if (out_lo) out_lo[(int64_t)c * R + r] = __float2half_rn(v - __half2float(h));
    }
  }
}

__device__ __forceinline__ int mod_pos(int a, int m) {
  const int r = a % m;
  return r < 0 ? r + m : r;
}

// Centred templates, shift-major bf16 hi / lo: T[s][n] = x'_r(s)[n - t(s)], zero for
// padding.  One warp per shift: the phase, lag and sub-image mean are per shift, the
// lanes walk the pixels n2 of each row n1; the subtraction of the mean is float32 (a
// rounding of the mean common to a sub-image cancels in <y', T'>, every y' sums to zero).
__global__ void __launch_bounds__(256) k_templates_bf16(
    const float* __restrict__ x, const double* __restrict__ sub, int L, int K, int l, int S,
    int Spad, int l2, int ldk, __nv_bfloat16* __restrict__ Ah, __nv_bfloat16* __restrict__ Al) {
  const int s = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (s >= Spad) return;
  __nv_bfloat16* rh = Ah + (int64_t)s * ldk;
  __nv_bfloat16* rl = Al ? Al + (int64_t)s * ldk : nullptr;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  if (s >= S) {
    for (int n = lane; n < ldk; n += 32) {
      rh[n] = zero;
      if (rl) rl[n] = zero;
    }
    return;
  }
  const int s1 = s / L, s2 = s % L;
  const int r1 = mod_pos(-s1, K), r2 = mod_pos(-s2, K);
  const int t1 = ((s1 + r1) / K) % l, t2 = ((s2 + r2) / K) % l;
  const float mr = (float)sub[r1 * K + r2];
  for (int n1 = 0; n1 < l; ++n1) {
    const float* row = x + (r1 + mod_pos(n1 - t1, l) * K) * L + r2;
    for (int n2 = lane; n2 < l; n2 += 32) {
      int m2 = n2 - t2;
      m2 += m2 < 0 ? l : 0;
      const float v = row[m2 * K] - mr;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      rh[n1 * l + n2] = h;
      if (rl) rl[n1 * l + n2] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
  for (int n = l2 + lane; n < ldk; n += 32) {
    rh[n] = zero;
    if (rl) rl[n] = zero;
  }
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

// the clustered pass-2 kernels: their shared memory, and clusters above the portable
// size for the interleaved form
template <int NPROD>
cudaError_t set_p2c_attrs() {
  cudaError_t e = set_smem(k_p2c_tc<NPROD>, P2R_SMEM);
  if (e == cudaSuccess) e = set_smem(k_p2i_tc<NPROD>, P2I_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_p2i_tc<NPROD>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

template <int NPROD, int BN>
cudaError_t set_p1_attrs() {
  return set_smem(k_p1_tc<NPROD, BN>, P1_SMEM);
}
template <int NPROD>
cudaError_t set_p2_attrs() {
  return set_smem(k_p2_tc<NPROD, false>, P2_SMEM);
}
cudaError_t set_p2comp_attrs() { return set_smem(k_p2_tc<3, true>, P2_SMEM_COMP); }
cudaError_t set_p2p_attrs() { return set_smem(k_p2p_tc<3>, P2P_SMEM); }

// The cluster form for clusters of G: the ring form up to P2R_MAX_G, the interleaved
// form above.
bool p2_ring_form(int G) { return G <= P2R_MAX_G; }

// The launch shape of that form.
template <int NPROD>
void p2c_form(int G, const void** fn, int* threads, size_t* smem) {
  if (p2_ring_form(G)) {
    *fn = (const void*)k_p2c_tc<NPROD>;
    *threads = TC_THREADS;
    *smem = P2R_SMEM;
  } else {
    *fn = (const void*)k_p2i_tc<NPROD>;
    *threads = P2I_THREADS;
    *smem = P2I_SMEM;
  }
}

}  // namespace

int choose_p2_cluster(int chunks, int l2, int64_t n_iblk, int prec, int num_sms);
template <int NPROD>
int max_clusters_p2(int G, int num_sms);
int max_clusters_pair(int G, int num_sms);

// Whether a bf16x3 context takes the compensated M-step (hi + lo fp16 operands for
// Z' = W^T Y').  With single fp16 operands the rounding of the weights and of Y'
// (2^-11 relative each) reaches x through sums over the observations of each
// sub-image, so its effect shrinks as they grow in number: measured (emulated in
// float64 with the same roundings, one iteration from the workloads' initial guess) it
// is 1.5e-4 at L = 128, K = 2, N = 300, sigma = 0.5; 2.3e-5 with N = 1200; 9.6e-5 at
// L = 96, K = 2, N = 300; 4.4e-5 at L = 64, K = 2, N = 300; below 1e-5 from a few
// thousand observations, at sigma = 1 included.  Below N = 31.25 l max(1, 2 sigma)
// (2000 at l = 64, sigma <= 0.5) that estimate can pass 2e-5, a fifth of the mixed
// form's 1e-4 target, and the compensated per-chunk kernel is used instead of the
// cluster forms.  SRMRA_FLAG_MSTEP_COMP forces it, SRMRA_FLAG_MSTEP_FP16 rules it out.
bool tc_comp_mstep(const Geom& g, int prec, unsigned flags) {
  if (prec != SRMRA_BF16X3) return false;
  if (flags & SRMRA_FLAG_MSTEP_COMP) return true;
  if (flags & SRMRA_FLAG_MSTEP_FP16) return false;
  const double n_min = 31.25 * (double)g.l * std::max(1.0, 2.0 * g.sigma);
  return (double)g.N < n_min;
}

// Pass-2 launch group of a context: its cluster size, 0 for the compensated per-chunk
// kernel, P2_KEY_PAIR + G for the pair form with G pairs.
int tc_p2_key(const srmra_ctx* c) {
  if (c->plan.p2_comp) return 0;
  return c->plan.p2_pair ? P2_KEY_PAIR + c->plan.p2_gc : c->plan.p2_gc;
}

// Whether a context takes the pair form of pass 2: split-bf16 operands with the single
// fp16 M-step, clusters allowed, up to four 256-pixel chunks (one per pair), and
// SRMRA_FLAG_P2_PAIR set.
bool tc_pair_form(const Geom& g, int prec, unsigned flags, bool comp) {
  if (prec != SRMRA_BF16X3 || comp || (flags & SRMRA_FLAG_NO_CLUSTER)) return false;
  if (!(flags & SRMRA_FLAG_P2_PAIR)) return false;
  const int chunks = (g.l2 + 255) / 256;
  return chunks >= 1 && chunks <= P2P_MAX_G;
}

// Work decomposition of the tensor-core passes.  s1 multiplies the number of shift
// groups of pass 1 and s2 the number of observation ranges of pass 2: finer units
// balance a grouped launch better at the price of more partial sums.  The result is
// clamped to the capacities the context's buffers were sized for.
void plan_tc(srmra_ctx* c, int s1, int s2) {
  const Geom& g = c->g;
  Plan& p = c->plan;
  const int sms = c->num_sms;
  const int n_st1 = g.Spad / p.p1_bn;
  const int iblk1 = (int)(g.Npad / 128);
  // pass 1 is a persistent kernel that deals its (observation block, shift group) units
  // round-robin to one CTA per SM: pick the shift-group size that minimises the rounds
  // times the tiles per unit (plus a quarter tile of per-unit overhead), i.e. the time
  // of the busiest CTA, so that the last round is not left mostly empty
  int groups = 1;
  double best = 0.0;
  for (int tpg = n_st1; tpg >= 1; --tpg) {
    const int gr = (int)ceil_div(n_st1, tpg);
    if (ceil_div(n_st1, gr) != tpg) continue;
    const int64_t rounds = ceil_div((int64_t)gr * iblk1, sms);
    const double cost = (double)rounds * (tpg + 0.25);
    if (best == 0.0 || cost < best) {
      best = cost;
      groups = gr;
    }
  }
  groups *= s1;
  groups = groups < 1 ? 1 : (groups > n_st1 ? n_st1 : groups);
  if (p.cap_p1_groups > 0 && groups > p.cap_p1_groups) groups = p.cap_p1_groups;
  p.p1_tiles_per_group = (int)ceil_div(n_st1, groups);
  p.p1_groups = (int)ceil_div(n_st1, p.p1_tiles_per_group);

  const int n_st2 = g.Spad / 128;
  const int chunks = (int)ceil_div(g.l2, 256);
  const int n_iblk = (int)(g.Npad / 128);
  // cluster size of pass 2: CTAs that share each weight tile, one pixel chunk each
  const int G = p.p2_pair ? chunks
                          : (c->no_cluster || p.p2_comp)
                                ? 1
                                : choose_p2_cluster(chunks, g.l2, n_iblk, c->prec, sms);
  // observation splits of pass 2: each split adds a partial Z' (Spad x l2 float32) that
  // pass 2 writes and the finalize reads, so take the split count that minimises the
  // busiest cluster's block-rounds plus the partials' cost in the same units (a partial
  // of 4096 x 1024 floats measured about 1.4 block-rounds)
  const int ncg = (int)ceil_div(chunks, G);
  const int64_t slots2 = p.p2_pair ? (int64_t)std::max(1, max_clusters_pair(G, sms))
                         : G > 1 ? (int64_t)(c->prec == SRMRA_BF16X3 ? max_clusters_p2<3>(G, sms)
                                                                     : max_clusters_p2<1>(G, sms))
                                 : (int64_t)sms;
  // work units per observation range: (shift tile, chunk group), or pairs of shift tiles
  const int64_t st_units = p.p2_pair ? n_st2 / 2 : n_st2;
  const double part_cost = 1.4 * (double)g.Spad * (double)g.ldy / (4096.0 * 1024.0);
  // no more splits than about four units per SM would give (bounds the partial buffers)
  const int64_t per_split_old = (int64_t)n_st2 * chunks;
  const int ns_max = (int)std::max<int64_t>(1, (4 * (int64_t)sms + per_split_old / 2) /
                                                   per_split_old);
  // The tensor cores add each MMA's products into the f32 TMEM accumulator rounding
  // toward zero, so a Z' entry summed over many MMAs drifts toward zero by about half
  // an ulp per addition: measured (L=96, K=3, sigma=1, one iteration against the FP64
  // oracle) 4.2e-5 on x with the 3128 additions of 5e4 observations in one split, 9.8e-6
  // with 6000, and three times as much with the three MMAs of the compensated M-step.
  // So no split adds more than P2_MAX_ACC MMAs into one accumulator (8 per block of
  // 128 observations, 24 compensated); the partial sums of the splits are added in the
  // finalize with ordinary rounding.
  const int acc_per_block = p.p2_comp ? 24 : 8;
  const int blocks_max = std::max(1, P2_MAX_ACC / acc_per_block);
  const int ns_acc = (int)std::min<int64_t>(64, ceil_div(n_iblk, blocks_max));
  int ns = 1;
  double best_ns = 0.0;
  for (int cand = ns_acc; cand <= std::max(ns_max, ns_acc) && cand <= 64 && cand <= n_iblk;
       ++cand) {
    const int64_t per = ceil_div(n_iblk, cand);
    if (cand > 1 && ceil_div(n_iblk, per) != cand) continue;
    const int64_t units = st_units * ncg * cand;
    const double cost = (double)ceil_div(units, slots2) * (double)per + part_cost * cand;
    if (best_ns == 0.0 || cost < best_ns) {
      best_ns = cost;
      ns = cand;
    }
  }
  ns *= s2;
  ns = std::max(ns, ns_acc);
  ns = ns < 1 ? 1 : (ns > n_iblk ? n_iblk : ns);
  if (ns > 64) ns = 64;
  if (p.cap_nsplit > 0 && ns > p.cap_nsplit) ns = p.cap_nsplit;
  p.p2_iblk_per_split = (int)ceil_div(n_iblk, ns);
  p.p2_nsplit = (int)ceil_div(n_iblk, p.p2_iblk_per_split);
  p.p2_gc = G;
  p.p2_chunk_groups = (int)ceil_div(chunks, G);
  p.nparts_z = p.p2_nsplit;
  p.nparts_c = p.p2_nsplit * G;
  p.ll_blocks = (int)ceil_div(g.Npad, 256);
}

cudaError_t tc_replan(srmra_ctx* c, int s1, int s2, int p1_bn) {
  c->plan.p1_bn = p1_bn;
  plan_tc(c, s1, s2);
  return tc_upload_inst(c);
}

cudaError_t tc_set_attributes(int prec) {
  cudaError_t e;
  if (prec == SRMRA_BF16X3) {
    e = set_smem(k_p1_tc<3, 256>, P1_SMEM);
    if (e == cudaSuccess) e = set_smem(k_p1_tc<3, 128>, P1_SMEM);
    if (e == cudaSuccess) e = set_smem(k_p2_tc<3, false>, P2_SMEM);
    if (e == cudaSuccess) e = set_p2comp_attrs();
    if (e == cudaSuccess) e = set_p2c_attrs<3>();
    if (e == cudaSuccess) e = set_p2p_attrs();
  } else {
    e = set_smem(k_p1_tc<1, 256>, P1_SMEM);
    if (e == cudaSuccess) e = set_smem(k_p1_tc<1, 128>, P1_SMEM);
    if (e == cudaSuccess) e = set_smem(k_p2_tc<1, false>, P2_SMEM);
    if (e == cudaSuccess) e = set_p2c_attrs<1>();
  }
  return e;
}

cudaError_t prep_obs_tc(srmra_ctx* c) {
  const Geom& g = c->g;
  const int64_t n = g.Npad * g.ldk;
  k_split_obs<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(
      c->Yc, g.ldy, g.l2, g.Npad, g.ldk, c->Yh, c->prec == SRMRA_BF16X3 ? c->Yl : nullptr);
  dim3 grid((unsigned)ceil_div(g.l2, 32), (unsigned)ceil_div(g.Npad, 32));
  k_transpose_f16<<<grid, dim3(32, 8), 0, c->stream>>>(c->Yc, g.Npad, g.ldy, g.l2, c->YTf,
                                                      c->plan.p2_comp ? c->YTfl : nullptr);
  c->launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // tensor maps over the fixed operands
  bool ok = make_map(&c->tmY128, c->Yh, g.ldk, g.Npad, g.ldk, 128) &&
            make_map(&c->tmYT, c->YTf, g.Npad, g.l2, g.Npad, 256,
                     CU_TENSOR_MAP_DATA_TYPE_FLOAT16) &&
            make_map(&c->tmA128, c->Ah, g.ldk, g.Spad, g.ldk, 128) &&
            make_map(&c->tmA256, c->Ah, g.ldk, g.Spad, g.ldk, 256);
  if (ok && c->plan.p2_comp)
    ok = make_map(&c->tmYTl, c->YTfl, g.Npad, g.l2, g.Npad, 256, CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
  if (ok && c->prec == SRMRA_BF16X3)
    ok = make_map(&c->tmYl128, c->Yl, g.ldk, g.Npad, g.ldk, 128) &&
         make_map(&c->tmAl128, c->Al, g.ldk, g.Spad, g.ldk, 128) &&
         make_map(&c->tmAl256, c->Al, g.ldk, g.Spad, g.ldk, 256) &&
         make_map(&c->tmY64, c->Yh, g.ldk, g.Npad, g.ldk, 64) &&
         make_map(&c->tmYl64, c->Yl, g.ldk, g.Npad, g.ldk, 64) &&
         make_map(&c->tmYT128, c->YTf, g.Npad, g.l2, g.Npad, 128,
                  CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
  if (!ok) return cudaErrorInvalidValue;
  return tc_upload_inst(c);
}

void launch_templates_tc(srmra_ctx* c) {
  const Geom& g = c->g;
  k_templates_bf16<<<(unsigned)ceil_div(g.Spad, 8), 256, 0, c->stream>>>(
      c->x, c->sub, g.L, g.K, g.l, g.S, g.Spad, g.l2, g.ldk, c->Ah,
      c->prec == SRMRA_BF16X3 ? c->Al : nullptr);
  c->launches++;
}

namespace {

// Fills the descriptor of one context (arguments of both passes and its tensor maps).
void fill_inst(const srmra_ctx* c, TcInst* I) {
  const Geom& g = c->g;
  const Plan& p = c->plan;
  const LogitScalars ls = logit_scalars(g);
  memset(I, 0, sizeof(TcInst));
  I->tmY = c->tmY128;
  I->tmYl = (c->prec == SRMRA_BF16X3) ? c->tmYl128 : c->tmY128;
  I->tmA256 = c->tmA256;
  I->tmAl256 = (c->prec == SRMRA_BF16X3) ? c->tmAl256 : c->tmA256;
  I->tmA128 = c->tmA128;
  I->tmAl128 = (c->prec == SRMRA_BF16X3) ? c->tmAl128 : c->tmA128;
  I->tmYT = c->tmYT;
  I->tmYTl = c->plan.p2_comp ? c->tmYTl : c->tmYT;
  I->tmY64 = c->tmY64;
  I->tmYl64 = c->tmYl64;
  I->tmYT128 = c->tmYT128;
  TcP1Args& a = I->p1;
  a.nk = (int)ceil_div(g.l2, 64);
  a.n_stiles = g.Spad / p.p1_bn;
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
  a.wait_ns = c->wait_ns;
  a.hook = c->test_hook;
  TcP2Args& b = I->p2;
  b.nk = a.nk;
  b.n_stiles = g.Spad / 128;
  b.n_chunks = (int)ceil_div(g.l2, 256);
  b.n_iblk = (int)(g.Npad / 128);
  b.iblk_per_split = p.p2_iblk_per_split;
  // work units of pass 2: (shift tile, chunk group, observation range); a chunk group is
  // one pixel chunk for the per-chunk kernel and G chunks for the cluster kernel
  // (the pair form takes two shift tiles per unit, one per CTA of a pair)
  b.n_units = (int64_t)(p.p2_pair ? b.n_stiles / 2 : b.n_stiles) * p.p2_chunk_groups *
              p.p2_nsplit;
  b.N = g.N;
  b.Spad = g.Spad;
  b.ldy = g.ldy;
  b.ybar = c->ybar;
  b.colb = c->colb;
  b.colm = c->colm;
  b.lse2 = c->lse2;
  b.a2 = ls.a2;
  b.c2 = ls.c2;
  b.Zp = c->Zp;
  b.cp = c->cp;
  b.zbp = c->zbp;
  b.status = c->status;
  b.wait_ns = c->wait_ns;
  b.hook = c->test_hook;
}

// Co-resident clusters of G CTAs of the clustered pass-2 kernel of that size (queried
// once per G); 0 for a cluster size above the portable limit that the GPU cannot place.
template <int NPROD>
int max_clusters(int G, int num_sms) {
  // per (device, G): the answer depends on the device's GPC layout
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  std::lock_guard<std::mutex> lock(mu);
  {
    auto hit = cache.find({dev, G});
    if (hit != cache.end()) return hit->second > 0 ? hit->second : 0;
  }
  cudaGetLastError();
  set_p2c_attrs<NPROD>();
  const void* fn;
  int threads;
  size_t smem;
  p2c_form<NPROD>(G, &fn, &threads, &smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(G * (num_sms / G)), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess || n < 1) {
    cudaGetLastError();
    if (G > P2C_PORTABLE_G) {
      cache[{dev, G}] = -1;
      return 0;
    }
    n = num_sms / G / 2 > 0 ? num_sms / G / 2 : 1;
  }
  cache[{dev, G}] = n;
  return n;
}

template <int NPROD>
cudaError_t launch_cluster_p2(int G, const TcInst* d_insts, const int64_t* d_ustart, int n,
                              int64_t total, int* status, cudaStream_t stream, int num_sms) {
  {
    cudaError_t e = once_per_device(ATTR_TC_P2C + NPROD, set_p2c_attrs<NPROD>);
    if (e != cudaSuccess) return e;
  }
  if (G < 2 || G > P2C_MAX_G) return cudaErrorInvalidValue;
  int ncl = max_clusters<NPROD>(G, num_sms);
  if (ncl < 1) return cudaErrorInvalidConfiguration;  // chosen only where it can be placed
  if (total < ncl) ncl = (int)total;
  if (ncl < 1) return cudaSuccess;
  const void* fn;
  int threads;
  size_t smem;
  p2c_form<NPROD>(G, &fn, &threads, &smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(G * ncl), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)G;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (p2_ring_form(G))
    return cudaLaunchKernelEx(&cfg, k_p2c_tc<NPROD>, d_insts, d_ustart, n, G, status);
  return cudaLaunchKernelEx(&cfg, k_p2i_tc<NPROD>, d_insts, d_ustart, n, G, status);
}

// Co-resident clusters of G pairs (2G CTAs) of the pair-form kernel (queried once per
// device and G); 0 if the GPU cannot place one.
int max_clusters_pair_impl(int G, int num_sms) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  std::lock_guard<std::mutex> lock(mu);
  {
    auto hit = cache.find({dev, G});
    if (hit != cache.end()) return hit->second;
  }
  cudaGetLastError();
  set_p2p_attrs();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * G * (num_sms / (2 * G))), 1, 1);
  cfg.blockDim = dim3((unsigned)TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = P2P_SMEM;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)(2 * G);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_p2p_tc<3>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cache[{dev, G}] = n > 0 ? n : 0;
  return n > 0 ? n : 0;
}

cudaError_t launch_pair_p2(int G, const TcInst* d_insts, const int64_t* d_ustart, int n,
                           int64_t total, int* status, cudaStream_t stream, int num_sms) {
  {
    cudaError_t e = once_per_device(ATTR_TC_P2P, set_p2p_attrs);
    if (e != cudaSuccess) return e;
  }
  if (G < 1 || G > P2P_MAX_G) return cudaErrorInvalidValue;
  int ncl = max_clusters_pair_impl(G, num_sms);
  if (ncl < 1) return cudaErrorInvalidConfiguration;
  if (total < ncl) ncl = (int)total;
  if (ncl < 1) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * G * ncl), 1, 1);
  cfg.blockDim = dim3((unsigned)TC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = P2P_SMEM;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)(2 * G);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_p2p_tc<3>, d_insts, d_ustart, n, G, status);
}

template <int NPROD>
cudaError_t launch_group(int pass, int bn, const TcInst* d_insts, const int64_t* d_ustart, int n,
                         int64_t total, int* status, cudaStream_t stream, int num_sms) {
  cudaError_t e = cudaSuccess;
  const unsigned grid = (unsigned)(total < num_sms ? total : num_sms);
  if (grid == 0) return cudaSuccess;
  if (pass == 1 && bn == 128) {
    e = once_per_device(ATTR_TC_P1N + NPROD, set_p1_attrs<NPROD, 128>);
    if (e != cudaSuccess) return e;
    k_p1_tc<NPROD, 128><<<grid, TC_THREADS, P1_SMEM, stream>>>(d_insts, d_ustart, n, status);
  } else if (pass == 1) {
    e = once_per_device(ATTR_TC_P1 + NPROD, set_p1_attrs<NPROD, 256>);
    if (e != cudaSuccess) return e;
    k_p1_tc<NPROD, 256><<<grid, TC_THREADS, P1_SMEM, stream>>>(d_insts, d_ustart, n, status);
  } else {
    e = once_per_device(ATTR_TC_P2 + NPROD, set_p2_attrs<NPROD>);
    if (e != cudaSuccess) return e;
    k_p2_tc<NPROD, false><<<grid, TC_THREADS, P2_SMEM, stream>>>(d_insts, d_ustart, n, status);
  }
  return cudaGetLastError();
}

}  // namespace

template <int NPROD>
int max_clusters_p2(int G, int num_sms) {
  return max_clusters<NPROD>(G, num_sms);
}
template int max_clusters_p2<1>(int, int);
template int max_clusters_p2<3>(int, int);
int max_clusters_pair(int G, int num_sms) { return max_clusters_pair_impl(G, num_sms); }

// Cluster size of pass 2 for `chunks` 256-pixel chunks of Z' (l2 pixels, n_iblk blocks of
// 128 observations).  Up to 4 chunks one cluster covers them all (G = chunks, ring form).
// Beyond, the weights of a (shift tile, observation block) are computed once per group
// of G chunks, and G trades that recompute against the cost of a round and how many
// clusters of G co-reside (GPC packing).  A cluster round takes about a * NPROD * l2 (the
// logits of the CTA's own block) + b * G (one weight tile handed over per member), with
// a = 2.93 ns and b = 4.3 us (ring form, G <= 4) or 3.3 us (interleaved form), fitted
// to measured pass-2 times (L = 72..128, K = 2, G = 3..16); the busiest
// cluster runs groups * ceil(n_iblk / G) / clusters(G) rounds per shift tile.
int choose_p2_cluster(int chunks, int l2, int64_t n_iblk, int prec, int num_sms) {
  if (chunks <= 1) return 1;
  if (chunks <= P2R_MAX_G) return chunks;
  const int nprod = prec == SRMRA_BF16X3 ? 3 : 1;
  constexpr double a_us = 2.93e-3, b_ring_us = 4.3, b_inter_us = 3.3;
  int best = P2R_MAX_G;
  double best_cost = 0.0;
  for (int G = 2; G <= P2C_MAX_G && G <= chunks; ++G) {
    const int ncl = nprod == 3 ? max_clusters<3>(G, num_sms) : max_clusters<1>(G, num_sms);
    if (ncl < 1) continue;
    const double groups = (double)((chunks + G - 1) / G);
    const double rounds = groups * (double)((n_iblk + G - 1) / G) / (double)ncl;
    const double b_us = G <= P2R_MAX_G ? b_ring_us : b_inter_us;
    const double cost = rounds * (a_us * nprod * l2 + b_us * G);
    if (best_cost == 0.0 || cost < best_cost) {
      best = G;
      best_cost = cost;
    }
  }
  return best;
}

size_t tc_inst_bytes() { return sizeof(TcInst); }

void tc_fill_inst(const srmra_ctx* c, void* host_dst) { fill_inst(c, (TcInst*)host_dst); }

int64_t tc_units(const srmra_ctx* c, int pass) {
  TcInst I;
  fill_inst(c, &I);
  return pass == 1 ? I.p1.n_units : I.p2.n_units;
}

cudaError_t tc_launch_group_p2(int G, int prec, const void* d_insts, const int64_t* d_ustart,
                               int n, int64_t total, int* status, cudaStream_t stream,
                               int num_sms) {
  const TcInst* insts = (const TcInst*)d_insts;
  if (G > P2_KEY_PAIR) {  // the pair form (bf16x3 only)
    if (prec != SRMRA_BF16X3) return cudaErrorInvalidValue;
    return launch_pair_p2(G - P2_KEY_PAIR, insts, d_ustart, n, total, status, stream, num_sms);
  }
  if (G == 0) {  // the per-chunk kernel with the compensated M-step (bf16x3 only)
    if (prec != SRMRA_BF16X3) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)(total < num_sms ? total : num_sms);
    if (grid == 0) return cudaSuccess;
    cudaError_t e = once_per_device(ATTR_TC_P2COMP, set_p2comp_attrs);
    if (e != cudaSuccess) return e;
    k_p2_tc<3, true><<<grid, TC_THREADS, P2_SMEM_COMP, stream>>>(insts, d_ustart, n, status);
    return cudaGetLastError();
  }
  if (G <= 1)
    return tc_launch_group(2, prec, 256, d_insts, d_ustart, n, total, status, stream, num_sms);
  if (prec == SRMRA_BF16X3)
    return launch_cluster_p2<3>(G, insts, d_ustart, n, total, status, stream, num_sms);
  return launch_cluster_p2<1>(G, insts, d_ustart, n, total, status, stream, num_sms);
}

cudaError_t tc_launch_group(int pass, int prec, int p1_bn, const void* d_insts,
                            const int64_t* d_ustart, int n, int64_t total, int* status,
                            cudaStream_t stream, int num_sms) {
  const TcInst* insts = (const TcInst*)d_insts;
  if (pass == 1 && p1_bn != 256 && p1_bn != 128) return cudaErrorInvalidValue;
  if (prec == SRMRA_BF16X3)
    return launch_group<3>(pass, p1_bn, insts, d_ustart, n, total, status, stream, num_sms);
  return launch_group<1>(pass, p1_bn, insts, d_ustart, n, total, status, stream, num_sms);
}

// The context's own descriptor (a group of one) in device memory, uploaded once.
cudaError_t tc_upload_inst(srmra_ctx* c) {
  c->h_inst.resize(sizeof(TcInst) + 64);
  TcInst* I = (TcInst*)(((uintptr_t)c->h_inst.data() + 63) & ~(uintptr_t)63);
  fill_inst(c, I);
  c->h_ustart[0] = 0;
  c->h_ustart[1] = I->p1.n_units;
  c->h_ustart[2] = 0;
  c->h_ustart[3] = I->p2.n_units;
  cudaError_t e = cudaMemcpyAsync(c->d_inst, I, sizeof(TcInst), cudaMemcpyHostToDevice,
                                  c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_ustart, c->h_ustart, sizeof(c->h_ustart), cudaMemcpyHostToDevice,
                        c->stream);
  return e;
}

cudaError_t launch_pass1_tc(srmra_ctx* c) {
  c->launches++;
  return tc_launch_group(1, c->prec, c->plan.p1_bn, c->d_inst, c->d_ustart, 1, c->h_ustart[1],
                         c->status, c->stream, c->num_sms);
}

cudaError_t launch_pass2_tc(srmra_ctx* c) {
  c->launches++;
  return tc_launch_group_p2(tc_p2_key(c), c->prec, c->d_inst, c->d_ustart + 2, 1,
                            c->h_ustart[3], c->status, c->stream, c->num_sms);
}

}  // namespace srmra
