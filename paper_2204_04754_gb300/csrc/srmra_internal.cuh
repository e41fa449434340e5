// Internal declarations of libsrmra: the context, device-buffer layout and the kernel
// launchers shared by the host driver (api.cu) and the kernel files.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/srmra.h"

namespace srmra {

// Device status word bits (set by kernels, read by the host after a sync).
enum : int {
  STATUS_TIMEOUT = 1,   // a bounded mbarrier / flag wait gave up
  STATUS_NUMERIC = 2,   // NaN / Inf in LL, x or rho
};

// Tile sizes of the float32 (CUDA-core) kernels.
constexpr int P1_BM = 128;  // pass 1: observations per tile
constexpr int P1_BN = 128;  // pass 1: shifts per tile
constexpr int P2_BS = 64;   // pass 2: shifts per tile
constexpr int P2_BI = 64;   // pass 2: observations per round
constexpr int P2_BP = 256;  // pass 2: pixels of the M-step sum per CTA
constexpr int NPAD = 128;   // observation padding (multiple of every i-tile)
constexpr int SPAD = 256;   // shift padding (multiple of every s-tile)

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Kernel attributes (opt-in shared memory, non-portable cluster sizes) apply to the
// device that is current when they are set, and a process may hold contexts on several
// devices.  once_per_device(key, set) runs `set` once for each (current device, key)
// pair, under a mutex (contexts may be driven from several threads), and remembers only
// a success.
enum : int {
  ATTR_SIMT_P2 = 0,
  ATTR_TC_P1 = 1,     // + NPROD (1 or 3)
  ATTR_TC_P2 = 5,     // + NPROD
  ATTR_TC_P2C = 9,    // + NPROD
  ATTR_TC_P2COMP = 13,
  ATTR_TC_P1N = 14,   // + NPROD: the 128-shift pass-1 tiles
  ATTR_TC_P2P = 18,   // the pair form of pass 2
};
cudaError_t once_per_device(int key, cudaError_t (*set)());

// Geometry of one problem, shared by all kernels.
struct Geom {
  int L, K, l, l2;  // L_high, factor, L_low, L_low^2
  int S;            // L^2 shifts
  int Spad;         // S rounded up to SPAD
  int ldy;          // pitch (pixels) of a centred observation row, l2 rounded up to 16
  int ldk;          // pitch of the bf16 operand rows (tensor-core form), l2 rounded up to 64
  int64_t N;        // observations
  int64_t Npad;     // N rounded up to NPAD
  double sigma;
};

// Per-iteration scalars of the logit in base-2 units:
//   logit2[i,s] = acc[i,s] * a2 + colb[s] - c2 * (ybar[i] - colm[s])^2
// with acc = <y'_i, T'_s> (centred operands), a2 = log2(e)/sigma^2,
// c2 = log2(e) * l^2 / (2 sigma^2), colb[s] = log2(e) (-nu'_r / (2 sigma^2) + log rho[s]),
// colm[s] = m_r (mean of sub-image r(s)).
struct LogitScalars {
  float a2;
  float c2;
};

// Algorithm 2 schedule of one context kept in device memory while a batch replays its
// iteration graph.
struct DevSched {
  int t;             // EM iterations done
  int F;             // projection cadence (0 = none)
  double sigma_bm;   // current denoiser level
  double decay;      // sigma_BM <- decay * sigma_BM after each projection
};

struct Plan {
  int p1_bn = 256;          // tensor-core pass 1: shifts per tile (256 or 128)
  int p1_groups = 1;        // shift groups per observation tile in pass 1
  int p1_tiles_per_group = 1;
  int p2_gc = 1;            // cluster size (pixel chunks sharing one weight tile)
  int p2_chunk_groups = 1;  // groups of gc chunks (each recomputes the logits)
  int p2_nsplit = 1;        // observation ranges with separate M-step partial sums
  int p2_iblk_per_split = 1;
  int p2_rounds = 1;        // float32 pass 2: rounds per (shift tile, chunk group) unit
  int64_t p2_units = 1;     // float32 pass 2: (shift tile, chunk group) units
  int64_t p2_units_whole = 0;  // float32 pass 2: units dealt out whole to the clusters
  int p2_ncl = 1;           // float32 pass 2: persistent clusters
  int p2_nseg = 1;          // float32 pass 2: partial-sum segments per unit
  int nparts_c = 1;         // number of partial c / zb slices
  int nparts_z = 1;         // number of partial Z slices
  int ll_blocks = 1;        // blocks of the lse-combine kernel
  int fft_obs_per_block = 1;  // FFT form: observations per (block, phase) CTA
  int fft_blocks = 1;         // FFT form: observation blocks (pass 2: one partial each)
  int fft_p1_obs_per_block = 1;  // FFT form, pass 1 (per-observation outputs only)
  int fft_p1_blocks = 1;
  bool p2_comp = false;     // tensor-core pass 2 with the compensated M-step (bf16x3)
  bool p2_pair = false;     // tensor-core pass 2 in the pair form (2-CTA MMAs, bf16x3)
  int cap_p1_groups = 0;    // capacity of the pass-1 partial buffers (0 = unbounded)
  int cap_nsplit = 0;       // capacity of the pass-2 partial buffers (0 = unbounded)
};

}  // namespace srmra

struct srmra_ctx {
  srmra::Geom g;
  int prec = 0;
  unsigned flags = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  srmra::Plan plan;

  // --- observations (fixed for the life of the context)
  float* Yc = nullptr;     // [Npad][ldy]  centred observations y'_i = y_i - ybar_i (fp32)
  float* YcT = nullptr;    // [ldy][Npad]  the same, pixel-major (fp32 kernels)
  float* ybar = nullptr;   // [Npad]       mean of each observation
  double* yy = nullptr;    // [Npad]       ||y'_i||^2
  __nv_bfloat16* Yh = nullptr;   // [Npad][ldk] bf16(y')            (tensor-core form)
  __nv_bfloat16* Yl = nullptr;   // [Npad][ldk] bf16(y' - Yh)       (split form only)
  __half* YTf = nullptr;         // [l2][Npad]  fp16(y') pixel-major (M-step operand)
  __half* YTfl = nullptr;        // [l2][Npad]  fp16(y' - YTf) (compensated M-step only)
  __nv_bfloat16* Ah = nullptr;   // [Spad][ldk] centred templates, bf16 hi
  __nv_bfloat16* Al = nullptr;   // [Spad][ldk] bf16 lo (split form only)
  CUtensorMap tmY128, tmYl128, tmYT, tmYTl, tmA128, tmAl128, tmA256, tmAl256;
  CUtensorMap tmY64, tmYl64, tmYT128;  // pair form of pass 2 (split form only)
  void* d_inst = nullptr;           // this context's launch descriptor (tensor-core form)
  int64_t* d_ustart = nullptr;      // [4] unit prefix sums of pass 1 and pass 2
  int64_t h_ustart[4] = {0, 0, 0, 0};
  std::vector<unsigned char> h_inst;

  // --- estimate theta_t
  float* x = nullptr;      // [L*L]
  double* rho1 = nullptr;  // [L]
  double* rho2 = nullptr;  // [L]
  double sigma_bm = 1.0;
  int32_t t = 0;

  // --- per-iteration work buffers
  double* sub = nullptr;   // [2*K*K]  m_r, nu'_r
  float* colb = nullptr;   // [Spad]
  float* colm = nullptr;   // [Spad]
  float* AxT = nullptr;    // [ldy][Spad] centred templates, pixel-major (fp32 kernels)
  float* pm = nullptr;     // [p1_groups][Npad] running max (base 2)
  float* ps = nullptr;     // [p1_groups][Npad] running sum
  float* lse2 = nullptr;   // [Npad] log2 sum_s 2^{logit2}
  double* lse = nullptr;   // [Npad] per-observation log-likelihood (natural log)
  double* llpart = nullptr;// [ll_blocks]
  float* Zp = nullptr;     // [nparts_z][Spad][ldy] partial sum_i w y'_i
  float* cp = nullptr;     // [nparts_c][Spad] partial sum_i w
  float* zbp = nullptr;    // [nparts_c][Spad] partial sum_i w ybar_i
  double* cfin = nullptr;  // [2*Spad] c_s and zb_s of the last E-step
  float* bpart = nullptr;  // [fin_t_splits][K*K][l2] partial b' per lag range
  float2* Yf = nullptr;    // FFT form: [Npad][l2] FFT2(y'_i)
  float2* Xf = nullptr;    // FFT form: [K*K][l2] FFT2(x'_r), per iteration
  float2* Gp = nullptr;    // FFT form: [fft_blocks][K*K][l2] partial sum_i conj(W^) Y^'
  double* Ar = nullptr;    // [K*K] coverage per sub-image, then ZB per sub-image [K*K]
  double* dstats = nullptr;  // [3 L^2 + 1] packed E-step statistics (host transfers)
  double* ll_hist = nullptr;  // [ll_cap]
  int ll_cap = 0;
  int* status = nullptr;   // device status word
  srmra::DevSched* d_sched = nullptr;  // Algorithm 2 schedule for graph replay
  bool have_estep = false;

  int64_t launches = 0;
  int64_t device_bytes = 0;   // device memory held by this context
  bool no_cluster = false;    // force the per-chunk pass-2 kernel (SRMRA_FLAG_NO_CLUSTER)
  uint64_t wait_ns = 2000000000ull;  // limit of the kernels' bounded waits (ns)
  int test_hook = 0;          // srmra_set_wait_limit test hook (1: pass 1, 2: pass 2)
  int sched_F = 0;            // Algorithm 2 cadence used by batches with F < 0
  int dn_mode = 0;            // built-in denoiser: 0 hard, 1 soft threshold
  bool dn_spin = false;       // average over the 64 block-grid offsets
  double dn_thr = 2.7;        // threshold multiplier of sigma_BM
  double* dn_acc = nullptr;   // [64][L*L] per-offset results (cycle spinning)
  double sched_decay = 0.93303299153680741598;  // 2^{-1/10}
  std::string err;
  // per-phase timing (srmra_profile)
  bool profiling = false;
  struct Mark { int phase; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> event_pool;
  std::vector<void*> owned;  // every device buffer allocated for this context
};

namespace srmra {

// ---- k_common.cu
void launch_center_obs(srmra_ctx* c, const float* y_dev);
void launch_prep_iter(srmra_ctx* c);           // sub-image stats, column terms, templates
void launch_lse_combine(srmra_ctx* c, int groups);
void launch_finalize(srmra_ctx* c, int ll_index);  // launch_stats + launch_mstep
int stats_t_splits(const srmra_ctx* c);
void launch_stats(srmra_ctx* c);
void launch_mstep(srmra_ctx* c, const double* cfin, const float* bpart, int n_ts,
                  const double* llpart, int ll_blocks, double* rho1, double* rho2, double* Ar,
                  double* ll_out, float* x, int* status, cudaStream_t stream);
void launch_pack_stats(srmra_ctx* c, double* out);       // [c | zb | b' | LL], 3 L^2 + 1
void launch_unpack_stats(srmra_ctx* c, const double* in);
srmra_status run_estep_stats(srmra_ctx* c);  // prep, both passes, combine, launch_stats
void launch_dct_denoise(srmra_ctx* c, double sigma_bm, double thr);
void launch_dct_sched(srmra_ctx* c, double thr);  // projection from the device schedule
LogitScalars logit_scalars(const Geom& g);
cudaError_t launch_sum_f64(const double* in, int n, double* out, cudaStream_t stream);
int fin_t_splits(const Geom& g, int num_sms);

// ---- k_tc.cu (tensor-core forms)
bool tc_comp_mstep(const Geom& g, int prec, unsigned flags);
int tc_p2_key(const srmra_ctx* c);  // pass-2 launch group (cluster size; 0 = compensated)
bool tc_pair_form(const Geom& g, int prec, unsigned flags, bool comp);
void plan_tc(srmra_ctx* c, int s1 = 1, int s2 = 1);
cudaError_t tc_replan(srmra_ctx* c, int s1, int s2, int p1_bn);
cudaError_t tc_set_attributes(int prec);
cudaError_t prep_obs_tc(srmra_ctx* c);
void launch_templates_tc(srmra_ctx* c);
cudaError_t launch_pass1_tc(srmra_ctx* c);
cudaError_t launch_pass2_tc(srmra_ctx* c);
cudaError_t tc_upload_inst(srmra_ctx* c);
size_t tc_inst_bytes();
void tc_fill_inst(const srmra_ctx* c, void* host_dst);
int64_t tc_units(const srmra_ctx* c, int pass);
cudaError_t tc_launch_group(int pass, int prec, int p1_bn, const void* d_insts,
                            const int64_t* d_ustart, int n, int64_t total, int* status,
                            cudaStream_t stream, int num_sms);
// pass 2 for instances with cluster size G (G = 1: the per-chunk kernel, G = 0: the
// per-chunk kernel with the compensated M-step)
cudaError_t tc_launch_group_p2(int G, int prec, const void* d_insts, const int64_t* d_ustart,
                               int n, int64_t total, int* status, cudaStream_t stream,
                               int num_sms);

// ---- k_simt.cu (float32 form)
void plan_simt(srmra_ctx* c);
cudaError_t simt_set_attributes();

// polyphase-FFT form (k_fft.cu)
bool fft_supported(int l);
void plan_fft(srmra_ctx* c);
cudaError_t fft_set_attributes();
cudaError_t prep_obs_fft(srmra_ctx* c);
void launch_templates_fft(srmra_ctx* c);
void launch_pass1_fft(srmra_ctx* c);
cudaError_t launch_pass2_fft(srmra_ctx* c);
void launch_fin_b_fft(srmra_ctx* c);
inline bool is_tc_prec(int prec) { return prec == SRMRA_BF16 || prec == SRMRA_BF16X3; }
void launch_pass1_f32(srmra_ctx* c);
cudaError_t launch_pass2_f32(srmra_ctx* c);

}  // namespace srmra
