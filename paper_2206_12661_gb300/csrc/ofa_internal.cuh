// Internal declarations shared by the CUDA translation units of libofa.
//
// Data layout in device memory (rows along y, row-major, complex = interleaved
// float pairs):
//   phi, amp        [ny][nx] float32                 CGH phi and amplitude A
//   fx, fy          [K][nx], [K][ny] complex float32 DFT rows of Eq. 2 at the foci
//   fyT             [nyp][kp] complex float32         Fy transposed, zero padded
//   tensor-core operands (16-bit hi/lo planes, or one float32 plane for TF32):
//   e_pl            [nyp][2*nxp]   E = A exp(i phi), re/im interleaved along m
//   bx_pl           [2*kp][2*nxp]  real block form of Fx for the forward product
//   p_pl            [nyp][2*kp]    conj(Fy)^T diag(c), rebuilt every iteration
//   q_pl            [2*nxp][2*kp]  real block form of conj(Fx) for the inverse
// nxp, nyp, kp are the sizes rounded up to whole tensor-core tiles; the
// padding is zero and stays zero.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ofa.h"

#define OFA_HIST_CAP 65536
#define OFA_ERRBIT_TIMEOUT 1
#define OFA_ERRBIT_NUMERIC 2
#define OFA_ERRBIT_LAUNCH 4   // a kernel found its launch shape not the one it was built for

// Loop state and control words that live in device memory.
struct OfaDevState {
  int j;              // completed iterations
  int done;           // threshold reached: the remaining kernels of a launch skip
  int err;            // OFA_ERRBIT_* raised by kernels
  int hist_count;     // xi values recorded so far
  double threshold;   // stop test of Algorithm 1 (<= 0 or >= 1: disabled)
  double xi;          // statistics of the latest forward
  double uniformity;
  double sum_i;
  double energy_fraction;
  float c_scale;      // power-of-two factor applied to c this iteration
  float adam_step_size;   // lr / (1 - b1^t) of the latest ofa_adam_step
  float adam_bc2_sqrt;    // sqrt(1 - b2^t) of the latest ofa_adam_step
  int amp_exp;            // plan set-up: the amplitude is stored scaled by 2^-amp_exp
  double amp_max;         // plan set-up: peak and energy of the amplitude as given
  double amp_energy;
  int amp_bad;            // plan set-up: a value was negative, infinite or NaN
  int pad_;
};

struct TcOperands {
  int elem_bytes = 0;      // 2 (fp16 / bf16) or 4 (tf32)
  int npass = 1;           // 1 or 3 (hi*hi + hi*lo + lo*hi)
  void* e_hi = nullptr; void* e_lo = nullptr;
  void* bx_hi = nullptr; void* bx_lo = nullptr;
  void* p_hi = nullptr; void* p_lo = nullptr;
  void* q_hi = nullptr; void* q_lo = nullptr;
  CUtensorMap tm_e_hi, tm_e_lo, tm_bx_hi, tm_bx_lo, tm_p_hi, tm_p_lo, tm_q_hi, tm_q_lo;
  int fwd_bn = 256, fwd_split = 1, bwd_bn = 256;
  int fwd_rb = 128, bwd_rb = 128;                          // operand row bytes per stage
  int fwd_cg = 1, bwd_cg = 1;                              // 2 = 2-SM MMA pairs
  int kp = 0;   // padded focus dimension of the planes: K_p, or U_x rounded up (separable)
};

// Fused loop kernel (all of an iteration in one persistent cooperative launch):
// its configuration and tensor maps over the plan's operand planes.
struct LoopOperands {
  bool ready = false;
  int cg = 1, split = 1;       // CTA group (2 = 2-SM pairs), forward split of the contraction
  int grid = 0, smem = 0;      // CTAs (all resident), dynamic shared memory per CTA
  int kb_fwd = 0, kb_inv = 0;  // k-blocks of the two contractions
  CUtensorMap tm_e_hi, tm_e_lo, tm_bx_hi, tm_bx_lo, tm_p_hi, tm_p_lo, tm_q_hi, tm_q_lo;
};

// FP32 form scratch: the inverse's transposed operands and the forward's
// contraction-split workspace (each part writes its per-focus partial dots; the
// last part to arrive at a tile, by arrival counter, sums them in fixed order).
struct SimtWork {
  // pitch simt_ldk(contraction length), zero padded:
  float2* p32 = nullptr;      // [ny][ldk] conj(Fy[k,n]) c_k
  float2* fxT = nullptr;      // [nx][ldk] conj(Fx)^T (separable: of the first inverse product)
  float2* fyT = nullptr;      // [ny][ldk] Fy^T (separable form: Fyu^T)
  float2* fws = nullptr;      // forward: [fwd_tiles][parts][64] partial per-focus dots
  unsigned* cnt = nullptr;    // forward: [fwd_tiles + column tiles + 1] arrival counters
};

struct ofa_plan {
  int device = 0;
  cudaStream_t stream = nullptr;       // stream the plan's work is enqueued on
  cudaStream_t cap_stream = nullptr;   // private stream used only for graph capture
  bool own_stream = false;
  int nx = 0, ny = 0, K = 0, precision = 0, weighting = 1;
  int row0 = 0, ny_total = 0;          // row shard: rows [row0, row0 + ny) of ny_total
  double px = 0, py = 0, lambda = 0, focal = 0;
  int nxp = 0, nyp = 0, kp = 0;        // padded sizes (tensor-core tiles)
  int amp_exp = 0;                     // stored A = user A * 2^-amp_exp
  double amp_energy = 0;               // sum of user A^2

  double* focus_xy = nullptr;          // [K][2]
  double* focus_z = nullptr;           // [K] axial offsets, or NULL (2D)
  float* t = nullptr;                  // [K] normalised targets
  float* amp = nullptr;                // [ny][nx]
  float* phi = nullptr;                // [ny][nx]
  float* w = nullptr;                  // [K]
  float2* fx = nullptr;                // [K][nx]
  float2* fy = nullptr;                // [K][ny]
  float2* fyT = nullptr;               // [nyp][kp]
  float2* part = nullptr;              // [n_part][kp] per-tile partial Theta
  int n_part = 0;
  float2* theta = nullptr;             // [K]
  float* inten = nullptr;              // [K]
  float2* c = nullptr;                 // [kp] focused field (scaled), zero padded
  double* hist = nullptr;              // [OFA_HIST_CAP]
  unsigned int* counters = nullptr;    // [kp / 64 + 1] arrival counters of the fused forward
  OfaDevState* st = nullptr;
  OfaDevState* st_host = nullptr;      // pinned mirror for readback
  float* scratch_phi = nullptr;        // for ofa_forward / ofa_adjoint on the tensor path
  float2* e32 = nullptr;               // FP32 form: pupil field A exp(i phi) [ny][nx]
  float2* e32_aux = nullptr;           // FP32 form: field of an external phase
  SimtWork simt;                       // FP32 form: inverse operand and split workspaces
  float* meas = nullptr;               // [K] captured intensities (camera in the loop)
  // separable grid form (sep): products through the ux distinct x and uy distinct y
  bool sep = false;
  int ux = 0, uy = 0, sep_parts = 1;
  float2* fxu = nullptr;               // [ux][nx] DFT rows of the distinct x
  float2* fyu = nullptr;               // [uy][ny] DFT rows of the distinct y
  float2* gt = nullptr;                // [ux][ny] first forward product, transposed
  float2* tconj = nullptr;             // [uy][nx] first inverse product, conjugated
  float2* ones = nullptr;              // [uy] unit weights of the second inverse product
  int2* ixy = nullptr;                 // [K] (ix, iy) of each focus
  bool sep_fast = false;               // the three-launch separable iteration (k_sep.cu)
  bool sep_loop = false;               // the separable form's persistent loop (k_sep.cu)
  bool sep_tc = false;                 // the separable form's iteration on the tensor cores
  int sep_loop_grid = 0;               // its blocks
  int sm_count = 0;
  int* row_ptr = nullptr;              // [uy + 1] foci of each grid row ...
  int* row_foci = nullptr;             // [K] ... in increasing ix order
  int* sep_gridk = nullptr;            // [uy][ux] focus at each grid point, or -1
  float* sep_wprev = nullptr;          // [K] weights before the focal step (tensor-core form)
  TcOperands tc;
  TcOperands tc_aux;                   // E planes of an external phase (forward/adjoint)
  LoopOperands loop;                   // fused loop kernel (tensor-core forms, K <= 4096)
  int loop_mode = -1;                  // ofa_options.fused_loop
  unsigned* loop_bar = nullptr;        // its three grid barrier counters
  bool aux_ready = false;

  cudaGraphExec_t chunk_exec = nullptr;
  cudaGraphExec_t one_exec = nullptr;
  int chunk_iters = 16;

  void* arena = nullptr;               // one allocation holding the buffers above
  size_t arena_bytes = 0;
  std::vector<void**> arena_slots;     // the pointers carved out of it
  double* sep_coord = nullptr;         // separable form: distinct coordinates (set-up)
  double* amp_part = nullptr;          // [3 AMP_STAT_BLOCKS] amplitude statistics (set-up)
  unsigned* amp_count = nullptr;       // their arrival counter

  std::string last_error;
};

// ---------------------------------------------------------------- host helpers
ofa_status ofa_fail(ofa_plan* p, ofa_status s, const std::string& msg);
ofa_status ofa_cuda_check(ofa_plan* p, cudaError_t e, const char* what);
void ofa_set_thread_error(const std::string& msg);

// ---------------------------------------------------------------- kernels (k_gen.cu)
// origin: index of the optical axis along the sampled coordinate ((n - 1) / 2 for a
// whole pupil; a row shard passes the whole pupil's axis relative to its first row);
// 2 origin must be an integer.
void launch_dft_rows(const double* focus_xy, const double* focus_z, int coord, int K, int n,
                     double pitch, double origin, double lam_f, double lam_f2, float2* out,
                     cudaStream_t s);
// rows [row0, row0 + ny) of the default amplitude / phase of a pupil of ny_total rows
void launch_default_amplitude(float* amp, int nx, int ny, int row0, int ny_total, double px,
                              double py, double waist_frac, cudaStream_t s);
void launch_default_phase(float* phi, int nx, int ny, int row0, uint64_t seed, cudaStream_t s);
// Amplitude statistics of plan set-up: peak, energy, validity and the power-of-two
// exponent of the peak into st (amp_*); part holds 3 AMP_STAT_BLOCKS doubles, count
// one zeroed word (left zero).  launch_scale_pow2 then scales by 2^-amp_exp.
constexpr int AMP_STAT_BLOCKS = 1024;
void launch_amp_stats(const float* amp, size_t n, double* part, unsigned* count,
                      OfaDevState* st, cudaStream_t s);
void launch_scale_pow2(float* x, size_t n, const OfaDevState* st, cudaStream_t s);
// dst [nyp][kp] = src [K][ny] transposed (conjugated when conj), zero padded
void launch_transpose_fy(const float2* fy, int K, int ny, int kp, int nyp, float2* fyT,
                         cudaStream_t s, bool conj = false);
// Build the real block forms of Fx (forward, conj=0) or conj(Fx) (inverse, conj=1).
void launch_pack_fx(const float2* fx, int K, int nx, int kp, int nxp, int inverse,
                    int prec, void* hi, void* lo, cudaStream_t s);
void launch_field_planes(const float* phi, const float* amp, int nx, int ny, int nxp,
                         int prec, void* hi, void* lo, cudaStream_t s);

// ---------------------------------------------------------------- kernels (k_simt.cu)
void launch_field_f32(const float* phi, const float* amp, int nx, int ny, float2* e,
                      cudaStream_t s);
// Element counts of the SimtWork buffers for a plan (rows = the longest inverse
// contraction the plan runs, K or the separable form's uy).
// The focal step's operands for a kernel that runs it in its last block (on != 0);
// counter: the arrival counters that kernel uses (zero between launches).
struct FocalTail {
  const float* t;
  float* w;
  float2* c;
  double* hist;
  OfaDevState* st;
  int weighting;
  unsigned* counter;
  int on;
};

struct SimtSizes {
  size_t p32, fxT, fyT, fws, cnt;
  int fwd_tiles;
};
SimtSizes simt_sizes(int nx, int ny, int K, int rows);
int simt_ldk(int K);   // row pitch of the transposed FP32 inverse operands

// With f (f->on), the forward also sums the partial rows into Theta (row 0) and runs
// the focal step in its last arriving block when simt_fwd_fuses_focal(K); otherwise
// Theta is left as simt_fwd_tiles(ny) partial rows for launch_focal.
bool simt_fwd_fuses_focal(int K);
void launch_fwd_simt(const float2* e32, const float2* fx, const float2* fy, int nx, int ny, int K,
                     int kp, float2* part, const int* done, const SimtWork& w, cudaStream_t s,
                     const FocalTail* f = nullptr);
int simt_fwd_tiles(int ny);   // partial Theta rows the forward writes
// The inverse's left operand w.p32 = conj(fyT) c (the FP32 counterpart of build_p).
void launch_scale_conj(const float2* c, const float2* fyT, int ny, int K, float2* pT,
                       const int* done, cudaStream_t s);
// The inverse product alone, from w.p32 and fxT.
void launch_bwd_simt_product(const float2* fxT, int nx, int ny, int K, const float* amp,
                             float* phi, float2* e32, const int* done, const SimtWork& w,
                             cudaStream_t s);
// Inverse product from the transposed operands fxT = conj(Fx)^T [nx][ldk], fyT = Fy^T [ny][ldk]
// (launch_scale_conj, then launch_bwd_simt_product).
void launch_bwd_simt(const float2* c, const float2* fxT, const float2* fyT, int nx, int ny, int K,
                     const float* amp, float* phi, float2* e32, const int* done,
                     const SimtWork& w, cudaStream_t s);
// Separable grid form (foci on a grid of ux distinct x and uy distinct y values):
// gt[ix][n] = sum_m E[n][m] Fxu[ix][m]; Theta_k = sum_n Fyu[iy_k][n] gt[ix_k][n];
// tconj[iy][m] = conj(sum_{k in row iy} c_k conj(Fxu[ix_k][m])).
// The first forward product is split over `parts` contraction slices (enough blocks
// to fill the SMs when ux is small); gt holds [parts][ux][ny].
int sep_parts(int nx, int ny, int ux, int sms);
void launch_sep_forward(const float2* e32, const float2* fxu, int nx, int ny, int ux, int parts,
                        float2* gt, cudaStream_t s);
void launch_sep_theta(float2* gt, const float2* fyu, const int2* ixy, int K, int ny, int ux,
                      int parts, float2* part, cudaStream_t s);
void launch_sep_t(const float2* c, const float2* fxu, const int2* ixy, const int* row_ptr,
                  const int* row_foci, int uy, int nx, float2* tconj, cudaStream_t s);
// ---------------------------------------------------------------- kernels (k_sep.cu)
// The separable iteration in three launches: partial Theta rows of blocks of pupil rows,
// their fixed-order sum (Theta written over partial row 0) with the focal step in the
// last block (focal != 0), and the inverse with C gathered from c through gridk
// ([uy][ux] focus index or -1) and T formed per tile.
int sep_fwd_blocks(int ny, int sms);
size_t sep_fwd_smem(int ny, int ux, int uy, int sms);
size_t sep_inv_smem(int ux, int uy);
bool sep_fast_shape(int nx, int uy);
size_t sep_smem_limit();
cudaError_t sep_prepare();
// With f.on the forward runs the focal step itself when sep_fwd_fuses_focal (small
// K); otherwise launch_sep_sum_focal follows it.
bool sep_fwd_fuses_focal(int ny, int K, int sms);
void launch_sep_fwd(const float2* e32, const float2* fxu, const float2* fyu, const int2* ixy,
                    int nx, int ny, int ux, int uy, int K, int kp, int sms, float2* part,
                    const FocalTail& f, const int* done, cudaStream_t s);
void launch_sep_sum_focal(const float2* part, int nb, int K, int kp, float2* theta, int focal,
                          const float* t, float* w, float2* c, double* hist, OfaDevState* st,
                          int weighting, unsigned* counter, const int* done, cudaStream_t s);
void launch_sep_inverse(const float2* c, const int* gridk, const float2* fxu, const float2* fyu,
                        const float* amp, int nx, int ny, int ux, int uy, float* phi,
                        float2* e32, const int* done, cudaStream_t s);
// The persistent separable loop (K <= 2560): whether the shape fits (shared memory,
// one block per SM for the forward's row blocks; grid and smem on output), the kernel
// attributes and the blocks per SM that can be resident, and n_iter iterations in
// cooperative launches on s (threshold as in ofa_iterate).
bool sep_loop_shape(int nx, int ny, int ux, int uy, int K, int sms, size_t* smem, int* grid);
cudaError_t sep_loop_prepare(int ny, int sms, int* resident);
cudaError_t launch_sep_loop(ofa_plan* p, int n_iter, double threshold, cudaStream_t s);
void launch_grad_simt(const float2* c, const float2* fxT, const float2* fyT, int nx, int ny, int K,
                      const float* phi, const float* amp, float amp_factor,
                      const OfaDevState* st, float* grad, const SimtWork& w, cudaStream_t s);

// ---------------------------------------------------------------- kernels (k_focal.cu)
// mode 0: loop iteration (record xi, threshold test, weight update, c)
// mode 1: statistics only (xi, uniformity, sums into st)
// mode 2: forward output only (theta, intensity to caller buffers, user scale)
void launch_focal(const float2* part, int n_part, int kp, int K, const float* t, float* w,
                  float2* theta, float* inten, float2* c, double* hist, OfaDevState* st,
                  int mode, int weighting, float out_scale, double energy, cudaStream_t s);
void launch_focal_measured(const float2* part, int n_part, int kp, int K, const float* t,
                           float* w, float2* theta, float2* c, double* hist, OfaDevState* st,
                           int weighting, const float* meas, cudaStream_t s);
void launch_control(OfaDevState* st, double threshold, int reset_done, cudaStream_t s);
void launch_set_j(OfaDevState* st, int j, int reset_hist, cudaStream_t s);
void launch_grad_c(const float2* theta, const float* g, int K, int kp, float in_scale,
                   float2* c, OfaDevState* st, cudaStream_t s);
void launch_build_p(const float2* fyT, const float2* c, const int* done, int nyp, int kp,
                    int prec, void* hi, void* lo, cudaStream_t s);
// Separable grid form on the tensor cores: the focal step of the loop on theta [K]
// (the weights read from wprev, the new ones written to w) and the inverse's left
// operand U[n][ix] = sum_iy conj(Fyu[iy][n]) C[iy][ix], C the grid of the new c_k, into
// operand planes [nyp][2 kpad], in one launch; sep_focal_u_fits: the grid and the foci
// this launch covers, sep_focal_u_prepare: its shared-memory opt-in (once per process).
bool sep_focal_u_fits(int ux, int uy, int K);
cudaError_t sep_focal_u_prepare();
void launch_sep_focal_u(const float2* theta, const float* t, const float* wprev, float* w,
                        float2* c, double* hist, OfaDevState* st, int weighting, const int2* ixy,
                        int K, const float2* fyu, const int* done, int ny, int ux, int uy,
                        int kpad, int prec, void* hi, void* lo, cudaStream_t s);
constexpr int SEP_TC_MAX_UX = 128, SEP_TC_MAX_UY = 128, SEP_TC_MAX_PARTS = 16;
// Separable form on the tensor cores: Theta_k = T[iy_k][ix_k] with T = Fyu G from the
// forward's contraction parts gt [parts][ux][ny] (parts <= 16, summed in fixed order),
// into theta [K]; the blocks also copy w [K] to wprev (nullable) for the focal step.
void launch_sep_tc_theta(const float2* gt, int parts, const float2* fyu, const int* gridk, int ny,
                         int ux, int uy, int K, float2* theta, const float* w, float* wprev,
                         const int* done, cudaStream_t s);
void launch_sep_u_planes(const float2* cgrid, const float2* fyu, const int* done, int ny, int ux,
                         int uy, int kpad, int prec, void* hi, void* lo, cudaStream_t s);
// Intensity loss sum (I/S - t)^2 of Theta, its gradient g = dL/dI folded into
// c = g Theta (scaled; st->c_scale), loss_hist[*step] = L when the index lies in
// [0, loss_cap) (step, loss_hist nullable).
void launch_loss_grad_c(const float2* theta, const float* t, int K, int kp, float2* c,
                        OfaDevState* st, float* loss_hist, int loss_cap, const int* step,
                        cudaStream_t s);
// Adam update of n parameters: the device step counter is advanced first and the
// bias corrections for it are kept in st (adam_step_size, adam_bc2_sqrt).
void launch_adam(float* x, const float* g, float* m, float* v, int* step, OfaDevState* st,
                 size_t n, float lr, float b1, float b2, float eps, cudaStream_t s);

// ---------------------------------------------------------------- kernels (k_umma.cu)
cudaError_t tc_prepare(int prec);
// Time the candidate shapes of both products on scratch outputs and keep the
// fastest in t (cached per device, size and precision for the process).
bool tc_autotune(ofa_plan* p, TcOperands& t, std::string& err);
bool tc_encode_maps(ofa_plan* p, TcOperands& t, std::string& err);
// Whether a kernel configuration (tile widths in accumulator columns 128 | 256,
// forward split-K 1 | 2 | 4, CTA groups 1 | 2) can run this plan's sizes.
bool tc_config_valid(const ofa_plan* p, const TcOperands& t, int fwd_bn, int fwd_split,
                     int fwd_cg, int bwd_bn, int bwd_cg);
// One thread waits, with the bounded wait of the tensor-core kernels, on an mbarrier
// nothing arrives at; it sets OFA_ERRBIT_TIMEOUT in st->err when the wait gives up.
void launch_selftest_wait(OfaDevState* st, cudaStream_t s);
// fuse_focal: the last CTA runs the focal step of the loop (mode 0) on the final Theta.
void launch_fwd_tc(ofa_plan* p, const TcOperands& t, const int* done, cudaStream_t s,
                   bool fuse_focal);
// Separable grid form: G = E Fxu^T per contraction part into p->gt [split][ux][ny].
void launch_fwd_sep_tc(ofa_plan* p, const TcOperands& t, const int* done, cudaStream_t s);
void launch_bwd_tc(ofa_plan* p, const TcOperands& t, const int* done, cudaStream_t s);
void launch_grad_tc(ofa_plan* p, const TcOperands& t, const float* phi, float scale,
                    float* grad, cudaStream_t s);

// ---------------------------------------------------------------- kernels (k_loop.cu)
// Whether the fused loop kernel can run this plan (tensor-core form, general form,
// K <= 4096); loop_prepare picks its configuration (cg, split: 0 = automatic),
// encodes its tensor maps and checks co-residency; launch_loop runs n iterations
// in one cooperative launch.
bool loop_eligible(const ofa_plan* p);
bool loop_prepare(ofa_plan* p, int cg, int split, std::string& err);
// clock (nullable, device [6]): accumulates the ns CTA 0 spends per phase.
cudaError_t launch_loop(ofa_plan* p, int n_iter, double threshold, cudaStream_t s,
                        unsigned long long* clock = nullptr);

// Batched holograms on the tensor-core path: one grouped launch per product over
// the tiles of every plan (same precision), the inverse operand build grouped too.
struct BpGroupItem {
  const float2* fyT;
  const float2* c;
  void* hi;
  void* lo;
  int kp;
  int pad_;
};
void launch_build_p_group(const BpGroupItem* items, const int4* chunks, int n_chunks, int prec,
                          cudaStream_t s);
struct TcBatch;
bool tc_batch_create(ofa_plan* const* plans, int count, cudaStream_t s, TcBatch** out,
                     std::string& err);
void tc_batch_enqueue_iteration(const TcBatch* b, cudaStream_t s);
void tc_batch_config(const TcBatch* b, int* fwd_bn, int* bwd_bn);
void tc_batch_destroy(TcBatch* b);

inline bool prec_is_tc(int prec) { return prec != OFA_PREC_FP32; }
// Rows of forward partials [n_part][kp] complex the focal step sums.
inline int fwd_n_part(int nyp, const TcOperands& t) { return (nyp / 128) * t.fwd_split; }
inline int prec_elem_bytes(int prec) { return prec == OFA_PREC_TF32 ? 4 : 2; }
inline int prec_npass(int prec) {
  return (prec == OFA_PREC_BF16X3 || prec == OFA_PREC_F16X3) ? 3 : 1;
}
inline int round_up(int a, int b) { return (a + b - 1) / b * b; }
