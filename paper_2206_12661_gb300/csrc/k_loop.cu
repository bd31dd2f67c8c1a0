// Persistent tensor-core form of the whole GSW-MTP iteration: one cooperative
// launch runs n iterations of the loop (Eq. 2 forward at the foci, the generalized
// weighting update, the adjoint of Eq. 2, phase projection), with every CTA resident
// for the whole launch and three grid-wide barriers per iteration:
//
//   forward   tiles (pupil rows x accumulator columns x split of the contraction) of
//             G = E Bx^T on tcgen05 (TMA -> 128-byte-swizzled stages -> TMEM), each
//             epilogue dotting its rows with Fy and writing a partial Theta row
//   barrier 1
//   focal     every CTA sums the partials in fixed order and runs the statistics and
//             weight update itself (identical results in every CTA, no serial tail);
//             CTA 0 alone writes w, c, the xi history and the loop state; each CTA
//             then builds its slice of pupil rows of the inverse's left operand
//             P = conj(Fy)^T diag(c) in operand format
//   barrier 2
//   inverse   tiles (pupil rows x pixel columns) of E' = P Q^T, whose epilogue writes
//             phi = arg E' and the next pupil field A exp(i phi) in operand format
//   barrier 3
//
// Warp roles (576 threads): warps 0-15 are the work warps (epilogues, focal step,
// operand build; warp w reads TMEM lanes 32*(w%4).. and column group w/4), warp 16
// issues the TMA loads, warp 17 allocates TMEM and issues the MMAs.  With 2-SM pairs
// (cta_group::2) the even CTA of a cluster issues the MMAs of 256-row tiles whose B
// operand is split between the two CTAs.  The operand pipeline runs continuously
// across units, phases and iterations; two TMEM accumulator buffers let the MMAs of
// one unit start while the epilogue of the previous one reads its accumulator.
//
// Each of the three grid barriers has its own counter in global memory (zeroed before
// every launch): a CTA arrives with a release add once its writes of the phase are
// done (after a proxy fence, since the next phase reads them with TMA) and waits with
// acquire loads until the counter reaches (iteration + 1) x CTAs.  One counter per
// barrier keeps that test exact: between two arrivals on the same counter every CTA
// waits on a barrier that all CTAs reach only after their previous arrival there, so
// no CTA can count towards iteration j + 1 before all have arrived for iteration j.
// Every wait -- mbarrier, accumulator, grid barrier -- gives up after one second,
// raises OFA_ERRBIT_TIMEOUT and leaves the loop; the CTA then frees its TMEM and exits.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>

#include "ofa_internal.cuh"
#include "ofa_math.cuh"
#include "ofa_split.cuh"
#include "umma_ptx.cuh"

using namespace ofa_ptx;

namespace {

constexpr int BM = 128;
constexpr int WORK_WARPS = 16;
constexpr int WORK_THREADS = WORK_WARPS * 32;
constexpr int WARP_TMA = WORK_WARPS;
constexpr int WARP_MMA = WORK_WARPS + 1;
constexpr int THREADS = WORK_THREADS + 64;
constexpr int KPR = 8;                 // foci per work thread in the focal step (K <= 4096)
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int TMEM_COLS = 512;         // two accumulator buffers of up to 256 columns

struct LoopArgs {
  int nx, ny, nxp, nyp, K, kp;
  int prec;
  int n_iter;
  int split;                 // forward split of the contraction
  int kb_fwd, kb_inv;        // k-blocks of the forward and inverse contractions
  int weighting;
  double threshold;          // stop test in (0, 1); anything else disables it
  const float2* fyT;         // [nyp][kp] Fy transposed, zero padded
  const float* amp;          // [ny][nx] stored amplitude
  float* phi;                // [ny][nx]
  void* e_hi;                // next pupil field, operand planes [nyp][2 nxp]
  void* e_lo;
  void* p_hi;                // inverse left operand planes [nyp][2 kp]
  void* p_lo;
  float* part;               // [tiles_m * split][2 kp] partial Theta rows
  const float* t;            // [K] normalised targets
  float* w;                  // [K] weights
  float2* c;                 // [kp] focused field (written by CTA 0, for inspection)
  double* hist;              // xi history
  OfaDevState* st;
  unsigned* bar;             // [3] grid barrier counters (after forward, focal, inverse)
  unsigned long long* clock; // nullable [6]: ns spent per phase by CTA 0 (measurement)
};

template <int KIND, int NPASS, int CG, int BNF, int BNI>
struct LCfg {
  static constexpr int EB = KIND == KIND_TF32 ? 4 : 2;
  static constexpr int RB = 128;                          // bytes of K per stage row
  static constexpr int BK = RB / EB;                      // elements of K per stage
  static constexpr int PLANES = NPASS == 3 ? 2 : 1;
  static constexpr int A_BYTES = BM * RB;
  static constexpr int BF_BYTES = (BNF / CG) * RB;        // a pair holds half of B per CTA
  static constexpr int BI_BYTES = (BNI / CG) * RB;
  static constexpr int FWD_STAGE = PLANES * (A_BYTES + BF_BYTES);
  static constexpr int INV_STAGE = PLANES * (A_BYTES + BI_BYTES);
  static constexpr int STAGE = FWD_STAGE > INV_STAGE ? FWD_STAGE : INV_STAGE;
  static constexpr int RED_BYTES = 4 * BNF * 4;           // forward cross-quarter reduction
  static constexpr int FOCAL_BYTES = 1024;                // focal reductions (<= 133 floats)
  static constexpr int BAR_BYTES = 256;
  static constexpr int FIXED = RED_BYTES + FOCAL_BYTES + BAR_BYTES + 1024;
  static constexpr int STAGES_FIT = (SMEM_LIMIT - FIXED) / STAGE;
  static constexpr int STAGES = STAGES_FIT > 8 ? 8 : STAGES_FIT;
  static_assert(STAGES >= 2, "need at least two operand stages");
  static constexpr int RED_OFF = STAGES * STAGE;
  static constexpr int FOCAL_OFF = RED_OFF + RED_BYTES;
  static constexpr int BAR_OFF = FOCAL_OFF + FOCAL_BYTES;
  static constexpr int SMEM = BAR_OFF + BAR_BYTES + 1024;  // + alignment slack
  static constexpr int UK = RB / 32;                       // MMAs per stage (32 bytes of K)
  static constexpr uint32_t IDESC_F = idesc_make(BM * CG, BNF, KIND);
  static constexpr uint32_t IDESC_I = idesc_make(BM * CG, BNI, KIND);
  static constexpr int CPW_F = BNF / 128;                  // 32-column chunks per work warp
  static constexpr int CPW_I = BNI / 128;
  static_assert(BNF % 128 == 0 && BNI % 128 == 0 && BNF <= 256 && BNI <= 256, "tile widths");
  static_assert(BNI == 128, "the inverse epilogue gives each work warp one 16-pixel chunk");
  // inverse epilogue staging: per TMEM lane quarter, phase and two field words for
  // 32 rows x 64 pixels at a pitch of 65 words, in the (then idle) operand ring
  static constexpr int PITCH = 65, ARR = 32 * PITCH;
  static_assert(STAGES * STAGE >= 4 * 3 * ARR * 4, "staging fits the operand ring");
};

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ void work_bar() { asm volatile("bar.sync 1, 512;" ::: "memory"); }
// True on every work thread if v is true on any of them (a work_bar with an OR vote).
__device__ __forceinline__ bool work_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, 512, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async;" ::: "memory");
}
__device__ __forceinline__ void grid_arrive(unsigned* bar) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Bounded wait until the grid barrier counter reaches target.
__device__ __forceinline__ bool grid_wait(const unsigned* bar, unsigned target) {
  if (ld_acquire(bar) >= target) return true;
  const uint64_t t0 = gtimer();
  while (ld_acquire(bar) < target) {
    __nanosleep(32);
    if (gtimer() - t0 > WAIT_NS) return ld_acquire(bar) >= target;
  }
  return true;
}
__device__ __forceinline__ void mbar_arrive_local(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster)
               : "memory");
}

// 16 consecutive TMEM columns of this warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Store 32 consecutive TMEM columns of this warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Sum over the warp's 32 lanes of 16 values: afterwards lane l holds the sum of
// element l % 16 (15 shuffles in a butterfly over the 16-lane halves, one across them).
__device__ __forceinline__ float warp_reduce_scatter16(float (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 8; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = upper ? v[i] : v[i + off];
      const float keep = upper ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// Sum (N values) and max (optional) over the 512 work threads; every thread gets the
// same bits (fixed-order trees).  sh: 32 * N + N floats.
template <int N>
__device__ __forceinline__ void work_sum(float (&v)[N], float* sh) {
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  work_bar();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < N; ++i) sh[i * 32 + w] = v[i];
  work_bar();
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float x = lane < WORK_WARPS ? sh[i * 32 + lane] : 0.f;
#pragma unroll
      for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) sh[32 * N + i] = x;
    }
  }
  work_bar();
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = sh[32 * N + i];
}
__device__ __forceinline__ float work_max(float v, float* sh) {
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  work_bar();
  if (lane == 0) sh[w] = v;
  work_bar();
  if (w == 0) {
    float x = lane < WORK_WARPS ? sh[lane] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) sh[32] = x;
  }
  work_bar();
  return sh[32];
}

// Forward unit u -> (pair row tile, accumulator column tile, split); inverse unit
// u -> (pair row tile, pixel column tile).  Consecutive units share a column tile,
// so the pairs running them together read its B operand from L2 in lockstep.
struct Unit {
  int mt, nt, s;
};
__device__ __forceinline__ Unit fwd_unit(int u, int mtiles, int ntiles) {
  const int per = mtiles * ntiles;
  const int r = u % per;
  return {r % mtiles, r / mtiles, u / per};
}
__device__ __forceinline__ Unit inv_unit(int u, int mtiles) { return {u % mtiles, u / mtiles, 0}; }


// The focal step of one iteration, run identically by every CTA (KP foci per work
// thread, K <= 512 KP), then this CTA's slice of pupil rows of the inverse's left
// operand P = conj(Fy)^T diag(c).  CTA 0 (writer) also records xi, w, c and the loop
// state.  Loads of several partial rows (and Fy rows) are issued together so that a
// round costs one L2 latency.  Returns true when the loop stops (threshold reached, or
// the intensities sum to zero / are not finite).
template <int KP, int NPASS>
__device__ __noinline__ bool focal_and_build(const LoopArgs& args, int n_part, bool writer,
                                             int& hcount, int j0, int it, bool thr_on,
                                             float* fsh, unsigned G,
                                             unsigned long long* clock, uint64_t* tprev) {
  constexpr int RB = KP <= 2 ? 8 : 2;          // partial (or Fy) rows per round
  const int tid = threadIdx.x;
  // parameters as restricted locals: the stores below cannot alias them
  struct {
    int K, kp, nyp, prec, weighting;
    double threshold;
    const float* __restrict__ t;
    float* __restrict__ w;
    float2* __restrict__ c;
    double* __restrict__ hist;
    OfaDevState* __restrict__ st;
    const float2* __restrict__ fyT;
    const float* __restrict__ part;
    void* __restrict__ p_hi;
    void* __restrict__ p_lo;
  } a = {args.K,   args.kp, args.nyp,  args.prec, args.weighting, args.threshold, args.t,
         args.w,   args.c,  args.hist, args.st,   args.fyT,       args.part,      args.p_hi,
         args.p_lo};
  float2 th[KP];
  float tk[KP], wk[KP], ik[KP];
  bool in[KP];
#pragma unroll
  for (int i = 0; i < KP; ++i) {
    const int k = tid + i * WORK_THREADS;
    in[i] = k < a.K;
    th[i] = make_float2(0.f, 0.f);
    tk[i] = in[i] ? __ldg(a.t + k) : 0.f;
    wk[i] = in[i] ? __ldcg(a.w + k) : 0.f;
  }
  const float2* part = reinterpret_cast<const float2*>(a.part);
  for (int p0 = 0; p0 < n_part; p0 += RB) {
    float2 v[RB][KP];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int i = 0; i < KP; ++i)
        v[r][i] = (in[i] && p0 + r < n_part)
                      ? __ldcg(part + (size_t)(p0 + r) * a.kp + tid + i * WORK_THREADS)
                      : make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < RB; ++r)          // fixed order p = 0, 1, ...
#pragma unroll
      for (int i = 0; i < KP; ++i) {
        th[i].x += v[r][i].x;
        th[i].y += v[r][i].y;
      }
  }
  float r1[1] = {0.f};
#pragma unroll
  for (int i = 0; i < KP; ++i) {
    ik[i] = th[i].x * th[i].x + th[i].y * th[i].y;
    r1[0] += ik[i];
  }
  work_sum<1>(r1, fsh);
  const float S = r1[0];
  if (!(S > 0.f) || !isfinite(S)) {
    if (writer && tid == 0) {
      atomicOr(&a.st->err, OFA_ERRBIT_NUMERIC);
      a.st->done = 1;
    }
    return true;
  }
  const float inv_s = 1.f / S;
  float r2[2] = {0.f, 0.f};
  float mx = 0.f;
  float sq[KP];
#pragma unroll
  for (int i = 0; i < KP; ++i) {
    sq[i] = sqrtf(tk[i]);
    if (!in[i]) continue;
    const float ih = ik[i] * inv_s;
    const float d = tk[i] - ih;
    r2[0] += d * d;
    r2[1] += ih * ih;
    if (a.weighting) wk[i] *= sq[i] * rsqrtf(fmaxf(ih, 1e-30f));  // w sqrt(t / Ihat)
    mx = fmaxf(mx, wk[i] * sq[i]);
  }
  work_sum<2>(r2, fsh + 40);
  mx = work_max(mx, fsh + 120);
  const float xi = 1.f - sqrtf(r2[0] / r2[1]);
  if (writer && tid == 0) {
    a.hist[hcount % OFA_HIST_CAP] = (double)xi;
    a.st->hist_count = hcount + 1;
    a.st->xi = (double)xi;
  }
  ++hcount;
  if (thr_on && (double)xi > a.threshold) {
    if (writer && tid == 0) a.st->done = 1;
    return true;
  }
  int e = 0;
  frexpf(mx, &e);
  const float scale = mx > 0.f ? exp2f((float)-e) : 1.f;
  float2 ck[KP];
#pragma unroll
  for (int i = 0; i < KP; ++i) {
    const int k = tid + i * WORK_THREADS;
    ck[i] = make_float2(0.f, 0.f);
    if (!in[i]) continue;
    const float mag = wk[i] * sq[i] * scale;
    if (ik[i] > 0.f) {
      const float inv = rsqrtf(ik[i]);
      ck[i] = make_float2(mag * th[i].x * inv, mag * th[i].y * inv);
    } else {
      ck[i] = make_float2(mag, 0.f);  // arg(0) = 0
    }
    if (writer) {
      if (a.weighting) a.w[k] = wk[i];
      a.c[k] = ck[i];
    }
  }
  if (writer && tid == 0) {
    a.st->j = j0 + it + 1;
    a.st->c_scale = scale;
  }
  if (clock) {   // phase clock: the focal step ends here
    const uint64_t tn = gtimer();
    clock[2] += tn - *tprev;
    *tprev = tn;
  }
  // this CTA's rows of P = conj(Fy)^T diag(c) in operand format
  const int rpc = (a.nyp + (int)G - 1) / (int)G;
  const int row0 = blockIdx.x * rpc, row1 = min(a.nyp, row0 + rpc);
  const bool wide = a.prec == OFA_PREC_TF32;
  for (int n0 = row0; n0 < row1; n0 += RB) {
    float2 f[RB][KP];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int i = 0; i < KP; ++i) {
        const int k = tid + i * WORK_THREADS;
        f[r][i] = (n0 + r < row1 && k < a.kp) ? __ldg(a.fyT + (size_t)(n0 + r) * a.kp + k)
                                            : make_float2(0.f, 0.f);
      }
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int i = 0; i < KP; ++i) {
        const int k = tid + i * WORK_THREADS;
        if (n0 + r >= row1 || k >= a.kp) continue;
        const size_t el = (size_t)(n0 + r) * a.kp + k;
        uint2 h, l;
        split_pack(a.prec, f[r][i].x * ck[i].x + f[r][i].y * ck[i].y,
                   f[r][i].x * ck[i].y - f[r][i].y * ck[i].x, h, l);
        if (wide) {
          reinterpret_cast<uint2*>(a.p_hi)[el] = h;
        } else {
          reinterpret_cast<uint32_t*>(a.p_hi)[el] = h.x;
          if (NPASS == 3) reinterpret_cast<uint32_t*>(a.p_lo)[el] = l.x;
        }
      }
  }
  return false;
}

// ------------------------------------------------------------------ the kernel
template <int KIND, int NPASS, int CG, int BNF, int BNI>
__global__ void __launch_bounds__(THREADS, 1)
    loop_kernel(const __grid_constant__ CUtensorMap tm_e_hi,
                const __grid_constant__ CUtensorMap tm_e_lo,
                const __grid_constant__ CUtensorMap tm_bx_hi,
                const __grid_constant__ CUtensorMap tm_bx_lo,
                const __grid_constant__ CUtensorMap tm_p_hi,
                const __grid_constant__ CUtensorMap tm_p_lo,
                const __grid_constant__ CUtensorMap tm_q_hi,
                const __grid_constant__ CUtensorMap tm_q_lo, const __grid_constant__ LoopArgs a) {
  using C = LCfg<KIND, NPASS, CG, BNF, BNI>;
  constexpr bool PAIR = CG == 2;
  // A launch without the 2-CTA clusters the pair MMAs need (or with a grid that does
  // not split into them) must not issue a single tcgen05 instruction: report it and leave.
  {
    uint32_t ncta;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
    if (ncta != (uint32_t)CG || gridDim.x % CG != 0 || gridDim.y != 1 || gridDim.z != 1) {
      if (threadIdx.x == 0) atomicOr(&a.st->err, OFA_ERRBIT_LAUNCH);
      return;
    }
  }
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base_u32 = (raw + 1023u) & ~1023u;
  uint8_t* base = smem_raw + (base_u32 - raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const uint32_t bar_full = base_u32 + C::BAR_OFF;        // [STAGES]
  const uint32_t bar_empty = bar_full + 8 * C::STAGES;    // [STAGES]
  const uint32_t bar_afull = bar_empty + 8 * C::STAGES;   // [2] accumulator complete
  const uint32_t bar_aempty = bar_afull + 16;             // [2] accumulator read (leader)
  const uint32_t bar_ringfree = bar_aempty + 16;          // work warps done with the ring
  const uint32_t bar_b3 = bar_ringfree + 8;                // grid barrier 3 passed
  const uint32_t slot_u32 = bar_b3 + 8;                    // TMEM address
  volatile uint32_t* slot = reinterpret_cast<volatile uint32_t*>(base + C::BAR_OFF +
                                                                 16 * C::STAGES + 48);
  volatile int* s_done = reinterpret_cast<volatile int*>(base + C::BAR_OFF + 16 * C::STAGES + 56);
  float* red = reinterpret_cast<float*>(base + C::RED_OFF);
  float* fsh = reinterpret_cast<float*>(base + C::FOCAL_OFF);

  const int crank = PAIR ? (int)cluster_ctarank() : 0;
  const bool leader = (crank & 1) == 0;
  const int npairs = gridDim.x / CG, pair = blockIdx.x / CG;
  const int tiles_m = a.nyp / BM;               // 128-row tiles
  const int mtiles = a.nyp / (BM * CG);         // row tiles of a pair
  const int ntf = 2 * a.kp / BNF, nti = 2 * a.nxp / BNI;
  const int units_f = mtiles * ntf * a.split, units_i = mtiles * nti;
  const int kbps = (a.kb_fwd + a.split - 1) / a.split;
  const unsigned G = gridDim.x;
  // accumulator buffers: with at most one unit per CTA in each phase every unit uses
  // columns 0.., and columns 256..511 hold the forward epilogue's Fy values, staged by
  // the work warps while the MMAs run; otherwise units alternate between two buffers
  const int nbuf = (units_f <= npairs && units_i <= npairs) ? 1 : 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_afull + 8 * b, 1);
      mbar_init(bar_aempty + 8 * b, CG * WORK_WARPS);
    }
    mbar_init(bar_ringfree, WORK_WARPS);
    mbar_init(bar_b3, 1);
    *s_done = 0;
    fence_mbar_init();
  }
  if (warp == WARP_TMA && lane == 0) {
    tmap_prefetch(&tm_e_hi);
    tmap_prefetch(&tm_bx_hi);
    tmap_prefetch(&tm_p_hi);
    tmap_prefetch(&tm_q_hi);
    if (NPASS == 3) {
      tmap_prefetch(&tm_e_lo);
      tmap_prefetch(&tm_bx_lo);
      tmap_prefetch(&tm_p_lo);
      tmap_prefetch(&tm_q_lo);
    }
  }
  if (warp == WARP_MMA) tmem_alloc<CG>(slot_u32, TMEM_COLS);
  tc_fence_before();
  if (PAIR) cluster_sync_all();
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  bool abort = false;
  // A loop that an earlier launch stopped (threshold, numeric failure) stays stopped.
  // Every CTA reads the flag before its first barrier arrival, and CTA 0 writes it only
  // after the first barrier, so all CTAs see the same value.
  const int n_iter = __ldcg(&a.st->done) ? 0 : a.n_iter;

  if (warp == WARP_TMA) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t q = 0;        // stages claimed so far (the ring position)
      uint32_t q_f0 = 0;     // ring position of the first forward stage of the coming iteration
      int prefetched = 0;    // forward stages of the coming iteration whose B is already loaded
      // claim the next ring slot for a stage of stage_bytes (A and B of every CTA of a pair)
      auto claim = [&](int stage_bytes) -> int {
        const int s = (int)(q % C::STAGES);
        if (q >= (uint32_t)C::STAGES &&
            !mbar_wait(bar_empty + 8 * s, ((q / C::STAGES) - 1) & 1))
          return -1;
        if (PAIR) {
          if (leader) mbar_expect_tx(bar_full + 8 * s, 2 * stage_bytes);
        } else {
          mbar_expect_tx(bar_full + 8 * s, stage_bytes);
        }
        ++q;
        return s;
      };
      auto full_bar = [&](int s) -> uint32_t {
        return (!PAIR || leader) ? bar_full + 8 * s : mapa_shared(bar_full + 8 * s, crank & ~1);
      };
      auto load = [&](uint32_t dst, const CUtensorMap* m, uint32_t fb, int x, int row) {
        if (PAIR) tma_load_2d_pair(dst, m, fb, x, row);
        else tma_load_2d(dst, m, fb, x, row);
      };
      auto load_a = [&](int s, const CUtensorMap* m_hi, const CUtensorMap* m_lo, int arow, int x) {
        const uint32_t st = base_u32 + s * C::STAGE, fb = full_bar(s);
        load(st, m_hi, fb, x, arow);
        if (NPASS == 3) load(st + C::A_BYTES, m_lo, fb, x, arow);
      };
      auto load_b = [&](int s, const CUtensorMap* m_hi, const CUtensorMap* m_lo, int b_bytes,
                        int brow, int x) {
        const uint32_t st = base_u32 + s * C::STAGE + C::PLANES * C::A_BYTES, fb = full_bar(s);
        load(st, m_hi, fb, x, brow);
        if (NPASS == 3) load(st + b_bytes, m_lo, fb, x, brow);
      };
      // forward stage idx of this CTA in an iteration: A (pupil field) row, B (Fx block)
      // row and contraction offset; false past the last
      auto fwd_item = [&](int idx, int& arow, int& brow, int& x) -> bool {
        for (int u = pair; u < units_f; u += npairs) {
          const Unit un = fwd_unit(u, mtiles, ntf);
          const int kb0 = un.s * kbps, nkb = min(kbps, a.kb_fwd - kb0);
          if (idx < nkb) {
            arow = (un.mt * CG + crank) * BM;
            brow = un.nt * BNF + crank * (BNF / CG);
            x = (kb0 + idx) * C::BK;
            return true;
          }
          idx -= nkb;
        }
        return false;
      };
      for (int it = 0; it < n_iter && !abort; ++it) {
        // forward: E rows come from the previous iteration's inverse (barrier 3); the B
        // halves of the first stages were loaded while waiting
        // barrier 3 of the previous iteration, awaited by a work thread (a thread with
        // bulk copies in flight polls global memory slowly)
        if (it > 0 && !mbar_wait(bar_b3, (it - 1) & 1)) { abort = true; break; }
        fence_proxy_async();
        for (int idx = 0;; ++idx) {
          int arow, brow, x;
          if (!fwd_item(idx, arow, brow, x)) break;
          int s;
          if (idx < prefetched) {
            s = (int)((q_f0 + idx) % C::STAGES);
          } else {
            s = claim(C::FWD_STAGE);
            if (s < 0) { abort = true; break; }
            load_b(s, &tm_bx_hi, &tm_bx_lo, C::BF_BYTES, brow, x);
          }
          load_a(s, &tm_e_hi, &tm_e_lo, arow, x);
        }
        prefetched = 0;
        if (abort) break;
        // inverse: P is built after the focal step (barrier 2)
        if (!grid_wait(a.bar + 1, (unsigned)(it + 1) * G)) { abort = true; break; }
        if (*s_done) break;
        fence_proxy_async();
        for (int u = pair; u < units_i && !abort; u += npairs) {
          const Unit un = inv_unit(u, mtiles);
          const int arow = (un.mt * CG + crank) * BM;
          const int brow = un.nt * BNI + crank * (BNI / CG);
          for (int kb = 0; kb < a.kb_inv; ++kb) {
            const int s = claim(C::INV_STAGE);
            if (s < 0) { abort = true; break; }
            load_b(s, &tm_q_hi, &tm_q_lo, C::BI_BYTES, brow, kb * C::BK);
            load_a(s, &tm_p_hi, &tm_p_lo, arow, kb * C::BK);
          }
        }
        if (abort) break;
        // the next forward's B (the static Fx block form) as soon as the work warps have
        // left the ring (the inverse epilogue stages its output there)
        if (it + 1 < n_iter) {
          if (!mbar_wait(bar_ringfree, it & 1)) { abort = true; break; }
          q_f0 = q;
          for (int idx = 0; idx < C::STAGES; ++idx) {
            int arow, brow, x;
            if (!fwd_item(idx, arow, brow, x)) break;
            const int s = claim(C::FWD_STAGE);
            if (s < 0) { abort = true; break; }
            load_b(s, &tm_bx_hi, &tm_bx_lo, C::BF_BYTES, brow, x);
            ++prefetched;
          }
        }
      }
      if (abort) {
        atomicOr(&a.st->err, OFA_ERRBIT_TIMEOUT);
        // copies issued but not consumed must land before the CTA may exit
        for (uint32_t k = q > (uint32_t)C::STAGES ? q - C::STAGES : 0; leader && k < q; ++k)
          if (!mbar_wait(bar_full + 8 * (k % C::STAGES), (k / C::STAGES) & 1)) break;
      }
    }
  } else if (warp == WARP_MMA) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0 && leader) {
      uint32_t q = 0, acc = 0;
      const uint16_t pair_mask = (uint16_t)(3u << (crank & ~1));
      auto run_unit = [&](int nkb, uint32_t idesc, int stage_bytes) -> bool {
        const uint32_t b = acc % nbuf, use = acc / nbuf;
        if (use >= 1 && !mbar_wait(bar_aempty + 8 * b, (use - 1) & 1)) return false;
        tc_fence_after();
        const uint32_t d = tmem + b * 256;
        const int a_bytes = C::A_BYTES;
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = (int)(q % C::STAGES);
          if (!mbar_wait(bar_full + 8 * s, (q / C::STAGES) & 1)) return false;
          tc_fence_after();
          const uint32_t st = base_u32 + s * C::STAGE;
          const uint32_t b_off = C::PLANES * a_bytes;
          const uint64_t ah = sdesc<C::RB>(st);
          const uint64_t al = sdesc<C::RB>(st + a_bytes);
          const uint64_t bh = sdesc<C::RB>(st + b_off);
          const uint64_t bl = sdesc<C::RB>(st + b_off + (stage_bytes / C::PLANES - a_bytes));
#pragma unroll
          for (int kk = 0; kk < C::UK; ++kk) {
            const uint64_t adv = (uint64_t)((kk * 32) >> 4);
            umma<KIND, CG>(d, ah + adv, bh + adv, idesc, (kb | kk) != 0);
            if (NPASS == 3) {
              umma<KIND, CG>(d, ah + adv, bl + adv, idesc, 1);
              umma<KIND, CG>(d, al + adv, bh + adv, idesc, 1);
            }
          }
          if (PAIR) umma_commit_pair(bar_empty + 8 * s, pair_mask);
          else umma_commit(bar_empty + 8 * s);
          ++q;
        }
        if (PAIR) umma_commit_pair(bar_afull + 8 * b, pair_mask);
        else umma_commit(bar_afull + 8 * b);
        ++acc;
        return true;
      };
      for (int it = 0; it < n_iter && !abort; ++it) {
        for (int u = pair; u < units_f && !abort; u += npairs) {
          const Unit un = fwd_unit(u, mtiles, ntf);
          const int kb0 = un.s * kbps, nkb = min(kbps, a.kb_fwd - kb0);
          if (!run_unit(nkb, C::IDESC_F, C::FWD_STAGE)) abort = true;
        }
        if (abort) break;
        if (!grid_wait(a.bar + 1, (unsigned)(it + 1) * G)) { abort = true; break; }
        if (*s_done) break;
        for (int u = pair; u < units_i && !abort; u += npairs)
          if (!run_unit(a.kb_inv, C::IDESC_I, C::INV_STAGE)) abort = true;
      }
      if (abort) atomicOr(&a.st->err, OFA_ERRBIT_TIMEOUT);
    }
  } else {
    // ------------------------------------------------------------ work warps
    const int tid = threadIdx.x;
    const int quarter = warp & 3, grp = warp >> 2;
    const bool writer = blockIdx.x == 0;
    const bool thr_on = a.threshold > 0.0 && a.threshold < 1.0;
    int hcount = 0, j0 = 0;
    if (writer) {
      hcount = a.st->hist_count;
      j0 = a.st->j;
    }
    uint32_t acc = 0;
    // arrive on the leader's accumulator-free barrier once this warp's TMEM reads are done
    auto release_acc = [&](uint32_t b) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (PAIR) mbar_arrive_cluster(mapa_shared(bar_aempty + 8 * b, crank & ~1));
        else mbar_arrive_local(bar_aempty + 8 * b);
      }
    };
    // phase clock of CTA 0 (ofa_profile_loop): forward epilogues done, barrier 1 passed,
    // focal step done, P rows built, barrier 2 passed, inverse epilogues done
    const bool clk = a.clock != nullptr && blockIdx.x == 0 && tid == 0;
    uint64_t tprev = clk ? gtimer() : 0;
    auto stamp = [&](int slot) {
      if (clk) {
        const uint64_t tn = gtimer();
        a.clock[slot] += tn - tprev;
        tprev = tn;
      }
    };
    for (int it = 0; it < n_iter && !abort; ++it) {
      // ---------------- forward epilogues: Theta partials of this CTA's 128 rows
      for (int u = pair; u < units_f; u += npairs) {
        const Unit un = fwd_unit(u, mtiles, ntf);
        const int m_tile = un.mt * CG + crank;
        const int n = m_tile * BM + quarter * 32 + lane;
        // Fy of this row for the warp's foci, 16 accumulator columns (8 foci) at a time:
        // from TMEM where it was staged, else from global memory
        constexpr int SUB = C::CPW_F * 2;               // 16-column sub-chunks per warp
        const float4* fr = reinterpret_cast<const float4*>(
            a.fyT + (size_t)n * a.kp + ((un.nt * BNF + grp * C::CPW_F * 32) >> 1));

        const uint32_t b = acc % nbuf, use = acc / nbuf;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const uint32_t tfy = tmem + 256 + lane_off + grp * C::CPW_F * 32;   // staged Fy
        if (nbuf == 1) {
          // Fy of this row for the warp's 32 foci into TMEM columns 256.. (the MMAs
          // write columns 0..255 meanwhile)
#pragma unroll
          for (int h = 0; h < C::CPW_F; ++h) {
            uint32_t r[32];
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) {
              const float4 f = __ldg(fr + 8 * h + qq);
              r[4 * qq] = __float_as_uint(f.x);
              r[4 * qq + 1] = __float_as_uint(f.y);
              r[4 * qq + 2] = __float_as_uint(f.z);
              r[4 * qq + 3] = __float_as_uint(f.w);
            }
            tmem_st32(tfy + h * 32, r);
          }
          tmem_wait_st();
        }
        // warp-uniform: tcgen05.ld below is a whole-warp instruction
        if (!__all_sync(0xffffffffu, mbar_wait_sleep(bar_afull + 8 * b, use & 1)))
          abort = true;
        tc_fence_after();
        const uint32_t tw = tmem + b * 256 + lane_off + grp * C::CPW_F * 32;
#pragma unroll
        for (int sc = 0; sc < SUB; ++sc) {
          float p[16];
          if (!abort) {
            float4 fy[4];
            if (nbuf == 1) {
              uint32_t fv[16];
              tmem_ld16(tfy + sc * 16, fv);
#pragma unroll
              for (int qq = 0; qq < 4; ++qq)
                fy[qq] = make_float4(__uint_as_float(fv[4 * qq]), __uint_as_float(fv[4 * qq + 1]),
                                     __uint_as_float(fv[4 * qq + 2]),
                                     __uint_as_float(fv[4 * qq + 3]));
            } else {
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) fy[qq] = __ldg(fr + 4 * sc + qq);
            }
            uint32_t v[16];
            tmem_ld16(tw + sc * 16, v);
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const float4 f = fy[qq];
              const float g0r = __uint_as_float(v[4 * qq]), g0i = __uint_as_float(v[4 * qq + 1]);
              const float g1r = __uint_as_float(v[4 * qq + 2]),
                          g1i = __uint_as_float(v[4 * qq + 3]);
              p[4 * qq] = f.x * g0r - f.y * g0i;
              p[4 * qq + 1] = f.x * g0i + f.y * g0r;
              p[4 * qq + 2] = f.z * g1r - f.w * g1i;
              p[4 * qq + 3] = f.z * g1i + f.w * g1r;
            }
          } else {
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) p[qq] = 0.f;
          }
          const float r = warp_reduce_scatter16(p);
          if (lane < 16) red[quarter * BNF + grp * C::CPW_F * 32 + sc * 16 + lane] = r;
        }
        release_acc(b);
        ++acc;
        work_bar();
        float* dst = a.part + (size_t)(un.s * tiles_m + m_tile) * 2 * a.kp + un.nt * BNF;
        for (int col = tid; col < BNF; col += WORK_THREADS)
          dst[col] = ((red[col] + red[BNF + col]) + red[2 * BNF + col]) + red[3 * BNF + col];
        work_bar();
      }
      if (work_any(abort)) {   // one decision for all work warps
        abort = true;
        break;
      }
      work_bar();
      stamp(0);
      // barrier 1: this CTA's partials are written.  The CTA barrier orders every work
      // thread's stores before thread 0's fence, so one gpu-scope fence (and the release
      // of the arrival) publishes them all; readers use TMA only after a proxy fence.
      if (tid == 0) {
        __threadfence();
        grid_arrive(a.bar);
      }

      // ---------------- focal step (every CTA, identical results)
      if (tid == 0) {
        if (!grid_wait(a.bar, (unsigned)(it + 1) * G)) *s_done = 2;
        __threadfence();
      }
      work_bar();
      stamp(1);
      if (*s_done == 2) {
        abort = true;
        break;
      }
      const bool stop = a.kp <= 2 * WORK_THREADS
                            ? focal_and_build<2, NPASS>(a, tiles_m * a.split, writer, hcount, j0, it,
                                                        thr_on, fsh, G, clk ? a.clock : nullptr,
                                                        &tprev)
                            : focal_and_build<KPR, NPASS>(a, tiles_m * a.split, writer, hcount, j0,
                                                          it, thr_on, fsh, G,
                                                          clk ? a.clock : nullptr, &tprev);
      work_bar();                        // every thread's P rows are written
      stamp(3);
      if (tid == 0) {
        *s_done = stop ? 1 : 0;
        __threadfence();
        grid_arrive(a.bar + 1);          // barrier 2: P rows written (or the loop stops)
      }
      work_bar();
      if (stop) break;

      // ---------------- inverse epilogues: phi and the next pupil field
      if (clk) grid_wait(a.bar + 1, (unsigned)(it + 1) * G);  // for the phase clock only
      stamp(4);
      for (int u = pair; u < units_i; u += npairs) {
        const Unit un = inv_unit(u, mtiles);
        // the CTA's last inverse unit: no operand loads follow before barrier 3, so the
        // ring is idle and stages the outputs for row-contiguous stores
        const bool staged = u + npairs >= units_i;
        const int m_tile = un.mt * CG + crank;
        const int nbase = m_tile * BM + quarter * 32;
        const int n = nbase + lane;
        const bool row_ok = n < a.ny;
        const uint32_t b = acc % nbuf, use = acc / nbuf;
        const int px0 = (un.nt * BNI) >> 1;      // first pixel of the tile (64 pixels)
        const int mc = px0 + grp * 16;           // first pixel of this warp's chunk
        const bool wide = a.prec == OFA_PREC_TF32;
        float av[16];
        const size_t rb = (size_t)n * a.nx + mc;
        if (((a.nx & 3) == 0) && row_ok && mc + 16 <= a.nx) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 a4 = __ldg(reinterpret_cast<const float4*>(a.amp + rb) + j);
            av[4 * j] = a4.x; av[4 * j + 1] = a4.y; av[4 * j + 2] = a4.z; av[4 * j + 3] = a4.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            av[j] = (row_ok && mc + j < a.nx) ? __ldg(a.amp + rb + j) : 0.f;
        }
        if (!__all_sync(0xffffffffu, mbar_wait_sleep(bar_afull + 8 * b, use & 1)))
          abort = true;
        tc_fence_after();
        uint32_t* sq = reinterpret_cast<uint32_t*>(base) + quarter * 3 * C::ARR;
        float* s_o = reinterpret_cast<float*>(sq);   // phase
        uint32_t* s_a = sq + C::ARR;                 // field hi (TF32: real part bits)
        uint32_t* s_b = sq + 2 * C::ARR;             // field lo (TF32: imaginary part bits)
        if (!abort) {
          uint32_t v[32];
          tmem_ld32(tmem + b * 256 + ((uint32_t)(quarter * 32) << 16) + grp * 32, v);
          float ph[16];
          uint32_t hw[16], lw[16], iw[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float re = __uint_as_float(v[2 * j]), im = __uint_as_float(v[2 * j + 1]);
            ph[j] = ofa_arg(im, re);                      // phi = arg(E'), arg(0) = 0
            float sn, cs;
            __sincosf(ph[j], &sn, &cs);
            uint2 h, l;
            split_pack(a.prec, av[j] * cs, av[j] * sn, h, l);
            hw[j] = h.x;
            iw[j] = h.y;     // TF32: imaginary part
            lw[j] = l.x;
          }
          if (staged) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int slot_i = lane * C::PITCH + grp * 16 + j;
              s_o[slot_i] = ph[j];
              s_a[slot_i] = hw[j];
              s_b[slot_i] = wide ? iw[j] : lw[j];
            }
          } else {
            if (row_ok) {
              float* pr = a.phi + rb;
              if (((a.nx & 3) == 0) && mc + 16 <= a.nx) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                  reinterpret_cast<float4*>(pr)[j] =
                      make_float4(ph[4 * j], ph[4 * j + 1], ph[4 * j + 2], ph[4 * j + 3]);
              } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                  if (mc + j < a.nx) pr[j] = ph[j];
              }
            }
            // the next pupil field over all 16 pixels (zero beyond the pupil: A = 0 there)
            const size_t e = (size_t)n * a.nxp + mc;
            if (wide) {
              uint4* dh = reinterpret_cast<uint4*>(static_cast<uint32_t*>(a.e_hi) + 2 * e);
#pragma unroll
              for (int j = 0; j < 8; ++j)
                dh[j] = make_uint4(hw[2 * j], iw[2 * j], hw[2 * j + 1], iw[2 * j + 1]);
            } else {
              uint4* dh = reinterpret_cast<uint4*>(static_cast<uint32_t*>(a.e_hi) + e);
#pragma unroll
              for (int j = 0; j < 4; ++j)
                dh[j] = make_uint4(hw[4 * j], hw[4 * j + 1], hw[4 * j + 2], hw[4 * j + 3]);
              if (NPASS == 3) {
                uint4* dl = reinterpret_cast<uint4*>(static_cast<uint32_t*>(a.e_lo) + e);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                  dl[j] = make_uint4(lw[4 * j], lw[4 * j + 1], lw[4 * j + 2], lw[4 * j + 3]);
              }
            }
          }
        }
        release_acc(b);
        ++acc;
        if (staged) {
          // the quarter's four warps have staged 32 rows x 64 pixels; each warp now
          // stores 8 whole row segments (128 consecutive bytes per warp store)
          asm volatile("bar.sync %0, 128;" ::"r"(2 + quarter) : "memory");
          if (!abort) {
#pragma unroll 2
            for (int rr = 0; rr < 8; ++rr) {
              const int row = grp * 8 + rr, gn = nbase + row;
              if (gn >= a.ny) continue;
#pragma unroll
              for (int j = 0; j < 2; ++j) {
                const int px = lane + 32 * j, gm = px0 + px;
                if (gm >= a.nx) continue;
                a.phi[(size_t)gn * a.nx + gm] = s_o[row * C::PITCH + px];
                if (!wide) {
                  const size_t e = (size_t)gn * a.nxp + gm;
                  static_cast<uint32_t*>(a.e_hi)[e] = s_a[row * C::PITCH + px];
                  if (NPASS == 3) static_cast<uint32_t*>(a.e_lo)[e] = s_b[row * C::PITCH + px];
                }
              }
              if (wide) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  const int wi = lane + 32 * j, px = wi >> 1, gm = px0 + px;
                  if (gm >= a.nx) continue;
                  static_cast<uint32_t*>(a.e_hi)[2 * ((size_t)gn * a.nxp + px0) + wi] =
                      (wi & 1) ? s_b[row * C::PITCH + px] : s_a[row * C::PITCH + px];
                }
              }
            }
          }
        }
      }
      // this warp no longer reads the ring: the next forward's operands may load
      __syncwarp();
      if (lane == 0) mbar_arrive_local(bar_ringfree);
      if (work_any(abort)) {
        abort = true;
        break;
      }
      work_bar();
      stamp(5);
      if (tid == 0) {
        __threadfence();
        grid_arrive(a.bar + 2);           // barrier 3: phi and the pupil field written
        // hand the wait to the producer (it needs it before loading the next pupil field)
        if (it + 1 < n_iter) {
          const bool ok = grid_wait(a.bar + 2, (unsigned)(it + 1) * G);
          if (ok) mbar_arrive_local(bar_b3);
          else *s_done = 2;
        }
      }
    }
    if (abort && tid == 0) atomicOr(&a.st->err, OFA_ERRBIT_TIMEOUT);
  }

  // ------------------------------------------------------------ teardown
  // After a wait gave up, copies and MMAs issued by this CTA (or, in a pair, whose
  // completion only the partner's barriers track) may still be in flight: let them
  // land (they take microseconds) before TMEM and shared memory are released.
  if (__syncthreads_or(abort)) {
    const uint64_t t0 = gtimer();
    while (gtimer() - t0 < 200000ull) __nanosleep(1000);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == WARP_MMA) {
    tc_fence_after();
    tmem_dealloc<CG>(tmem, TMEM_COLS);
  }
  // no CTA of a pair may leave while its partner can still arrive on its barriers
  if (PAIR) cluster_sync_all();
}

// ------------------------------------------------------------------ host side
template <int V>
using IC = std::integral_constant<int, V>;

// f(kind, npass, cg) for a precision and CTA group.
template <class F>
void visit_loop(int prec, int cg, F&& f) {
  auto by_cg = [&](auto kind, auto npass) {
    if (cg == 2) f(kind, npass, IC<2>{});
    else f(kind, npass, IC<1>{});
  };
  switch (prec) {
    case OFA_PREC_TF32: by_cg(IC<KIND_TF32>{}, IC<1>{}); break;
    case OFA_PREC_BF16: by_cg(IC<KIND_BF16>{}, IC<1>{}); break;
    case OFA_PREC_BF16X3: by_cg(IC<KIND_BF16>{}, IC<3>{}); break;
    case OFA_PREC_F16X3: by_cg(IC<KIND_F16>{}, IC<3>{}); break;
    default: break;
  }
}

constexpr int LOOP_BNF = 256, LOOP_BNI = 128;

#define OFA_LOOP_TYPES                                                     \
  constexpr int K_ = decltype(kind)::value, NP_ = decltype(npass)::value;  \
  constexpr int CG_ = decltype(cgc)::value;                                \
  using C = LCfg<K_, NP_, CG_, LOOP_BNF, LOOP_BNI>;                        \
  auto kern = loop_kernel<K_, NP_, CG_, LOOP_BNF, LOOP_BNI>;               \
  (void)sizeof(C)

PFN_cuTensorMapEncodeTiled_v12000 loop_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool loop_encode(CUtensorMap* m, void* ptr, int elem_bytes, uint64_t cols, uint64_t rows,
                 uint32_t box_rows, std::string& err) {
  auto fn = loop_encode_fn();
  if (fn == nullptr) {
    err = "cuTensorMapEncodeTiled is not available from the driver";
    return false;
  }
  const CUtensorMapDataType dt =
      elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * (cuuint64_t)elem_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, dt, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r);
    return false;
  }
  return true;
}

}  // namespace

bool loop_eligible(const ofa_plan* p) {
  return prec_is_tc(p->precision) && !p->sep && p->kp <= KPR * WORK_THREADS;
}

// Configuration, tensor maps, shared-memory opt-in and the co-residency check of the
// fused loop kernel for a plan (cg = 0: 2-SM pairs when the row tiles pair up; split
// = 0: as many forward units as CTA pairs allow, at most 4).
bool loop_prepare(ofa_plan* p, int cg, int split, std::string& err) {
  LoopOperands& L = p->loop;
  L.ready = false;
  if (!loop_eligible(p)) {
    err = "the fused loop needs a tensor-core precision, the general form and K <= 4096";
    return false;
  }
  const TcOperands& t = p->tc;
  const int tiles_m = p->nyp / BM;
  if (cg == 0) cg = tiles_m % 2 == 0 ? 2 : 1;
  if (cg != 1 && cg != 2) { err = "loop CTA group must be 1 or 2"; return false; }
  if (cg == 2 && tiles_m % 2 != 0) {
    err = "2-SM pairs need an even number of 128-row tiles";
    return false;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  bool ok = true;
  int smem = 0, max_blocks = 0;
  visit_loop(p->precision, cg, [&](auto kind, auto npass, auto cgc) {
    OFA_LOOP_TYPES;
    smem = C::SMEM;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM);
    if (e != cudaSuccess) {
      err = std::string("loop kernel shared memory: ") + cudaGetErrorString(e);
      ok = false;
      return;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, C::SMEM);
    if (e != cudaSuccess || per_sm < 1) {
      err = "loop kernel does not fit an SM";
      ok = false;
      return;
    }
    max_blocks = per_sm * sms;
    if (CG_ == 2) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[2];
      cfg.gridDim = dim3(max_blocks);
      cfg.blockDim = dim3(THREADS);
      cfg.dynamicSmemBytes = C::SMEM;
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 2;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      at[1].id = cudaLaunchAttributeCooperative;
      at[1].val.cooperative = 1;
      cfg.attrs = at;
      cfg.numAttrs = 2;
      int clusters = 0;
      e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
      if (e != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        err = "no 2-CTA cluster of the loop kernel fits";
        ok = false;
        return;
      }
      max_blocks = std::min(max_blocks, 2 * clusters);
    }
  });
  if (!ok) return false;
  const int G = max_blocks - max_blocks % cg;
  const int npairs = G / cg;
  const int mtiles = p->nyp / (BM * cg);
  const int ntf = 2 * p->kp / LOOP_BNF;
  const int kb_fwd = (2 * p->nxp * t.elem_bytes) / 128;
  if (split == 0) {
    split = std::max(1, std::min(4, npairs / std::max(1, mtiles * ntf)));
    while (split > 1 && kb_fwd / split < 2) --split;
  }
  if (split < 1 || split > 4 || kb_fwd < split) {
    err = "loop split must be 1..4 and at most the forward k-blocks";
    return false;
  }
  if (tiles_m * split > tiles_m * 8) { err = "loop split beyond the partial buffer"; return false; }
  L.cg = cg;
  L.split = split;
  L.grid = G;
  L.smem = smem;
  L.kb_fwd = kb_fwd;
  L.kb_inv = (2 * p->kp * t.elem_bytes) / 128;
  const int eb = t.elem_bytes;
  const uint64_t e_cols = 2 * (uint64_t)p->nxp, k_cols = 2 * (uint64_t)p->kp;
  ok = loop_encode(&L.tm_e_hi, t.e_hi, eb, e_cols, p->nyp, BM, err) &&
       loop_encode(&L.tm_bx_hi, t.bx_hi, eb, e_cols, k_cols, LOOP_BNF / cg, err) &&
       loop_encode(&L.tm_p_hi, t.p_hi, eb, k_cols, p->nyp, BM, err) &&
       loop_encode(&L.tm_q_hi, t.q_hi, eb, k_cols, e_cols, LOOP_BNI / cg, err);
  if (ok && t.npass == 3) {
    ok = loop_encode(&L.tm_e_lo, t.e_lo, eb, e_cols, p->nyp, BM, err) &&
         loop_encode(&L.tm_bx_lo, t.bx_lo, eb, e_cols, k_cols, LOOP_BNF / cg, err) &&
         loop_encode(&L.tm_p_lo, t.p_lo, eb, k_cols, p->nyp, BM, err) &&
         loop_encode(&L.tm_q_lo, t.q_lo, eb, k_cols, e_cols, LOOP_BNI / cg, err);
  } else if (ok) {
    L.tm_e_lo = L.tm_e_hi;
    L.tm_bx_lo = L.tm_bx_hi;
    L.tm_p_lo = L.tm_p_hi;
    L.tm_q_lo = L.tm_q_hi;
  }
  if (!ok) return false;
  L.ready = true;
  return true;
}

// n_iter iterations of the loop in one cooperative launch on stream s (the barrier
// counters are zeroed first).  threshold in (0, 1) stops the loop as the multi-kernel
// form does; the launch leaves j, the history, w and the done flag in the plan state.
cudaError_t launch_loop(ofa_plan* p, int n_iter, double threshold, cudaStream_t s,
                        unsigned long long* clock) {
  const LoopOperands& L = p->loop;
  if (!L.ready || n_iter <= 0) return cudaSuccess;
  // a barrier counter reaches iterations x CTAs per launch: keep it in 32 bits
  constexpr int CHUNK = 1 << 20;
  if (n_iter > CHUNK) {
    for (int left = n_iter; left > 0; left -= CHUNK) {
      cudaError_t e = launch_loop(p, std::min(left, CHUNK), threshold, s, clock);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t e = cudaMemsetAsync(p->loop_bar, 0, 3 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  LoopArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nx = p->nx; a.ny = p->ny; a.nxp = p->nxp; a.nyp = p->nyp; a.K = p->K; a.kp = p->kp;
  a.prec = p->precision;
  a.n_iter = n_iter;
  a.split = L.split;
  a.kb_fwd = L.kb_fwd;
  a.kb_inv = L.kb_inv;
  a.weighting = p->weighting;
  a.threshold = threshold;
  a.fyT = p->fyT;
  a.amp = p->amp;
  a.phi = p->phi;
  a.e_hi = p->tc.e_hi; a.e_lo = p->tc.e_lo;
  a.p_hi = p->tc.p_hi; a.p_lo = p->tc.p_lo;
  a.part = reinterpret_cast<float*>(p->part);
  a.t = p->t;
  a.w = p->w;
  a.c = p->c;
  a.hist = p->hist;
  a.st = p->st;
  a.bar = p->loop_bar;
  a.clock = clock;
  visit_loop(p->precision, L.cg, [&](auto kind, auto npass, auto cgc) {
    OFA_LOOP_TYPES;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[2];
    cfg.gridDim = dim3(L.grid);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = CG_;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = CG_ == 2 ? 2 : 1;
    e = cudaLaunchKernelEx(&cfg, kern, L.tm_e_hi, L.tm_e_lo, L.tm_bx_hi, L.tm_bx_lo, L.tm_p_hi,
                           L.tm_p_lo, L.tm_q_hi, L.tm_q_lo, a);
  });
  return e;
}
