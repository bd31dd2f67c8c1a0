// Tensor-core form of the two MTP products (kernels (b) and (d)) for sm_103a:
// TMA (cp.async.bulk.tensor) stages 128-byte-swizzled operand tiles into
// shared memory, one thread issues tcgen05.mma into a TMEM accumulator, and
// four epilogue warps read it back with tcgen05.ld.
//
// A complex product is one real GEMM over interleaved (re, im) pairs:
//   forward  G_r[n][2k+h]  = sum_i E_r[n][i]  Bx[2k+h][i]   (i = 2m + g)
//   inverse  E'_r[n][2m+h] = sum_i P_r[n][i]  Q[2m+h][i]    (i = 2k + g)
// with Bx and Q the real block forms of Fx and conj(Fx) built once per plan
// and P = conj(Fy)^T diag(c) rebuilt every iteration (4 real MACs = 8 flops
// per complex MAC, no redundant work).  Both operands are K-major.
//
// Split forms issue three MMAs per k-step (hi*hi + hi*lo + lo*hi) into the
// same FP32 accumulator.
//
// Epilogues (fused, no intermediate goes to global memory):
//   FWD   Theta partial of the tile: sum over its 128 rows n of Fy[k,n] G[n,k]
//         (warp-shuffle reduce-scatter, then a fixed-order sum of four warps)
//   BWD   phi = arg(E') and the next pupil field A exp(i phi) in operand format
//   GRAD  2 A Im(exp(-i phi) B) for the adjoint
//
// Warp roles (320 threads): warps 0-7 epilogue (warp w reads TMEM lanes
// 32*(w%4).. and column half w/4; each prefetches its epilogue inputs into
// registers while the mainloop runs), warp 8 TMA producer, warp 9 TMEM
// allocator + MMA issuer.  Every mbarrier
// wait is bounded (one second of %globaltimer); a wait that gives up
// raises OFA_ERRBIT_TIMEOUT and the CTA drains and frees TMEM before exiting.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "ofa_internal.cuh"
#include "ofa_focal.cuh"
#include "ofa_math.cuh"
#include "ofa_split.cuh"
#include "umma_ptx.cuh"

using namespace ofa_ptx;

namespace {

constexpr int BM = 128;
enum { EPI_FWD = 0, EPI_BWD = 1, EPI_GRAD = 2, EPI_STORE = 3 };

// Epilogue warps: 8 (two per TMEM lane quarter) for the forward products, 16 (four
// per quarter) for the inverse, whose per-pixel epilogue needs more latency hiding.
// The two warps after them are the TMA producer and the MMA issuer.
template <int EPI> struct Warps {
  static constexpr int EPI_THREADS = EPI == EPI_FWD || EPI == EPI_STORE ? 256 : 512;
  static constexpr int TMA = EPI_THREADS / 32;
  static constexpr int MMA = TMA + 1;
  static constexpr int THREADS = EPI_THREADS + 64;
};
constexpr int NUM_EPI_THREADS = 256;  // forward epilogue (the fused focal step runs on these)
// Operand rows per stage are RB = 128 or 64 bytes of K (128B or 64B swizzle).
constexpr int SMEM_BUDGET = 200 * 1024;   // operand stages


struct EpiArgs {
  // forward
  const float2* fyT;
  int kp;
  float* part;          // [n_part][2 kp] floats
  int tiles_m;
  // inverse / gradient
  float* out;           // phi or grad [ny][nx]
  const float* phi_in;  // gradient: phase
  const float* amp;     // [ny][nx]
  int nx, ny, nxp;
  void* e_hi;
  void* e_lo;
  int prec;
  float amp_factor;
  const OfaDevState* st;
  int* err;
  // separable grid form (EPI_STORE): the product itself, per contraction part,
  // gt[split][j][n] = G[n][j] for the ep.K columns j and ep.ny rows n
  float2* gt;
  // forward with the focal step fused into its last CTA (fuse != 0)
  int fuse;
  unsigned int* counters;  // [n_tiles + 1], zero between launches
  int n_tiles;             // forward grid.x
  int n_part;              // partial rows = tiles_m * splits
  int K;
  float2* theta;           // [K] final Theta
  const float* t;
  float* w;
  float2* c;
  double* hist;
  OfaDevState* stw;
  int weighting;
};

__device__ __forceinline__ void named_bar_epi() {
  asm volatile("bar.sync 1, 256;" ::: "memory");
}
// Barrier of the four inverse-epilogue warps that read one TMEM lane quarter
// (barriers 2-5, 128 threads each).
__device__ __forceinline__ void named_bar_quarter(int quarter) {
  asm volatile("bar.sync %0, 128;" ::"r"(2 + quarter) : "memory");
}
struct BarEpi {
  __device__ __forceinline__ void operator()() const { named_bar_epi(); }
};

template <int KIND, int NPASS, int BN, int EPI, int RB, int CG>
struct Cfg {
  static constexpr int EB = KIND == KIND_TF32 ? 4 : 2;
  static constexpr int BK = RB / EB;                      // elements of K per stage
  static constexpr int PLANES = NPASS == 3 ? 2 : 1;
  static constexpr int A_BYTES = BM * RB;
  static constexpr int B_BYTES = (BN / CG) * RB;         // a pair holds half of B per CTA
  static constexpr int STAGE_BYTES = PLANES * (A_BYTES + B_BYTES);
  static constexpr int STAGES = SMEM_BUDGET / STAGE_BYTES > 12 ? 12 : SMEM_BUDGET / STAGE_BYTES;
  // the inverse epilogue stages its output through 4 x 3 x 32 x 65 words of the freed stages
  static_assert(EPI == EPI_FWD || EPI == EPI_STORE ||
                    STAGES * STAGE_BYTES >= 4 * 3 * 32 * 65 * 4,
                "epilogue staging");
  static constexpr int UMMA_K_STEPS = RB / 32;            // 32 bytes of K per MMA
  static constexpr int RED_BYTES = EPI == EPI_FWD ? 4 * BN * 4 : 0;
  static constexpr int BAR_OFF = STAGES * STAGE_BYTES + RED_BYTES;
  static constexpr int SMEM = BAR_OFF + 256 + 1024;        // barriers, slot, alignment
  static constexpr uint32_t IDESC = idesc_make(BM * CG, BN, KIND);
  static_assert(STAGES >= 2, "need at least two stages");
};

// One output tile (rows m_tile*128.., accumulator columns n_tile*BN..) over the
// k-blocks [kb0, kb0 + nkb) of the operands behind the four tensor maps, with the
// epilogue EPI.  tail_count: CTAs that arrive on ep.counters before the fused
// focal step may run (all tiles of the problem).
template <int KIND, int NPASS, int BN, int EPI, int RB, int CG>
__device__ __forceinline__ void umma_tile(const CUtensorMap* tma_hi, const CUtensorMap* tma_lo,
                                          const CUtensorMap* tmb_hi, const CUtensorMap* tmb_lo,
                                          const int m_tile, const int n_tile, const int split,
                                          const int kb0, const int nkb, const EpiArgs& ep,
                                          const int* __restrict__ done,
                                          const unsigned tail_count) {
  using C = Cfg<KIND, NPASS, BN, EPI, RB, CG>;
  constexpr bool PAIR = CG == 2;
  constexpr int WARP_TMA = Warps<EPI>::TMA, WARP_MMA = Warps<EPI>::MMA;
  constexpr int GROUPS = Warps<EPI>::EPI_THREADS / 128;   // epilogue warps per lane quarter
  constexpr int CPW = BN / (32 * GROUPS);                  // 32-column chunks per epilogue warp
  pdl_launch_dependents();  // the next kernel may start its own set-up on free SMs
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base_u32 = (raw + 1023u) & ~1023u;
  uint8_t* base = smem_raw + (base_u32 - raw);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const uint32_t bar_full = base_u32 + C::BAR_OFF;          // STAGES x 8 bytes
  const uint32_t bar_empty = bar_full + 8 * C::STAGES;      // STAGES x 8 bytes
  const uint32_t bar_accum = bar_empty + 8 * C::STAGES;     // 8 bytes
  const uint32_t slot_u32 = bar_accum + 8;                  // TMEM address slot
  volatile uint32_t* slot =
      reinterpret_cast<volatile uint32_t*>(base + C::BAR_OFF + 16 * C::STAGES + 8);

  // PAIR: clusters of two CTAs along the rows (cluster shape 2 x 1 over a grid whose x
  // runs over the row tiles) form a 2-SM MMA pair; each CTA loads its own A rows and
  // half of the B tile from global memory (no multicast).
  const int crank = PAIR ? (int)cluster_ctarank() : 0;
  const bool leader = !PAIR || (crank & 1) == 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_accum, 1);
    fence_mbar_init();
  }
  if (warp == WARP_TMA && lane == 0) {
    tmap_prefetch(tma_hi);
    tmap_prefetch(tmb_hi);
    if (NPASS == 3) {
      tmap_prefetch(tma_lo);
      tmap_prefetch(tmb_lo);
    }
  }
  if (warp == WARP_MMA) tmem_alloc<CG>(slot_u32, BN);
  tc_fence_before();
  if (PAIR) cluster_sync_all();  // partner's barriers exist before any remote signal
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  // The B operand (Fx or conj(Fx) in block form, written once per plan) of the first
  // stages is fetched before the wait for the previous kernel.  Its bytes are
  // registered on the stage's full barrier without an arrival, so a stage cannot
  // complete before its A tile (the previous kernel's output) is loaded and arrived for.
  const int npre = nkb < C::STAGES ? nkb : C::STAGES;
  if (warp == WARP_TMA && lane == 0) {
    for (int kb = 0; kb < npre; ++kb) {
      const uint32_t st = base_u32 + kb * C::STAGE_BYTES;
      const int x = (kb0 + kb) * C::BK;
      if (PAIR) {
        if (leader) mbar_expect_tx_only(bar_full + 8 * kb, 2 * C::PLANES * C::B_BYTES);
        const uint32_t fb =
            leader ? bar_full + 8 * kb : mapa_shared(bar_full + 8 * kb, crank & ~1);
        const int brow = n_tile * BN + (crank & 1) * (BN / 2);
        tma_load_2d_pair(st + C::PLANES * C::A_BYTES, tmb_hi, fb, x, brow);
        if (NPASS == 3)
          tma_load_2d_pair(st + C::PLANES * C::A_BYTES + C::B_BYTES, tmb_lo, fb, x, brow);
      } else {
        mbar_expect_tx_only(bar_full + 8 * kb, C::PLANES * C::B_BYTES);
        tma_load_2d(st + C::PLANES * C::A_BYTES, tmb_hi, bar_full + 8 * kb, x, n_tile * BN);
        if (NPASS == 3)
          tma_load_2d(st + C::PLANES * C::A_BYTES + C::B_BYTES, tmb_lo, bar_full + 8 * kb, x,
                      n_tile * BN);
      }
    }
  }
  // Everything above is independent of the previous kernel; from here on its
  // outputs (the dynamic operand, the loop flags) are read.
  pdl_wait();
  // skip: the loop already stopped, or an earlier launch gave up (uniform over the grid)
  const bool skip = (done != nullptr && *done) || (*ep.err & OFA_ERRBIT_TIMEOUT);

  if (skip) {
    // nothing to compute: the prefetched B copies must land before the CTA may leave
    // (the odd CTA of a pair waits at the teardown's cluster barrier)
    if (warp == WARP_TMA && lane == 0 && leader)
      for (int kb = 0; kb < npre; ++kb) {
        mbar_arrive(bar_full + 8 * kb);
        if (!mbar_wait(bar_full + 8 * kb, 0)) {
          atomicOr(ep.err, OFA_ERRBIT_TIMEOUT);
          break;
        }
      }
  } else if (warp == WARP_TMA) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % C::STAGES;
        if (kb >= C::STAGES) {
          if (!mbar_wait(bar_empty + 8 * s, ((kb / C::STAGES) - 1) & 1)) {
            ok = false;
            break;
          }
        }
        const uint32_t st = base_u32 + s * C::STAGE_BYTES;
        const int x = (kb0 + kb) * C::BK;
        const bool pre = kb < npre;   // B already in flight (registered above)
        if (PAIR) {
          // both CTAs' halves land on the leader's barrier, which expects them all
          if (leader)
            mbar_expect_tx(bar_full + 8 * s,
                           pre ? 2 * C::PLANES * C::A_BYTES : 2 * C::STAGE_BYTES);
          const uint32_t fb = leader ? bar_full + 8 * s : mapa_shared(bar_full + 8 * s, crank & ~1);
          const int brow = n_tile * BN + (crank & 1) * (BN / 2);
          tma_load_2d_pair(st, tma_hi, fb, x, m_tile * BM);
          if (!pre) tma_load_2d_pair(st + C::PLANES * C::A_BYTES, tmb_hi, fb, x, brow);
          if (NPASS == 3) {
            tma_load_2d_pair(st + C::A_BYTES, tma_lo, fb, x, m_tile * BM);
            if (!pre)
              tma_load_2d_pair(st + C::PLANES * C::A_BYTES + C::B_BYTES, tmb_lo, fb, x, brow);
          }
        } else {
          mbar_expect_tx(bar_full + 8 * s, pre ? C::PLANES * C::A_BYTES : C::STAGE_BYTES);
          tma_load_2d(st, tma_hi, bar_full + 8 * s, x, m_tile * BM);
          if (!pre)
            tma_load_2d(st + C::PLANES * C::A_BYTES, tmb_hi, bar_full + 8 * s, x, n_tile * BN);
          if (NPASS == 3) {
            tma_load_2d(st + C::A_BYTES, tma_lo, bar_full + 8 * s, x, m_tile * BM);
            if (!pre)
              tma_load_2d(st + C::PLANES * C::A_BYTES + C::B_BYTES, tmb_lo, bar_full + 8 * s,
                          x, n_tile * BN);
          }
        }
        ++issued;
      }
      if (!ok) atomicOr(ep.err, OFA_ERRBIT_TIMEOUT);
      // Drain: every issued copy must have landed before the CTA may exit.  (The
      // odd CTA of a pair signals the leader's barriers; its copies have landed
      // once the leader's MMAs, which read them, complete.)
      for (int kb = max(0, issued - C::STAGES); leader && kb < issued; ++kb)
        if (!mbar_wait(bar_full + 8 * (kb % C::STAGES), (kb / C::STAGES) & 1)) {
          atomicOr(ep.err, OFA_ERRBIT_TIMEOUT);
          break;
        }
    }
  } else if (warp == WARP_MMA) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0 && leader) {
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % C::STAGES;
        if (!mbar_wait(bar_full + 8 * s, (kb / C::STAGES) & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t st = base_u32 + s * C::STAGE_BYTES;
        const uint64_t a_hi = sdesc<RB>(st);
        const uint64_t a_lo = sdesc<RB>(st + C::A_BYTES);
        const uint64_t b_hi = sdesc<RB>(st + C::PLANES * C::A_BYTES);
        const uint64_t b_lo = sdesc<RB>(st + C::PLANES * C::A_BYTES + C::B_BYTES);
#pragma unroll
        for (int kk = 0; kk < C::UMMA_K_STEPS; ++kk) {
          const uint64_t adv = (uint64_t)((kk * 32) >> 4);  // 32 bytes of K per MMA
          umma<KIND, CG>(tmem, a_hi + adv, b_hi + adv, C::IDESC, (kb | kk) != 0);
          if (NPASS == 3) {
            umma<KIND, CG>(tmem, a_hi + adv, b_lo + adv, C::IDESC, 1);
            umma<KIND, CG>(tmem, a_lo + adv, b_hi + adv, C::IDESC, 1);
          }
        }
        // stage free (in this CTA, and in the partner of a pair) once these MMAs
        // have read it
        if (PAIR) umma_commit_pair(bar_empty + 8 * s, (uint16_t)(3u << (crank & ~1)));
        else umma_commit(bar_empty + 8 * s);
      }
      if (!ok) atomicOr(ep.err, OFA_ERRBIT_TIMEOUT);
      // accumulator complete (or drained, on abort), in both CTAs of a pair
      if (PAIR) umma_commit_pair(bar_accum, (uint16_t)(3u << (crank & ~1)));
      else umma_commit(bar_accum);
    }
  } else {
    // ------------------------------------------------------------ epilogue warps
    // warp w reads TMEM lanes 32*(w%4).. (rows of the tile) and column group w/4.
    const int quarter = warp & 3, half = warp >> 2;
    const int r = quarter * 32 + lane;             // accumulator row = TMEM lane
    const int n = m_tile * BM + r;                 // pupil row
    const uint32_t tw = tmem + ((uint32_t)(quarter * 32) << 16);
    const int col0 = half * CPW * 32;              // first accumulator column of this warp

    if (EPI == EPI_FWD) {
      // Prefetch this row's Fy values for the warp's foci while the mainloop runs.
      float4 fy[CPW][8];
      const float4* fr = reinterpret_cast<const float4*>(
          ep.fyT + (size_t)n * ep.kp + ((n_tile * BN + col0) >> 1));
#pragma unroll
      for (int c = 0; c < CPW; ++c)
#pragma unroll
        for (int q = 0; q < 8; ++q) fy[c][q] = __ldg(fr + c * 8 + q);
      const bool ready = mbar_wait_sleep(bar_accum, 0);
      tc_fence_after();
      if (!ready) atomicOr(ep.err, OFA_ERRBIT_TIMEOUT);
      const bool valid = ready && nkb > 0;
      float* red = reinterpret_cast<float*>(base + C::STAGES * C::STAGE_BYTES);
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        const int ch = half * CPW + c;
        uint32_t v[32];
        float p[32];
        if (valid) {
          tmem_ld32(tw + ch * 32, v);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 f = fy[c][q];
            const float g0r = __uint_as_float(v[4 * q]), g0i = __uint_as_float(v[4 * q + 1]);
            const float g1r = __uint_as_float(v[4 * q + 2]), g1i = __uint_as_float(v[4 * q + 3]);
            p[4 * q] = f.x * g0r - f.y * g0i;
            p[4 * q + 1] = f.x * g0i + f.y * g0r;
            p[4 * q + 2] = f.z * g1r - f.w * g1i;
            p[4 * q + 3] = f.z * g1i + f.w * g1r;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) p[q] = 0.f;
        }
        red[quarter * BN + ch * 32 + lane] = warp_reduce_scatter32(p);
      }
      named_bar_epi();
      const int t = threadIdx.x;  // 0..255
      float* dst = ep.part + (size_t)(split * ep.tiles_m + m_tile) * 2 * ep.kp + n_tile * BN;
      for (int col = t; col < BN; col += NUM_EPI_THREADS)
        dst[col] = ((red[col] + red[BN + col]) + red[2 * BN + col]) + red[3 * BN + col];
      if (ep.fuse) {
        // The last CTA to finish runs the focal step of the loop on the partials
        // of every tile (summed in fixed order, so the result does not depend on
        // which CTA finishes last).
        __shared__ int tail_flag;
        __shared__ float focal_sh[4 * 33];
        named_bar_epi();  // every partial of this CTA is written (CTA scope) ...
        if (t == 0) {
          __threadfence();  // ... and, cumulatively, visible GPU-wide before the arrival
          const unsigned prev = atomicAdd(ep.counters, 1u);
          tail_flag = prev == tail_count - 1u;
          if (tail_flag) {
            __threadfence();  // acquire the other CTAs' partials
            *ep.counters = 0u;
          }
        }
        named_bar_epi();
        if (tail_flag) {
          const float2* pt = reinterpret_cast<const float2*>(ep.part);
          if (ep.K <= NUM_EPI_THREADS * 4)
            ofa_focal::iterate_regs<NUM_EPI_THREADS, 4>(pt, ep.n_part, ep.K, ep.kp, ep.t, ep.w,
                                                        ep.c, ep.hist, ep.stw, ep.weighting,
                                                        focal_sh, t, BarEpi());
          else
            ofa_focal::iterate_regs<NUM_EPI_THREADS, 16>(pt, ep.n_part, ep.K, ep.kp, ep.t, ep.w,
                                                         ep.c, ep.hist, ep.stw, ep.weighting,
                                                         focal_sh, t, BarEpi());
        }
      }
    } else if (EPI == EPI_STORE) {
      // The product tile itself: lane = pupil row n, accumulator column pairs
      // (Re, Im) = complex column j; each warp store covers 32 consecutive rows of
      // one column of this contraction part's slice.
      const bool ready = mbar_wait_sleep(bar_accum, 0);
      tc_fence_after();
      if (!ready) atomicOr(ep.err, OFA_ERRBIT_TIMEOUT);
      const bool valid = ready && nkb > 0;
      float2* g = ep.gt + (size_t)split * ep.K * ep.ny;
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        const int ch = half * CPW + c;
        uint32_t v[32];
        if (valid) {
          tmem_ld32(tw + ch * 32, v);
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = 0u;
        }
        const int j0 = (n_tile * BN + ch * 32) >> 1;
        if (n < ep.ny) {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (j0 + q < ep.K)
              g[(size_t)(j0 + q) * ep.ny + n] =
                  make_float2(__uint_as_float(v[2 * q]), __uint_as_float(v[2 * q + 1]));
        }
      }
    } else {
      // Per-pixel work (thread = row).  Inputs are prefetched into registers while
      // the mainloop runs.  Warp `half` of a lane quarter takes accumulator chunks
      // c * GROUPS + half, so in pass c the quarter's four warps cover 64 consecutive
      // pixels of its 32 rows; they stage them in shared memory (free once the
      // accumulator is complete) and each warp then stores 8 whole 64-pixel row
      // segments, every warp store 128 consecutive bytes.
      const bool row_ok = n < ep.ny;
      float av[CPW * 16];
      float pv[EPI == EPI_GRAD ? CPW * 16 : 1];
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        const int mc = (n_tile * BN + (c * GROUPS + half) * 32) >> 1;  // first pixel of chunk
        const size_t rb = (size_t)n * ep.nx + mc;
        if (((ep.nx & 3) == 0) && row_ok && (mc + 16 <= ep.nx)) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 a4 = __ldg(reinterpret_cast<const float4*>(ep.amp + rb) + j);
            av[c * 16 + 4 * j] = a4.x; av[c * 16 + 4 * j + 1] = a4.y;
            av[c * 16 + 4 * j + 2] = a4.z; av[c * 16 + 4 * j + 3] = a4.w;
            if (EPI == EPI_GRAD) {
              const float4 p4 = __ldg(reinterpret_cast<const float4*>(ep.phi_in + rb) + j);
              pv[c * 16 + 4 * j] = p4.x; pv[c * 16 + 4 * j + 1] = p4.y;
              pv[c * 16 + 4 * j + 2] = p4.z; pv[c * 16 + 4 * j + 3] = p4.w;
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const bool ok = row_ok && (mc + j) < ep.nx;
            av[c * 16 + j] = ok ? __ldg(ep.amp + rb + j) : 0.f;
            if (EPI == EPI_GRAD) pv[c * 16 + j] = ok ? __ldg(ep.phi_in + rb + j) : 0.f;
          }
        }
      }
      const bool ready = mbar_wait_sleep(bar_accum, 0);
      tc_fence_after();
      if (!ready) atomicOr(ep.err, OFA_ERRBIT_TIMEOUT);
      const bool valid = ready && nkb > 0;
      constexpr int PITCH = 65;                    // words per staged row of 64 pixels
      constexpr int ARR = 32 * PITCH;              // one staged array of a quarter
      uint32_t* sq = reinterpret_cast<uint32_t*>(base) + quarter * 3 * ARR;
      float* s_o = reinterpret_cast<float*>(sq);   // phase or gradient
      uint32_t* s_a = sq + ARR;                    // field hi (TF32: real part bits)
      uint32_t* s_b = sq + 2 * ARR;                // field lo (TF32: imaginary part bits)
      const int nbase = m_tile * BM + quarter * 32;
      const bool wide = ep.prec == OFA_PREC_TF32;
      float factor = 0.f;
      if (EPI == EPI_GRAD) factor = 2.f * ep.amp_factor / ep.st->c_scale;
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        const int ch = c * GROUPS + half;
        if (valid) {
          uint32_t v[32];
          tmem_ld32(tw + ch * 32, v);
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float re = __uint_as_float(v[2 * q]), im = __uint_as_float(v[2 * q + 1]);
            const float a = av[c * 16 + q];
            const int slot = lane * PITCH + half * 16 + q;
            if (EPI == EPI_BWD) {
              // phi = arg(E') (atan2(0,0) = 0), then the next pupil field A exp(i phi),
              // formed exactly as the field-plane builder forms it from a stored phi
              const float ph = ofa_arg(im, re);
              s_o[slot] = ph;
              float sn, cs;
              __sincosf(ph, &sn, &cs);
              uint2 h, l;
              split_pack(ep.prec, a * cs, a * sn, h, l);
              s_a[slot] = h.x;
              s_b[slot] = wide ? h.y : l.x;
            } else {
              float sn, cs;
              sincosf(pv[c * 16 + q], &sn, &cs);
              s_o[slot] = factor * a * (cs * im - sn * re);
            }
          }
        }
        named_bar_quarter(quarter);
        if (valid) {
          const int px0 = ((n_tile * BN) >> 1) + c * 64;  // first pixel of this pass
#pragma unroll 2
          for (int rr = 0; rr < 8; ++rr) {
            const int row = half * 8 + rr, gn = nbase + row;
            if (gn >= ep.ny) continue;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const int px = lane + 32 * j, gm = px0 + px;
              if (gm >= ep.nx) continue;
              ep.out[(size_t)gn * ep.nx + gm] = s_o[row * PITCH + px];
              if (EPI == EPI_BWD && !wide) {
                const size_t e = (size_t)gn * ep.nxp + gm;   // complex element index
                reinterpret_cast<uint32_t*>(ep.e_hi)[e] = s_a[row * PITCH + px];
                if (ep.e_lo) reinterpret_cast<uint32_t*>(ep.e_lo)[e] = s_b[row * PITCH + px];
              }
            }
            if (EPI == EPI_BWD && wide) {
              // two words per pixel: 128 consecutive words per row segment
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int wi = lane + 32 * j, px = wi >> 1, gm = px0 + px;
                if (gm >= ep.nx) continue;
                const uint32_t word = (wi & 1) ? s_b[row * PITCH + px] : s_a[row * PITCH + px];
                reinterpret_cast<uint32_t*>(ep.e_hi)[2 * ((size_t)gn * ep.nxp + px0) + wi] = word;
              }
            }
          }
        }
        named_bar_quarter(quarter);
      }
    }
  }

  // ------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  if (warp == WARP_MMA) {
    tc_fence_after();
    tmem_dealloc<CG>(tmem, BN);
  }
  // No CTA of a pair may leave while its partner can still arrive on its barriers.
  if (PAIR) cluster_sync_all();
}

// One plan: tile coordinates from the grid (2-SM pairs lie along the cluster's x
// dimension, so their grids put the row tiles on x; otherwise the column tiles
// are on x), split-K over grid z.
template <int KIND, int NPASS, int BN, int EPI, int RB, int CG>
__global__ void __launch_bounds__(Warps<EPI>::THREADS, 1)
    umma_gemm_kernel(const __grid_constant__ CUtensorMap tma_hi,
                     const __grid_constant__ CUtensorMap tma_lo,
                     const __grid_constant__ CUtensorMap tmb_hi,
                     const __grid_constant__ CUtensorMap tmb_lo, int kb_per_split, int kb_total,
                     const __grid_constant__ EpiArgs ep, const int* __restrict__ done) {
  constexpr bool PAIR = CG == 2;
  const int n_tile = PAIR ? blockIdx.y : blockIdx.x, m_tile = PAIR ? blockIdx.x : blockIdx.y;
  const int split = blockIdx.z;
  const int kb0 = split * kb_per_split;
  const int nkb = min(kb_per_split, kb_total - kb0);
  umma_tile<KIND, NPASS, BN, EPI, RB, CG>(&tma_hi, &tma_lo, &tmb_hi, &tmb_lo, m_tile, n_tile,
                                          split, kb0, nkb, ep, done,
                                          gridDim.x * gridDim.y * gridDim.z);
}

// Many problems in one launch: block b computes tile tiles[b] = (problem, m_tile,
// n_tile) of problem items[problem], whose tensor maps and epilogue arguments sit
// in device memory (written once before the first launch and never modified).
struct GroupItem {  // aligned as its tensor maps are
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
  EpiArgs ep;
  int kb_total;
  unsigned tail_count;
};

template <int KIND, int NPASS, int BN, int EPI, int RB>
__global__ void __launch_bounds__(Warps<EPI>::THREADS, 1)
    umma_group_kernel(const GroupItem* __restrict__ items, const int4* __restrict__ tiles) {
  const int4 t = tiles[blockIdx.x];
  const GroupItem* g = items + t.x;
  umma_tile<KIND, NPASS, BN, EPI, RB, 1>(&g->a_hi, &g->a_lo, &g->b_hi, &g->b_lo, t.y, t.z, 0, 0,
                                         g->kb_total, g->ep, nullptr, g->tail_count);
}

// Diagnostic: the bounded wait of the pipelines above, on a barrier nothing
// arrives at (expected phase 0 of a barrier initialised with one arrival).
__global__ void selftest_wait_kernel(OfaDevState* st) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  fence_mbar_init();
  if (!mbar_wait(b, 0)) atomicOr(&st->err, OFA_ERRBIT_TIMEOUT);
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

bool encode(CUtensorMap* m, void* ptr, int elem_bytes, uint64_t cols, uint64_t rows,
            uint32_t box_rows, int rb, std::string& err) {
  auto fn = encode_fn();
  if (fn == nullptr) {
    err = "cuTensorMapEncodeTiled is not available from the driver";
    return false;
  }
  const CUtensorMapDataType dt =
      elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * (cuuint64_t)elem_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(rb / elem_bytes), box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, dt, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  rb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r);
    return false;
  }
  return true;
}

template <int V>
using IC = std::integral_constant<int, V>;

// Calls f(kind, npass, bn, rb, cg) (integral constants) for the kernel variant of
// a precision, tile width (accumulator columns), operand row width (bytes; only
// the 128-byte rows are instantiated: 64-byte rows never measured faster) and
// CTA group (1, or 2 for a 2-SM pair).
template <class F>
void visit_variant(int prec, int bn, int rb, int cg, F&& f) {
  (void)rb;
  auto by_cg = [&](auto kind, auto npass, auto bnc) {
    if (cg == 2) f(kind, npass, bnc, IC<128>{}, IC<2>{});
    else f(kind, npass, bnc, IC<128>{}, IC<1>{});
  };
  auto by_bn = [&](auto kind, auto npass) {
    if (bn == 256) by_cg(kind, npass, IC<256>{});
    else by_cg(kind, npass, IC<128>{});
  };
  switch (prec) {
    case OFA_PREC_TF32: by_bn(IC<KIND_TF32>{}, IC<1>{}); break;
    case OFA_PREC_BF16: by_bn(IC<KIND_BF16>{}, IC<1>{}); break;
    case OFA_PREC_BF16X3: by_bn(IC<KIND_BF16>{}, IC<3>{}); break;
    case OFA_PREC_F16X3: by_bn(IC<KIND_F16>{}, IC<3>{}); break;
    default: break;
  }
}

#define OFA_VARIANT_TYPES                                                        \
  constexpr int K_ = decltype(kind)::value, NP_ = decltype(npass)::value;        \
  constexpr int BN_ = decltype(bnc)::value, RB_ = decltype(rbc)::value;          \
  constexpr int CG_ = decltype(cgc)::value;                                       \
  using C = Cfg<K_, NP_, BN_, EPI, RB_, CG_>;                                     \
  (void)sizeof(C)

// Launch configuration: programmatic dependent launch always; a 2 x 1 cluster for
// the CTA pairs of cta_group::2 (cg = 2), no cluster otherwise.
cudaLaunchConfig_t make_cfg(dim3 grid, int threads, int smem, cudaStream_t s,
                            cudaLaunchAttribute* attr, int cg) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = cg;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cg == 2 ? 2 : 1;
  return cfg;
}

template <int EPI>
void launch_gemm(int prec, int bn, int rb, int cg, const CUtensorMap& a_hi,
                 const CUtensorMap& a_lo, const CUtensorMap& b_hi, const CUtensorMap& b_lo,
                 dim3 grid, int kbps, int kbt, const EpiArgs& ep, const int* done,
                 cudaStream_t s) {
  visit_variant(prec, bn, rb, cg, [&](auto kind, auto npass, auto bnc, auto rbc, auto cgc) {
    if constexpr (EPI == EPI_STORE && decltype(cgc)::value == 2) {
      return;  // the store epilogue runs on single CTAs only
    } else {
      OFA_VARIANT_TYPES;
      const dim3 g = CG_ == 2 ? dim3(grid.y, grid.x, grid.z) : grid;  // pairs: rows on x
      cudaLaunchAttribute attr[2];
      cudaLaunchConfig_t cfg = make_cfg(g, Warps<EPI>::THREADS, C::SMEM, s, attr, CG_);
      cudaLaunchKernelEx(&cfg, umma_gemm_kernel<K_, NP_, BN_, EPI, RB_, CG_>, a_hi, a_lo, b_hi,
                         b_lo, kbps, kbt, ep, done);
    }
  });
}

template <int EPI>
cudaError_t set_attr_epi(int prec) {
  cudaError_t e = cudaSuccess;
  for (int bn : {128, 256})
    for (int cg : {1, 2})
      visit_variant(prec, bn, 128, cg, [&](auto kind, auto npass, auto bnc, auto rbc, auto cgc) {
        if constexpr (!(EPI == EPI_STORE && decltype(cgc)::value == 2)) {
          OFA_VARIANT_TYPES;
          cudaError_t r = cudaFuncSetAttribute(umma_gemm_kernel<K_, NP_, BN_, EPI, RB_, CG_>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               C::SMEM);
          if (r != cudaSuccess) e = r;
        }
      });
  return e;
}

EpiArgs base_args(ofa_plan* p) {
  EpiArgs ep;
  std::memset(&ep, 0, sizeof(ep));
  ep.fyT = p->fyT;
  ep.kp = p->kp;
  ep.part = reinterpret_cast<float*>(p->part);
  ep.tiles_m = p->nyp / BM;
  ep.amp = p->amp;
  ep.nx = p->nx;
  ep.ny = p->ny;
  ep.nxp = p->nxp;
  ep.prec = p->precision;
  ep.amp_factor = ldexpf(1.f, p->amp_exp);
  ep.st = p->st;
  ep.err = &p->st->err;
  return ep;
}

}  // namespace


// Opt every kernel variant of a precision into its dynamic shared memory (done
// once per plan, outside any stream capture; the attribute is per device).
cudaError_t tc_prepare(int prec) {
  const cudaError_t es[4] = {set_attr_epi<EPI_FWD>(prec), set_attr_epi<EPI_BWD>(prec),
                             set_attr_epi<EPI_GRAD>(prec), set_attr_epi<EPI_STORE>(prec)};
  for (cudaError_t e : es)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

bool tc_encode_maps(ofa_plan* p, TcOperands& t, std::string& err);

void launch_selftest_wait(OfaDevState* st, cudaStream_t s) {
  selftest_wait_kernel<<<1, 1, 0, s>>>(st);
}

namespace {
struct TuneResult {
  int fwd_bn, fwd_split, fwd_cg, bwd_bn, bwd_cg;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, TuneResult> g_tune_cache;

void apply(TcOperands& t, const TuneResult& r) {
  t.fwd_bn = r.fwd_bn; t.fwd_split = r.fwd_split; t.fwd_cg = r.fwd_cg;
  t.bwd_bn = r.bwd_bn; t.bwd_cg = r.bwd_cg;
}
}  // namespace

bool tc_config_valid(const ofa_plan* p, const TcOperands& t, int fwd_bn, int fwd_split,
                     int fwd_cg, int bwd_bn, int bwd_cg) {
  const int tiles_m = p->nyp / BM;
  const int kb_fwd = (2 * p->nxp * t.elem_bytes) / 128;
  if (fwd_bn != 128 && fwd_bn != 256) return false;
  if (bwd_bn != 128 && bwd_bn != 256) return false;
  if (fwd_split != 1 && fwd_split != 2 && fwd_split != 4) return false;
  if (kb_fwd < fwd_split) return false;
  if (fwd_cg != 1 && fwd_cg != 2) return false;
  if (bwd_cg != 1 && bwd_cg != 2) return false;
  // a 2-SM pair covers two row tiles
  if ((fwd_cg == 2 || bwd_cg == 2) && tiles_m % 2 != 0) return false;
  return (2 * t.kp) % fwd_bn == 0 && (2 * p->nxp) % bwd_bn == 0;
}

bool tc_autotune(ofa_plan* p, TcOperands& t, std::string& err) {
  const auto key = std::make_tuple(p->device, p->nx, p->ny, p->K, p->precision);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      apply(t, it->second);
      return true;
    }
  }
  // OFA_AUTOTUNE_VERBOSE=1 prints every candidate's time to stderr
  const char* venv = getenv("OFA_AUTOTUNE_VERBOSE");
  const bool verbose = venv != nullptr && venv[0] == '1';
  // Scratch outputs: the inverse candidates must not touch the loop's phase and field.
  float* phi_scratch = nullptr;
  const size_t e_bytes = (size_t)p->nyp * 2 * p->nxp * t.elem_bytes;
  void* e_scr[2] = {nullptr, nullptr};
  bool ok = cudaMalloc(&phi_scratch, (size_t)p->nx * p->ny * 4) == cudaSuccess &&
            cudaMalloc(&e_scr[0], e_bytes) == cudaSuccess &&
            (t.npass == 1 || cudaMalloc(&e_scr[1], e_bytes) == cudaSuccess);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ok = ok && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  if (!ok) err = "allocating autotune scratch";
  const int reps = 5;
  auto time_it = [&](auto&& launch) -> float {
    launch();  // warm-up
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
      if (verbose) fprintf(stderr, "ofa autotune: candidate not launchable: %s\n",
                           cudaGetErrorString(le));
      return 1e30f;
    }
    cudaEventRecord(e0, p->stream);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, p->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (cudaGetLastError() != cudaSuccess) return 1e30f;
    return ms;
  };
  float best_f = 1e30f, best_b = 1e30f;
  TuneResult res = {t.fwd_bn, t.fwd_split, 1, t.bwd_bn, 1};
  const int kb_fwd = (2 * p->nxp * t.elem_bytes) / 128;
  for (int cg : {1, 2}) {
    for (int bn : {128, 256}) {
      for (int split = 1; split <= 4 && ok; split *= 2) {
        if (kb_fwd / split < 4) break;
        if (!tc_config_valid(p, t, bn, split, cg, 128, 1)) continue;
        TcOperands cand = t;
        cand.fwd_bn = bn; cand.fwd_split = split; cand.fwd_cg = cg;
        if (!tc_encode_maps(p, cand, err)) { ok = false; break; }
        const float ms = time_it([&] { launch_fwd_tc(p, cand, nullptr, p->stream, false); });
        if (verbose)
          fprintf(stderr, "ofa autotune forward bn=%d split=%d cg=%d: %.2f us\n", bn, split, cg,
                  1000.f * ms / reps);
        if (ms < best_f) {
          best_f = ms;
          res.fwd_bn = bn; res.fwd_split = split; res.fwd_cg = cg;
        }
      }
    }
  }
  for (int cg : {1, 2}) {
    for (int bn : {128, 256}) {
      if (!ok) break;
      if (!tc_config_valid(p, t, 128, 1, 1, bn, cg)) continue;
      TcOperands cand = t;
      cand.e_hi = e_scr[0];
      cand.e_lo = e_scr[1];
      cand.bwd_bn = bn; cand.bwd_cg = cg;
      if (!tc_encode_maps(p, cand, err)) { ok = false; break; }
      float* keep = p->phi;
      p->phi = phi_scratch;
      const float ms = time_it([&] { launch_bwd_tc(p, cand, nullptr, p->stream); });
      p->phi = keep;
      if (verbose)
        fprintf(stderr, "ofa autotune inverse bn=%d cg=%d: %.2f us\n", bn, cg,
                1000.f * ms / reps);
      if (ms < best_b) {
        best_b = ms;
        res.bwd_bn = bn; res.bwd_cg = cg;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(phi_scratch);
  cudaFree(e_scr[0]);
  if (e_scr[1]) cudaFree(e_scr[1]);
  cudaGetLastError();
  if (!ok) return false;
  apply(t, res);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = res;
  return true;
}

bool tc_encode_maps(ofa_plan* p, TcOperands& t, std::string& err) {
  const int eb = t.elem_bytes;
  const uint64_t e_cols = 2 * (uint64_t)p->nxp, k_cols = 2 * (uint64_t)t.kp;
  bool ok = true;
  // boxes are whole tiles; a 2-SM pair loads half of the B tile per CTA
  const uint32_t e_box = BM, bx_box = t.fwd_bn / t.fwd_cg;
  const uint32_t p_box = BM, q_box = t.bwd_bn / t.bwd_cg;
  const int fr = t.fwd_rb, br = t.bwd_rb;
  ok = ok && encode(&t.tm_e_hi, t.e_hi, eb, e_cols, p->nyp, e_box, fr, err);
  ok = ok && encode(&t.tm_bx_hi, t.bx_hi, eb, e_cols, 2 * (uint64_t)t.kp, bx_box, fr, err);
  ok = ok && encode(&t.tm_p_hi, t.p_hi, eb, k_cols, p->nyp, p_box, br, err);
  ok = ok && encode(&t.tm_q_hi, t.q_hi, eb, k_cols, 2 * (uint64_t)p->nxp, q_box, br, err);
  if (t.npass == 3) {
    ok = ok && encode(&t.tm_e_lo, t.e_lo, eb, e_cols, p->nyp, e_box, fr, err);
    ok = ok && encode(&t.tm_bx_lo, t.bx_lo, eb, e_cols, 2 * (uint64_t)t.kp, bx_box, fr, err);
    ok = ok && encode(&t.tm_p_lo, t.p_lo, eb, k_cols, p->nyp, p_box, br, err);
    ok = ok && encode(&t.tm_q_lo, t.q_lo, eb, k_cols, 2 * (uint64_t)p->nxp, q_box, br, err);
  } else {
    t.tm_e_lo = t.tm_e_hi;
    t.tm_bx_lo = t.tm_bx_hi;
    t.tm_p_lo = t.tm_p_hi;
    t.tm_q_lo = t.tm_q_hi;
  }
  return ok;
}

void launch_fwd_tc(ofa_plan* p, const TcOperands& t, const int* done, cudaStream_t s,
                   bool fuse_focal) {
  const int kb_total = (2 * p->nxp * t.elem_bytes) / t.fwd_rb;
  const int kbps = (kb_total + t.fwd_split - 1) / t.fwd_split;
  dim3 grid((2 * t.kp) / t.fwd_bn, p->nyp / BM, t.fwd_split);
  EpiArgs ep = base_args(p);
  if (fuse_focal) {
    ep.fuse = 1;
    ep.counters = p->counters;
    ep.n_tiles = (int)grid.x;
    ep.n_part = fwd_n_part(p->nyp, t);
    ep.K = p->K;
    ep.theta = p->theta;
    ep.t = p->t;
    ep.w = p->w;
    ep.c = p->c;
    ep.hist = p->hist;
    ep.stw = p->st;
    ep.weighting = p->weighting;
  }
  launch_gemm<EPI_FWD>(p->precision, t.fwd_bn, t.fwd_rb, t.fwd_cg, t.tm_e_hi,
                       t.tm_e_lo, t.tm_bx_hi, t.tm_bx_lo, grid, kbps, kb_total, ep, done, s);
}

// Separable grid form: G = E Fxu^T on the tensor cores, each contraction part's
// product into its slice of p->gt ([split][ux][ny]).
void launch_fwd_sep_tc(ofa_plan* p, const TcOperands& t, const int* done, cudaStream_t s) {
  const int kb_total = (2 * p->nxp * t.elem_bytes) / t.fwd_rb;
  const int kbps = (kb_total + t.fwd_split - 1) / t.fwd_split;
  dim3 grid((2 * t.kp) / t.fwd_bn, p->nyp / BM, t.fwd_split);
  EpiArgs ep = base_args(p);
  ep.gt = p->gt;
  ep.K = p->ux;
  launch_gemm<EPI_STORE>(p->precision, t.fwd_bn, t.fwd_rb, 1, t.tm_e_hi, t.tm_e_lo, t.tm_bx_hi,
                         t.tm_bx_lo, grid, kbps, kb_total, ep, done, s);
}

void launch_bwd_tc(ofa_plan* p, const TcOperands& t, const int* done, cudaStream_t s) {
  const int kb_total = (2 * t.kp * t.elem_bytes) / t.bwd_rb;
  dim3 grid((2 * p->nxp) / t.bwd_bn, p->nyp / BM, 1);
  EpiArgs ep = base_args(p);
  ep.out = p->phi;
  ep.e_hi = t.e_hi;
  ep.e_lo = t.e_lo;
  launch_gemm<EPI_BWD>(p->precision, t.bwd_bn, t.bwd_rb, t.bwd_cg, t.tm_p_hi,
                       t.tm_p_lo, t.tm_q_hi, t.tm_q_lo, grid, kb_total, kb_total, ep, done, s);
}

void launch_grad_tc(ofa_plan* p, const TcOperands& t, const float* phi, float scale_unused,
                    float* grad, cudaStream_t s) {
  (void)scale_unused;
  const int kb_total = (2 * t.kp * t.elem_bytes) / t.bwd_rb;
  dim3 grid((2 * p->nxp) / t.bwd_bn, p->nyp / BM, 1);
  EpiArgs ep = base_args(p);
  ep.out = grad;
  ep.phi_in = phi;
  launch_gemm<EPI_GRAD>(p->precision, t.bwd_bn, t.bwd_rb, t.bwd_cg, t.tm_p_hi,
                        t.tm_p_lo, t.tm_q_hi, t.tm_q_lo, grid, kb_total, kb_total, ep, nullptr, s);
}

// ------------------------------------------------------------------ batched (grouped) launches
// Every problem of a batch shares the precision and one tile width per product;
// each grouped launch covers all tiles of all problems, largest problems first.
namespace {

struct TcGroupSet {
  int bn = 0;
  GroupItem* items = nullptr;  // device [problems]
  int4* tiles = nullptr;       // device [n_tiles]: (problem, m_tile, n_tile, 0)
  int n_tiles = 0;
};

void free_set(TcGroupSet& s) {
  if (s.items) cudaFree(s.items);
  if (s.tiles) cudaFree(s.tiles);
  s = TcGroupSet();
}

// Items of one product (EPI_FWD: forward with the fused focal step when fuse;
// EPI_BWD: inverse, writing phi and the field planes, or the scratch outputs when
// given) at tile width bn.
bool build_set(const std::vector<ofa_plan*>& plans, const std::vector<int>& order, int epi,
               int bn, bool fuse, float* out_scratch, void* e_scratch_hi, void* e_scratch_lo,
               TcGroupSet& set, std::string& err) {
  std::vector<GroupItem> items(plans.size());
  std::vector<int4> tiles;
  for (size_t h = 0; h < plans.size(); ++h) {
    ofa_plan* p = plans[h];
    const TcOperands& t = p->tc;
    GroupItem& g = items[h];
    std::memset(&g, 0, sizeof(g));
    const int eb = t.elem_bytes;
    const uint64_t e_cols = 2 * (uint64_t)p->nxp, k_cols = 2 * (uint64_t)p->kp;
    bool ok = true;
    g.ep = base_args(p);
    if (epi == EPI_FWD) {
      ok = ok && encode(&g.a_hi, t.e_hi, eb, e_cols, p->nyp, BM, 128, err);
      ok = ok && encode(&g.b_hi, t.bx_hi, eb, e_cols, k_cols, bn, 128, err);
      if (t.npass == 3) {
        ok = ok && encode(&g.a_lo, t.e_lo, eb, e_cols, p->nyp, BM, 128, err);
        ok = ok && encode(&g.b_lo, t.bx_lo, eb, e_cols, k_cols, bn, 128, err);
      }
      g.kb_total = (int)(e_cols * eb / 128);
      g.tail_count = (unsigned)((k_cols / bn) * (p->nyp / BM));
      if (fuse) {
        g.ep.fuse = 1;
        g.ep.counters = p->counters;
        g.ep.n_tiles = (int)(k_cols / bn);
        g.ep.n_part = p->nyp / BM;
        g.ep.K = p->K;
        g.ep.theta = p->theta;
        g.ep.t = p->t;
        g.ep.w = p->w;
        g.ep.c = p->c;
        g.ep.hist = p->hist;
        g.ep.stw = p->st;
        g.ep.weighting = p->weighting;
      }
    } else {
      ok = ok && encode(&g.a_hi, t.p_hi, eb, k_cols, p->nyp, BM, 128, err);
      ok = ok && encode(&g.b_hi, t.q_hi, eb, k_cols, e_cols, bn, 128, err);
      if (t.npass == 3) {
        ok = ok && encode(&g.a_lo, t.p_lo, eb, k_cols, p->nyp, BM, 128, err);
        ok = ok && encode(&g.b_lo, t.q_lo, eb, k_cols, e_cols, bn, 128, err);
      }
      g.kb_total = (int)(k_cols * eb / 128);
      g.ep.out = out_scratch ? out_scratch : p->phi;
      g.ep.e_hi = e_scratch_hi ? e_scratch_hi : t.e_hi;
      g.ep.e_lo = e_scratch_hi ? e_scratch_lo : t.e_lo;
    }
    if (t.npass != 3) {
      g.a_lo = g.a_hi;
      g.b_lo = g.b_hi;
    }
    if (!ok) return false;
  }
  for (int h : order) {
    ofa_plan* p = plans[h];
    const int cols = epi == EPI_FWD ? 2 * p->kp : 2 * p->nxp;
    for (int m = 0; m < p->nyp / BM; ++m)
      for (int n = 0; n < cols / bn; ++n) tiles.push_back(make_int4(h, m, n, 0));
  }
  set.bn = bn;
  set.n_tiles = (int)tiles.size();
  if (cudaMalloc(&set.items, items.size() * sizeof(GroupItem)) != cudaSuccess ||
      cudaMalloc(&set.tiles, tiles.size() * sizeof(int4)) != cudaSuccess) {
    err = "allocating batch tile tables";
    return false;
  }
  if (cudaMemcpy(set.items, items.data(), items.size() * sizeof(GroupItem),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(set.tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    err = "uploading batch tile tables";
    return false;
  }
  return true;
}

template <int EPI>
void launch_group(int prec, const TcGroupSet& set, cudaStream_t s) {
  visit_variant(prec, set.bn, 128, 1, [&](auto kind, auto npass, auto bnc, auto rbc, auto cgc) {
    OFA_VARIANT_TYPES;
    if constexpr (CG_ == 1) {
      cudaLaunchAttribute attr[2];
      cudaLaunchConfig_t cfg =
          make_cfg(dim3(set.n_tiles), Warps<EPI>::THREADS, C::SMEM, s, attr, 1);
      cudaLaunchKernelEx(&cfg, umma_group_kernel<K_, NP_, BN_, EPI, RB_>, set.items, set.tiles);
    }
  });
}

template <int EPI>
cudaError_t set_attr_group(int prec) {
  cudaError_t e = cudaSuccess;
  for (int bn : {128, 256})
    visit_variant(prec, bn, 128, 1, [&](auto kind, auto npass, auto bnc, auto rbc, auto cgc) {
      OFA_VARIANT_TYPES;
      if constexpr (CG_ == 1) {
        cudaError_t r = cudaFuncSetAttribute(umma_group_kernel<K_, NP_, BN_, EPI, RB_>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (r != cudaSuccess) e = r;
      }
    });
  return e;
}

}  // namespace

struct TcBatch {
  int prec = 0;
  std::vector<ofa_plan*> plans;
  TcGroupSet fwd, bwd;
  BpGroupItem* bp_items = nullptr;  // device [problems]
  int4* bp_chunks = nullptr;        // device [n_bp]: (problem, first quad, end quad, 0)
  int n_bp = 0;
};

void tc_batch_destroy(TcBatch* b) {
  if (!b) return;
  free_set(b->fwd);
  free_set(b->bwd);
  if (b->bp_items) cudaFree(b->bp_items);
  if (b->bp_chunks) cudaFree(b->bp_chunks);
  delete b;
}

void tc_batch_enqueue_iteration(const TcBatch* b, cudaStream_t s) {
  launch_group<EPI_FWD>(b->prec, b->fwd, s);
  launch_build_p_group(b->bp_items, b->bp_chunks, b->n_bp, b->prec, s);
  launch_group<EPI_BWD>(b->prec, b->bwd, s);
}

void tc_batch_config(const TcBatch* b, int* fwd_bn, int* bwd_bn) {
  *fwd_bn = b->fwd.bn;
  *bwd_bn = b->bwd.bn;
}

bool tc_batch_create(ofa_plan* const* plans, int count, cudaStream_t s, TcBatch** out,
                     std::string& err) {
  *out = nullptr;
  TcBatch* b = new TcBatch();
  b->prec = plans[0]->precision;
  b->plans.assign(plans, plans + count);
  // largest problems first (per-tile work is proportional to the contraction length)
  std::vector<int> fwd_order(count), bwd_order(count);
  for (int i = 0; i < count; ++i) fwd_order[i] = bwd_order[i] = i;
  std::stable_sort(fwd_order.begin(), fwd_order.end(),
                   [&](int a, int c) { return plans[a]->nxp > plans[c]->nxp; });
  std::stable_sort(bwd_order.begin(), bwd_order.end(),
                   [&](int a, int c) { return plans[a]->kp > plans[c]->kp; });
  cudaError_t ae = set_attr_group<EPI_FWD>(b->prec);
  if (ae == cudaSuccess) ae = set_attr_group<EPI_BWD>(b->prec);
  if (ae != cudaSuccess) {
    err = std::string("setting grouped kernel attributes: ") + cudaGetErrorString(ae);
    tc_batch_destroy(b);
    return false;
  }
  // inverse operand build: chunks of up to 4096 quads (4 complex elements each)
  {
    std::vector<BpGroupItem> items(count);
    std::vector<int4> chunks;
    for (int h = 0; h < count; ++h) {
      ofa_plan* p = plans[h];
      items[h].fyT = p->fyT;
      items[h].c = p->c;
      items[h].hi = p->tc.p_hi;
      items[h].lo = p->tc.p_lo;
      items[h].kp = p->kp;
      const int quads = p->nyp * p->kp / 4;
      for (int q = 0; q < quads; q += 4096) chunks.push_back(make_int4(h, q, std::min(quads, q + 4096), 0));
    }
    b->n_bp = (int)chunks.size();
    if (cudaMalloc(&b->bp_items, items.size() * sizeof(BpGroupItem)) != cudaSuccess ||
        cudaMalloc(&b->bp_chunks, chunks.size() * sizeof(int4)) != cudaSuccess ||
        cudaMemcpy(b->bp_items, items.data(), items.size() * sizeof(BpGroupItem),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->bp_chunks, chunks.data(), chunks.size() * sizeof(int4),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      err = "allocating the batch's operand-build tables";
      tc_batch_destroy(b);
      return false;
    }
  }
  // Tile widths: time both for each product on this batch.  The forward candidates
  // run without the focal step (they only write partials); the inverse candidates
  // write scratch outputs, so the loop state is untouched.
  size_t max_pix = 0, max_e = 0;
  for (ofa_plan* p : b->plans) {
    max_pix = std::max(max_pix, (size_t)p->nx * p->ny);
    max_e = std::max(max_e, (size_t)p->nyp * 2 * p->nxp * p->tc.elem_bytes);
  }
  float* out_scr = nullptr;
  void* e_scr[2] = {nullptr, nullptr};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaMalloc(&out_scr, max_pix * 4) == cudaSuccess &&
            cudaMalloc(&e_scr[0], max_e) == cudaSuccess &&
            (prec_npass(b->prec) == 1 || cudaMalloc(&e_scr[1], max_e) == cudaSuccess) &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  if (!ok) err = "allocating batch autotune scratch";
  auto time_it = [&](auto&& launch) -> float {
    launch();
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r) launch();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return cudaGetLastError() == cudaSuccess ? ms : 1e30f;
  };
  const char* venv = getenv("OFA_AUTOTUNE_VERBOSE");
  const bool verbose = venv != nullptr && venv[0] == '1';
  float best_f = 1e30f, best_b = 1e30f;
  int bn_f = 128, bn_b = 128;
  for (int bn : {128, 256}) {
    if (!ok) break;
    TcGroupSet f, w;
    ok = build_set(b->plans, fwd_order, EPI_FWD, bn, false, nullptr, nullptr, nullptr, f, err) &&
         build_set(b->plans, bwd_order, EPI_BWD, bn, false, out_scr, e_scr[0], e_scr[1], w, err);
    if (ok) {
      const float tf = time_it([&] { launch_group<EPI_FWD>(b->prec, f, s); });
      const float tb = time_it([&] { launch_group<EPI_BWD>(b->prec, w, s); });
      if (verbose)
        fprintf(stderr, "ofa batch autotune bn=%d: forward %.1f us, inverse %.1f us\n", bn,
                1000.f * tf / 3, 1000.f * tb / 3);
      if (tf < best_f) { best_f = tf; bn_f = bn; }
      if (tb < best_b) { best_b = tb; bn_b = bn; }
    }
    cudaStreamSynchronize(s);
    free_set(f);
    free_set(w);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out_scr);
  cudaFree(e_scr[0]);
  if (e_scr[1]) cudaFree(e_scr[1]);
  ok = ok && best_f < 1e29f && best_b < 1e29f;
  if (!ok && err.empty()) err = "no grouped kernel variant could be launched";
  ok = ok &&
       build_set(b->plans, fwd_order, EPI_FWD, bn_f, true, nullptr, nullptr, nullptr, b->fwd,
                 err) &&
       build_set(b->plans, bwd_order, EPI_BWD, bn_b, false, nullptr, nullptr, nullptr, b->bwd,
                 err);
  cudaGetLastError();
  if (!ok) {
    tc_batch_destroy(b);
    return false;
  }
  *out = b;
  return true;
}
