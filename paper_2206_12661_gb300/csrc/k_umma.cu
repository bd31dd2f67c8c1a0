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
// Warp roles (192 threads): warps 0-3 epilogue (TMEM lanes 32w..32w+31),
// warp 4 TMA producer, warp 5 TMEM allocator + MMA issuer.  Every mbarrier
// wait is bounded (one second of %globaltimer); a wait that gives up
// raises OFA_ERRBIT_TIMEOUT and the CTA drains and frees TMEM before exiting.
#include <cudaTypedefs.h>

#include <cstring>

#include "ofa_internal.cuh"
#include "ofa_split.cuh"

namespace {

constexpr int BM = 128;
constexpr int NTHREADS = 192;
constexpr int ROW_BYTES = 128;            // one 128B-swizzle row per operand row per stage
constexpr int SMEM_BUDGET = 200 * 1024;   // operand stages
constexpr uint64_t WAIT_NS = 1000000000ull;

enum { EPI_FWD = 0, EPI_BWD = 1, EPI_GRAD = 2 };
enum { KIND_F16 = 0, KIND_BF16 = 1, KIND_TF32 = 2 };

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
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (gtimer() - t0 > WAIT_NS) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tmap_prefetch(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
template <int KIND>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                     uint32_t idesc, uint32_t accumulate) {
  if (KIND == KIND_TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row core-matrix groups 1024 bytes apart (SBO), LBO unused (1),
// descriptor version 1 (bits 46-48), swizzle mode 2 = 128B (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16 / kind::tf32: D = F32 (bits 4-5 = 1),
// A and B format (bits 7-9, 10-12: 0 F16, 1 BF16, 2 TF32), both K-major
// (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_make(int M, int N, int kind) {
  return (1u << 4) | ((uint32_t)kind << 7) | ((uint32_t)kind << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Butterfly reduce-scatter of 32 values over the 32 lanes: afterwards lane l
// holds the warp-wide sum of element l (31 shuffles for 32 sums).
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = upper ? v[i] : v[i + off];
      const float keep = upper ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

__device__ __forceinline__ void named_bar_epi() {
  asm volatile("bar.sync 1, 128;" ::: "memory");
}

template <int KIND, int NPASS, int BN, int EPI>
struct Cfg {
  static constexpr int EB = KIND == KIND_TF32 ? 4 : 2;
  static constexpr int BK = ROW_BYTES / EB;               // elements per stage
  static constexpr int PLANES = NPASS == 3 ? 2 : 1;
  static constexpr int A_BYTES = BM * ROW_BYTES;          // 16 KB
  static constexpr int B_BYTES = BN * ROW_BYTES;          // 16 or 32 KB
  static constexpr int STAGE_BYTES = PLANES * (A_BYTES + B_BYTES);
  static constexpr int STAGES = SMEM_BUDGET / STAGE_BYTES > 8 ? 8 : SMEM_BUDGET / STAGE_BYTES;
  static constexpr int UMMA_K_STEPS = 4;                  // 32 bytes of K per MMA
  static constexpr int RED_BYTES = EPI == EPI_FWD ? 4 * BN * 4 : 0;
  static constexpr int BAR_OFF = STAGES * STAGE_BYTES + RED_BYTES;
  static constexpr int SMEM = BAR_OFF + 256 + 1024;        // barriers, slot, alignment
  static constexpr uint32_t IDESC = idesc_make(BM, BN, KIND);
  static_assert(STAGES >= 2, "need at least two stages");
};

template <int KIND, int NPASS, int BN, int EPI>
__global__ void __launch_bounds__(NTHREADS, 1)
    umma_gemm_kernel(const __grid_constant__ CUtensorMap tma_hi,
                     const __grid_constant__ CUtensorMap tma_lo,
                     const __grid_constant__ CUtensorMap tmb_hi,
                     const __grid_constant__ CUtensorMap tmb_lo, int kb_per_split, int kb_total,
                     EpiArgs ep, const int* __restrict__ done) {
  using C = Cfg<KIND, NPASS, BN, EPI>;
  if (done != nullptr && *done) return;
  if (*ep.err & OFA_ERRBIT_TIMEOUT) return;  // an earlier launch already gave up
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base_u32 = (raw + 1023u) & ~1023u;
  uint8_t* base = smem_raw + (base_u32 - raw);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tile = blockIdx.x, m_tile = blockIdx.y, split = blockIdx.z;
  const int kb0 = split * kb_per_split;
  const int nkb = min(kb_per_split, kb_total - kb0);

  const uint32_t bar_full = base_u32 + C::BAR_OFF;          // STAGES x 8 bytes
  const uint32_t bar_empty = bar_full + 8 * C::STAGES;      // STAGES x 8 bytes
  const uint32_t bar_accum = bar_empty + 8 * C::STAGES;     // 8 bytes
  const uint32_t slot_u32 = bar_accum + 8;                  // TMEM address slot
  volatile uint32_t* slot = reinterpret_cast<volatile uint32_t*>(base + C::BAR_OFF + 16 * C::STAGES + 8);
  __shared__ int abort_flag;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_accum, 1);
    fence_mbar_init();
  }
  if (warp == 4 && lane == 0) {
    tmap_prefetch(&tma_hi);
    tmap_prefetch(&tmb_hi);
    if (NPASS == 3) {
      tmap_prefetch(&tma_lo);
      tmap_prefetch(&tmb_lo);
    }
  }
  if (warp == 5) tmem_alloc(slot_u32, BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  if (warp == 4) {
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
        mbar_expect_tx(bar_full + 8 * s, C::STAGE_BYTES);
        tma_load_2d(st, &tma_hi, bar_full + 8 * s, x, m_tile * BM);
        tma_load_2d(st + C::PLANES * C::A_BYTES, &tmb_hi, bar_full + 8 * s, x, n_tile * BN);
        if (NPASS == 3) {
          tma_load_2d(st + C::A_BYTES, &tma_lo, bar_full + 8 * s, x, m_tile * BM);
          tma_load_2d(st + C::PLANES * C::A_BYTES + C::B_BYTES, &tmb_lo, bar_full + 8 * s, x,
                      n_tile * BN);
        }
        ++issued;
      }
      if (!ok) {
        atomicOr(ep.err, OFA_ERRBIT_TIMEOUT);
        abort_flag = 1;
      }
      // Drain: every issued copy must have landed before the CTA may exit.
      for (int kb = max(0, issued - C::STAGES); kb < issued; ++kb)
        if (!mbar_wait(bar_full + 8 * (kb % C::STAGES), (kb / C::STAGES) & 1)) {
          atomicOr(ep.err, OFA_ERRBIT_TIMEOUT);
          break;
        }
    }
  } else if (warp == 5) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % C::STAGES;
        if (!mbar_wait(bar_full + 8 * s, (kb / C::STAGES) & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t st = base_u32 + s * C::STAGE_BYTES;
        const uint64_t a_hi = sdesc_sw128(st);
        const uint64_t a_lo = sdesc_sw128(st + C::A_BYTES);
        const uint64_t b_hi = sdesc_sw128(st + C::PLANES * C::A_BYTES);
        const uint64_t b_lo = sdesc_sw128(st + C::PLANES * C::A_BYTES + C::B_BYTES);
#pragma unroll
        for (int kk = 0; kk < C::UMMA_K_STEPS; ++kk) {
          const uint64_t adv = (uint64_t)((kk * 32) >> 4);  // 32 bytes of K per MMA
          umma<KIND>(tmem, a_hi + adv, b_hi + adv, C::IDESC, (kb | kk) != 0);
          if (NPASS == 3) {
            umma<KIND>(tmem, a_hi + adv, b_lo + adv, C::IDESC, 1);
            umma<KIND>(tmem, a_lo + adv, b_hi + adv, C::IDESC, 1);
          }
        }
        umma_commit(bar_empty + 8 * s);  // stage free once these MMAs have read it
      }
      if (!ok) {
        atomicOr(ep.err, OFA_ERRBIT_TIMEOUT);
        abort_flag = 1;
      }
      umma_commit(bar_accum);  // accumulator complete (or drained, on abort)
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const bool ready = mbar_wait(bar_accum, 0);
    tc_fence_after();
    if (!ready) atomicOr(ep.err, OFA_ERRBIT_TIMEOUT);
    const bool valid = ready && nkb > 0;
    const int r = warp * 32 + lane;               // accumulator row = TMEM lane
    const int n = m_tile * BM + r;                // pupil row
    const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);

    if (EPI == EPI_FWD) {
      float* red = reinterpret_cast<float*>(base + C::STAGES * C::STAGE_BYTES);
#pragma unroll 1
      for (int ch = 0; ch < BN / 32; ++ch) {
        uint32_t v[32];
        float p[32];
        if (valid) {
          tmem_ld32(tw + ch * 32, v);
          const int kbase = (n_tile * BN + ch * 32) >> 1;   // 16 foci in this chunk
          const float4* fr = reinterpret_cast<const float4*>(ep.fyT + (size_t)n * ep.kp + kbase);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 f = __ldg(fr + q);
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
        red[warp * BN + ch * 32 + lane] = warp_reduce_scatter32(p);
      }
      named_bar_epi();
      const int t = threadIdx.x;  // 0..127
      float* dst = ep.part + (size_t)(split * ep.tiles_m + m_tile) * 2 * ep.kp + n_tile * BN;
      for (int col = t; col < BN; col += 128)
        dst[col] = ((red[col] + red[BN + col]) + red[2 * BN + col]) + red[3 * BN + col];
    } else {
      // Per-pixel work (thread = row); global loads and stores are staged through
      // shared memory (the operand stages are free once the accumulator is
      // complete) so that every warp-wide access covers whole 64-byte row segments.
      uint8_t* wb = base + warp * 16384;
      float* s_a = reinterpret_cast<float*>(wb);      // [32][17] amplitude
      float* s_p = s_a + 32 * 17;                     // [32][17] phase in (gradient)
      float* s_o = s_p + 32 * 17;                     // [32][17] phase / gradient out
      uint2* s_h = reinterpret_cast<uint2*>(s_o + 32 * 17);  // [32][17] field, hi bits
      uint2* s_l = s_h + 32 * 17;                     // [32][17] field, lo bits
      const int nbase = m_tile * BM + warp * 32;
      const int lr = lane >> 4, lc = lane & 15;
      const bool wide = ep.prec == OFA_PREC_TF32;
      float factor = 0.f;
      if (EPI == EPI_GRAD) factor = 2.f * ep.amp_factor / ep.st->c_scale;
#pragma unroll 1
      for (int ch = 0; ch < BN / 32; ++ch) {
        uint32_t v[32];
        if (!valid) break;
        tmem_ld32(tw + ch * 32, v);
        const int mbase = (n_tile * BN + ch * 32) >> 1;   // 16 pupil columns
        const int gm = mbase + lc;
        __syncwarp();
#pragma unroll 4
        for (int it = 0; it < 16; ++it) {
          const int row = 2 * it + lr, gn = nbase + row;
          const bool ok = gn < ep.ny && gm < ep.nx;
          const size_t idx = (size_t)gn * ep.nx + gm;
          s_a[row * 17 + lc] = ok ? ep.amp[idx] : 0.f;
          if (EPI == EPI_GRAD) s_p[row * 17 + lc] = ok ? ep.phi_in[idx] : 0.f;
        }
        __syncwarp();
#pragma unroll 4
        for (int q = 0; q < 16; ++q) {
          const float re = __uint_as_float(v[2 * q]), im = __uint_as_float(v[2 * q + 1]);
          const float a = s_a[lane * 17 + q];
          if (EPI == EPI_BWD) {
            // phi = arg(E') (atan2(0,0) = 0), then the next pupil field A exp(i phi),
            // formed exactly as the field-plane builder forms it from a stored phi
            const float ph = atan2f(im, re);
            s_o[lane * 17 + q] = ph;
            float sn, cs;
            __sincosf(ph, &sn, &cs);
            uint2 h, l;
            split_pack(ep.prec, a * cs, a * sn, h, l);
            s_h[lane * 17 + q] = h;
            s_l[lane * 17 + q] = l;
          } else {
            float sn, cs;
            sincosf(s_p[lane * 17 + q], &sn, &cs);
            s_o[lane * 17 + q] = factor * a * (cs * im - sn * re);
          }
        }
        __syncwarp();
#pragma unroll 4
        for (int it = 0; it < 16; ++it) {
          const int row = 2 * it + lr, gn = nbase + row;
          if (gn >= ep.ny || gm >= ep.nx) continue;
          ep.out[(size_t)gn * ep.nx + gm] = s_o[row * 17 + lc];
          if (EPI == EPI_BWD) {
            const size_t e = (size_t)gn * ep.nxp + gm;   // complex element index
            const uint2 h = s_h[row * 17 + lc];
            if (wide) {
              reinterpret_cast<uint2*>(ep.e_hi)[e] = h;
            } else {
              reinterpret_cast<uint32_t*>(ep.e_hi)[e] = h.x;
              if (ep.e_lo) reinterpret_cast<uint32_t*>(ep.e_lo)[e] = s_l[row * 17 + lc].x;
            }
          }
        }
      }
    }
  }

  // ------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, BN);
  }
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
            uint32_t box_rows, std::string& err) {
  auto fn = encode_fn();
  if (fn == nullptr) {
    err = "cuTensorMapEncodeTiled is not available from the driver";
    return false;
  }
  const CUtensorMapDataType dt =
      elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * (cuuint64_t)elem_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / elem_bytes), box_rows};
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

template <int KIND, int NPASS, int BN, int EPI>
void launch_cfg(const TcOperands& t, const CUtensorMap& a_hi, const CUtensorMap& a_lo,
                const CUtensorMap& b_hi, const CUtensorMap& b_lo, dim3 grid, int kb_per_split,
                int kb_total, const EpiArgs& ep, const int* done, cudaStream_t s) {
  using C = Cfg<KIND, NPASS, BN, EPI>;
  umma_gemm_kernel<KIND, NPASS, BN, EPI><<<grid, NTHREADS, C::SMEM, s>>>(
      a_hi, a_lo, b_hi, b_lo, kb_per_split, kb_total, ep, done);
}

template <int EPI, int BN>
void dispatch_prec(int prec, const TcOperands& t, const CUtensorMap& a_hi,
                   const CUtensorMap& a_lo, const CUtensorMap& b_hi, const CUtensorMap& b_lo,
                   dim3 grid, int kbps, int kbt, const EpiArgs& ep, const int* done,
                   cudaStream_t s) {
  switch (prec) {
    case OFA_PREC_TF32:
      launch_cfg<KIND_TF32, 1, BN, EPI>(t, a_hi, a_lo, b_hi, b_lo, grid, kbps, kbt, ep, done, s);
      break;
    case OFA_PREC_BF16:
      launch_cfg<KIND_BF16, 1, BN, EPI>(t, a_hi, a_lo, b_hi, b_lo, grid, kbps, kbt, ep, done, s);
      break;
    case OFA_PREC_BF16X3:
      launch_cfg<KIND_BF16, 3, BN, EPI>(t, a_hi, a_lo, b_hi, b_lo, grid, kbps, kbt, ep, done, s);
      break;
    case OFA_PREC_F16X3:
      launch_cfg<KIND_F16, 3, BN, EPI>(t, a_hi, a_lo, b_hi, b_lo, grid, kbps, kbt, ep, done, s);
      break;
    default:
      break;
  }
}

template <int EPI>
void dispatch(int prec, int bn, const TcOperands& t, const CUtensorMap& a_hi,
              const CUtensorMap& a_lo, const CUtensorMap& b_hi, const CUtensorMap& b_lo,
              dim3 grid, int kbps, int kbt, const EpiArgs& ep, const int* done, cudaStream_t s) {
  if (bn == 128)
    dispatch_prec<EPI, 128>(prec, t, a_hi, a_lo, b_hi, b_lo, grid, kbps, kbt, ep, done, s);
  else
    dispatch_prec<EPI, 256>(prec, t, a_hi, a_lo, b_hi, b_lo, grid, kbps, kbt, ep, done, s);
}

template <int KIND, int NPASS>
cudaError_t set_attrs() {
  cudaError_t e = cudaSuccess;
  auto one = [&](auto kern, int bytes) {
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (r != cudaSuccess) e = r;
  };
  one(umma_gemm_kernel<KIND, NPASS, 128, EPI_FWD>, Cfg<KIND, NPASS, 128, EPI_FWD>::SMEM);
  one(umma_gemm_kernel<KIND, NPASS, 256, EPI_FWD>, Cfg<KIND, NPASS, 256, EPI_FWD>::SMEM);
  one(umma_gemm_kernel<KIND, NPASS, 128, EPI_BWD>, Cfg<KIND, NPASS, 128, EPI_BWD>::SMEM);
  one(umma_gemm_kernel<KIND, NPASS, 256, EPI_BWD>, Cfg<KIND, NPASS, 256, EPI_BWD>::SMEM);
  one(umma_gemm_kernel<KIND, NPASS, 128, EPI_GRAD>, Cfg<KIND, NPASS, 128, EPI_GRAD>::SMEM);
  one(umma_gemm_kernel<KIND, NPASS, 256, EPI_GRAD>, Cfg<KIND, NPASS, 256, EPI_GRAD>::SMEM);
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
  switch (prec) {
    case OFA_PREC_TF32: return set_attrs<KIND_TF32, 1>();
    case OFA_PREC_BF16: return set_attrs<KIND_BF16, 1>();
    case OFA_PREC_BF16X3: return set_attrs<KIND_BF16, 3>();
    case OFA_PREC_F16X3: return set_attrs<KIND_F16, 3>();
    default: return cudaSuccess;
  }
}

bool tc_encode_maps(ofa_plan* p, TcOperands& t, std::string& err) {
  const int eb = t.elem_bytes;
  const uint64_t e_cols = 2 * (uint64_t)p->nxp, k_cols = 2 * (uint64_t)p->kp;
  bool ok = true;
  ok = ok && encode(&t.tm_e_hi, t.e_hi, eb, e_cols, p->nyp, BM, err);
  ok = ok && encode(&t.tm_bx_hi, t.bx_hi, eb, e_cols, 2 * (uint64_t)p->kp, t.fwd_bn, err);
  ok = ok && encode(&t.tm_p_hi, t.p_hi, eb, k_cols, p->nyp, BM, err);
  ok = ok && encode(&t.tm_q_hi, t.q_hi, eb, k_cols, 2 * (uint64_t)p->nxp, t.bwd_bn, err);
  if (t.npass == 3) {
    ok = ok && encode(&t.tm_e_lo, t.e_lo, eb, e_cols, p->nyp, BM, err);
    ok = ok && encode(&t.tm_bx_lo, t.bx_lo, eb, e_cols, 2 * (uint64_t)p->kp, t.fwd_bn, err);
    ok = ok && encode(&t.tm_p_lo, t.p_lo, eb, k_cols, p->nyp, BM, err);
    ok = ok && encode(&t.tm_q_lo, t.q_lo, eb, k_cols, 2 * (uint64_t)p->nxp, t.bwd_bn, err);
  } else {
    t.tm_e_lo = t.tm_e_hi;
    t.tm_bx_lo = t.tm_bx_hi;
    t.tm_p_lo = t.tm_p_hi;
    t.tm_q_lo = t.tm_q_hi;
  }
  return ok;
}

void launch_fwd_tc(ofa_plan* p, const TcOperands& t, const int* done, cudaStream_t s) {
  const int kb_total = (2 * p->nxp * t.elem_bytes) / ROW_BYTES;
  const int kbps = (kb_total + t.fwd_split - 1) / t.fwd_split;
  dim3 grid((2 * p->kp) / t.fwd_bn, p->nyp / BM, t.fwd_split);
  EpiArgs ep = base_args(p);
  dispatch<EPI_FWD>(p->precision, t.fwd_bn, t, t.tm_e_hi, t.tm_e_lo, t.tm_bx_hi, t.tm_bx_lo, grid,
                    kbps, kb_total, ep, done, s);
}

void launch_bwd_tc(ofa_plan* p, const TcOperands& t, const int* done, cudaStream_t s) {
  const int kb_total = (2 * p->kp * t.elem_bytes) / ROW_BYTES;
  dim3 grid((2 * p->nxp) / t.bwd_bn, p->nyp / BM, 1);
  EpiArgs ep = base_args(p);
  ep.out = p->phi;
  ep.e_hi = t.e_hi;
  ep.e_lo = t.e_lo;
  dispatch<EPI_BWD>(p->precision, t.bwd_bn, t, t.tm_p_hi, t.tm_p_lo, t.tm_q_hi, t.tm_q_lo, grid,
                    kb_total, kb_total, ep, done, s);
}

void launch_grad_tc(ofa_plan* p, const TcOperands& t, const float* phi, float scale_unused,
                    float* grad, cudaStream_t s) {
  (void)scale_unused;
  const int kb_total = (2 * p->kp * t.elem_bytes) / ROW_BYTES;
  dim3 grid((2 * p->nxp) / t.bwd_bn, p->nyp / BM, 1);
  EpiArgs ep = base_args(p);
  ep.out = grad;
  ep.phi_in = phi;
  dispatch<EPI_GRAD>(p->precision, t.bwd_bn, t, t.tm_p_hi, t.tm_p_lo, t.tm_q_hi, t.tm_q_lo, grid,
                     kb_total, kb_total, ep, nullptr, s);
}
