// Separable grid form of one loop iteration in three launches (FP32, CUDA cores).
//
// With the foci on the grid of their U_x distinct x and U_y distinct y values, Eq. 2 at
// focus k = (ix_k, iy_k) is Theta_k = sum_n Fyu[iy_k][n] G[n][ix_k] with the first
// product G[n][ix] = sum_m E[n][m] Fxu[ix][m], and the adjoint factors the same way:
// E'[n][m] = sum_iy conj(Fyu[iy][n]) T[iy][m], T[iy][m] = sum_ix C[iy][ix] conj(Fxu[ix][m])
// with C the focused field c laid out on the grid (zero where the grid has no focus).
//
//   sep_fwd_kernel        block b: pupil rows [b R, b R + R), 512 threads in two groups
//                         of 256, each over half of the rows.  A thread holds E of its
//                         rows at 4 pixel columns in registers; the rows of Fxu stream
//                         through a block-wide cp.async ring four grid columns at a time;
//                         the per-thread G contributions are summed by a warp
//                         reduce-scatter and then over the group's 8 warps in order.  The
//                         block writes its partial Theta row (sum over its rows); for
//                         K <= 512 the last block to finish sums the rows and runs the
//                         focal step (no second launch).
//   sep_sum_focal_kernel  32 foci per block: the partial rows summed in fixed order into
//                         Theta; the block that finishes last runs the focal step
//   sep_inv_kernel        tile of 32 pixel columns x 256 pupil rows, 512 threads: C
//                         gathered from c, T for the tile's columns, the rank-U_y product
//                         (16 rows per warp, a lane per column), phi = arg E' and the next
//                         field A exp(i phi), formed as A E' / |E'|
//
// The three kernels are launched as programmatic dependents: each stages the operands
// that do not change over the loop (Fxu, Fyu, the grid map, A) while the kernel before
// it finishes, and waits for that kernel only before it reads what it produced.
//
// Every sum runs in a fixed order, so runs and resumes are bitwise reproducible.
#include <type_traits>

#include "ofa_focal.cuh"
#include "ofa_internal.cuh"
#include "ofa_math.cuh"
#include "umma_ptx.cuh"

namespace {

using ofa_ptx::pdl_launch_dependents;
using ofa_ptx::pdl_wait;

constexpr int SEP_THREADS = 256;  // the sum kernel
constexpr int SEP_WARPS = SEP_THREADS / 32;
constexpr int SEP_MAX_R = 8;      // pupil rows per forward block
constexpr int FWD_THREADS = 512;  // two groups of 256, each over half of the block's rows
constexpr int FWD_GROUP = 256;
constexpr int FWD_WARPS = FWD_THREADS / 32;
constexpr int FWD_MT = 4;         // pixel columns per forward thread: nx <= 1024
constexpr int FWD_STAGES = 3;     // quads of Fxu rows in the ring
constexpr int INV_THREADS = 512;
constexpr int INV_WARPS = INV_THREADS / 32;
constexpr int INV_COLS = 32;      // pixel columns of an inverse tile (a lane each)
constexpr int INV_ROWS = 256;     // pupil rows of an inverse tile (16 per warp)
constexpr int INV_RPW = INV_ROWS / INV_WARPS;
constexpr int INV_MAX_UY = 64;    // grid rows the inverse's T accumulators cover
constexpr size_t SEP_SMEM_LIMIT = 200 * 1024;   // dynamic shared memory of either kernel

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) b
__device__ __forceinline__ void cmac_conj(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

// 8-byte asynchronous copy global -> shared; with valid == false the destination is
// zero-filled and nothing is read (src must still be a valid address).
__device__ __forceinline__ void cp_async8(float2* dst, const float2* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// 16-byte copy through L2 only (both addresses 16-byte aligned; used also for data
// other blocks of this launch wrote); with valid == false the destination is
// zero-filled and nothing is read
__device__ __forceinline__ void cp_async16_cg(void* dst, const void* src, bool valid = true) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Butterfly reduce-scatter of 32 values over the 32 lanes: afterwards lane l holds
// the warp-wide sum of element l (31 shuffles for 32 sums, fixed order).
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
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

// Shared memory of the forward: the Fxu ring [FWD_STAGES][4][FWD_MT][FWD_GROUP], the
// per-warp sums [nquad][FWD_WARPS][32], G [R][ux] and the block's Fyu columns [uy][R].
constexpr size_t FWD_SLOT = (size_t)4 * FWD_MT * FWD_GROUP;
constexpr size_t FWD_RING = (size_t)FWD_STAGES * FWD_SLOT;

// Fxu rows 4q .. 4q + 3 into ring slot q % FWD_STAGES, all columns (element (c, j, t)
// is Fxu[4q + c][t + 256 j]), as one cp.async group of the calling thread; past the
// last quad the group is empty, which keeps the group count uniform.
__device__ __forceinline__ void fwd_issue(float2* ring, const float2* __restrict__ fxu, int ux,
                                          int nx, int q, int tid) {
  if (q < ((ux + 3) >> 2)) {
    float2* dst = ring + (size_t)(q % FWD_STAGES) * FWD_SLOT;
#pragma unroll
    for (int i = 0; i < (int)(FWD_SLOT / FWD_THREADS); ++i) {
      const int idx = tid + i * FWD_THREADS;
      const int c = idx / (FWD_MT * FWD_GROUP);
      const int m = idx % (FWD_MT * FWD_GROUP);   // = t' + 256 j'
      const int ix = 4 * q + c;
      const bool ok = ix < ux && m < nx;
      cp_async8(dst + idx, ok ? fxu + (size_t)ix * nx + m : fxu, ok);
    }
  }
  cp_async_commit();
}

// E of this thread's pupil rows n0 + g RT + r at the columns t + 256 j (zero outside).
template <int RT>
__device__ __forceinline__ void fwd_load_e(float2 (&e)[RT][FWD_MT], const float2* __restrict__ e32,
                                           int nx, int n0, int rows, int tid) {
  const int g = tid / FWD_GROUP, t = tid % FWD_GROUP;
  const int rows_g = max(0, min(RT, rows - g * RT));
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int j = 0; j < FWD_MT; ++j) {
      const int m = t + j * FWD_GROUP;
      e[r][j] = (r < rows_g && m < nx) ? __ldcg(e32 + (size_t)(n0 + g * RT + r) * nx + m)
                                       : make_float2(0.f, 0.f);
    }
}

// G of the block's R pupil rows into gs [R][ux]: E in registers, Fxu streamed through
// the ring (this thread has issued quads 0 .. FWD_STAGES - 2), each thread's
// contributions summed by a warp reduce-scatter into red, then over the 8 warps of the
// row's group in order.  Ends with a block barrier after gs is complete.
template <int RT>
__device__ __forceinline__ void fwd_g(const float2 (&e)[RT][FWD_MT], float2* ring, float* red,
                                      float2* gs, const float2* __restrict__ fxu, int ux, int nx,
                                      int R, int tid) {
  const int lane = tid & 31, warp = tid >> 5, t = tid % FWD_GROUP;
  const int nquad = (ux + 3) >> 2;
  for (int q = 0; q < nquad; ++q) {
    cp_async_wait<FWD_STAGES - 2>();   // this thread's copies of quad q have landed
    __syncthreads();                   // everyone's have; slot (q - 1) % S is free
    fwd_issue(ring, fxu, ux, nx, q + FWD_STAGES - 1, tid);
    const float2* src = ring + (size_t)(q % FWD_STAGES) * FWD_SLOT;
    // v[8 c + 2 r + {0, 1}]: this thread's part of G[g RT + r][4q + c]
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int j = 0; j < FWD_MT; ++j) {
        const float2 fv = src[(c * FWD_MT + j) * FWD_GROUP + t];
#pragma unroll
        for (int r = 0; r < RT; ++r) {
          float2 a = make_float2(v[8 * c + 2 * r], v[8 * c + 2 * r + 1]);
          cmac(a, e[r][j], fv);
          v[8 * c + 2 * r] = a.x;
          v[8 * c + 2 * r + 1] = a.y;
        }
      }
    red[((size_t)q * FWD_WARPS + warp) * 32 + lane] = reduce_scatter32(v, lane);
  }
  __syncthreads();
  for (int i = tid; i < R * ux; i += FWD_THREADS) {
    const int r = i / ux, ix = i - r * ux;
    const int gr = r / RT, rr = r - gr * RT;
    const int el = (ix & 3) * 8 + 2 * rr;
    const float* sp = red + ((size_t)(ix >> 2) * FWD_WARPS + gr * (FWD_GROUP / 32)) * 32;
    float2 gv = make_float2(0.f, 0.f);
#pragma unroll
    for (int w = 0; w < FWD_GROUP / 32; ++w) {
      gv.x += sp[w * 32 + el];
      gv.y += sp[w * 32 + el + 1];
    }
    gs[i] = gv;
  }
  __syncthreads();
}

// Block: pupil rows [n0, n0 + R), R <= 2 RT; thread (group g, t) holds E of rows
// n0 + g RT + [0, RT) at the columns t + 256 j, j < 4.  With f.on, the block that
// finishes last also sums the partial rows (staged in the idle ring) into Theta and
// runs the focal step (K <= FWD_THREADS).
template <int RT>
__global__ void __launch_bounds__(FWD_THREADS, 1) sep_fwd_kernel(
    const float2* __restrict__ e32, const float2* __restrict__ fxu,
    const float2* __restrict__ fyu, const int2* __restrict__ ixy, int nx, int ny, int ux, int uy,
    int K, int kp, int R, float2* __restrict__ part, const int* __restrict__ done, FocalTail f) {
  pdl_launch_dependents();
  extern __shared__ float4 sep_smem4[];
  float2* ring = reinterpret_cast<float2*>(sep_smem4);
  const int nquad = (ux + 3) >> 2;
  float* red = reinterpret_cast<float*>(ring + FWD_RING);                         // [nquad][16][32]
  float2* gs = reinterpret_cast<float2*>(red + (size_t)nquad * FWD_WARPS * 32);   // [R][ux]
  float2* fs = gs + (size_t)R * ux;                                                // [uy][R]
  const int tid = threadIdx.x;
  const int n0 = blockIdx.x * R;
  const int rows = min(R, ny - n0);

#pragma unroll
  for (int q = 0; q < FWD_STAGES - 1; ++q) fwd_issue(ring, fxu, ux, nx, q, tid);
  for (int i = tid; i < uy * R; i += FWD_THREADS) {
    const int iy = i / R, r = i - iy * R;
    fs[i] = r < rows ? __ldg(fyu + (size_t)iy * ny + n0 + r) : make_float2(0.f, 0.f);
  }
  // grid indices of this thread's first foci
  constexpr int KR = 4;
  int2 xyr[KR];
#pragma unroll
  for (int i = 0; i < KR; ++i) {
    const int k = tid + i * FWD_THREADS;
    xyr[i] = k < K ? __ldg(ixy + k) : make_int2(0, 0);
  }

  pdl_wait();   // E and the stop flag come from the kernels before this one
  const int stop = done != nullptr ? __ldcg(done) : 0;
  float2 e[RT][FWD_MT];
  fwd_load_e<RT>(e, e32, nx, n0, rows, tid);   // all loads in flight together
  if (stop) {
    cp_async_wait<0>();   // no copy may land after the block has left
    return;
  }
  fwd_g<RT>(e, ring, red, gs, fxu, ux, nx, R, tid);
  // this block's partial Theta: sum over its rows of Fyu[iy_k][n] G[n][ix_k]
  float2* dst = part + (size_t)blockIdx.x * kp;
#pragma unroll
  for (int i = 0; i < KR; ++i) {
    const int k = tid + i * FWD_THREADS;
    if (k >= kp) break;
    float2 a = make_float2(0.f, 0.f);
    if (k < K)
      for (int r = 0; r < R; ++r) cmac(a, fs[xyr[i].y * R + r], gs[r * ux + xyr[i].x]);
    dst[k] = a;
  }
  for (int k = tid + KR * FWD_THREADS; k < kp; k += FWD_THREADS) {
    float2 a = make_float2(0.f, 0.f);
    if (k < K) {
      const int2 xy = __ldg(ixy + k);
      for (int r = 0; r < R; ++r) cmac(a, fs[xy.y * R + r], gs[r * ux + xy.x]);
    }
    dst[k] = a;
  }
  if (!f.on) return;

  // the last block: Theta = sum of the partial rows in order, then the focal step
  __shared__ int last;
  __shared__ float focal_sh[4 * 33 + 4];
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    last = atomicAdd(f.counter, 1u) == gridDim.x - 1;
    if (last) {
      __threadfence();
      *f.counter = 0u;
    }
  }
  __syncthreads();
  if (!last) return;
  const int nb = gridDim.x, k2 = (K + 1) >> 1;   // 16-byte pairs of foci per row
  float2* ps = ring;                               // [nb][2 k2]
  for (int i = tid; i < nb * k2; i += FWD_THREADS) {
    const int p = i / k2, j = i - p * k2;
    cp_async16_cg(ps + 2 * i, part + (size_t)p * kp + 2 * j);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  if (tid < K) {
    float2 a = ps[tid];
    for (int p = 1; p < nb; ++p) {
      const float2 v = ps[(size_t)p * 2 * k2 + tid];
      a.x += v.x;
      a.y += v.y;
    }
    part[tid] = a;   // Theta over partial row 0
  }
  __syncthreads();
  ofa_focal::iterate_regs<FWD_THREADS, 1>(part, 1, K, kp, f.t, f.w, f.c, f.hist, f.st,
                                          f.weighting, focal_sh, tid, ofa_focal::BarBlock());
}

// Theta_k = sum over the nb partial rows in order; with focal != 0 the last block to
// finish runs the focal step of the loop on Theta.
__global__ void __launch_bounds__(SEP_THREADS) sep_sum_focal_kernel(
    const float2* __restrict__ part, int nb, int K, int kp, float2* __restrict__ theta,
    int focal, const float* __restrict__ t, float* __restrict__ w, float2* __restrict__ c,
    double* __restrict__ hist, OfaDevState* __restrict__ st, int weighting,
    unsigned* __restrict__ counter, const int* __restrict__ done) {
  pdl_launch_dependents();
  __shared__ float2 red[SEP_WARPS][32];
  __shared__ float focal_sh[4 * 33 + 4];
  __shared__ int last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = blockIdx.x * 32 + lane;
  pdl_wait();
  if (done != nullptr && __ldcg(done)) return;
  // warp w sums rows w, w + 8, ...; U rows of loads in flight at a time
  constexpr int U = 24;
  float2 a = make_float2(0.f, 0.f);
  if (k < K)
    for (int p0 = warp; p0 < nb; p0 += SEP_WARPS * U) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int p = p0 + u * SEP_WARPS;
        v[u] = p < nb ? __ldcg(part + (size_t)p * kp + k) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (p0 + u * SEP_WARPS < nb) {
          a.x += v[u].x;
          a.y += v[u].y;
        }
    }
  red[warp][lane] = a;
  __syncthreads();
  if (tid < 32 && k < K) {
    float2 s = red[0][tid];
#pragma unroll
    for (int q = 1; q < SEP_WARPS; ++q) {
      s.x += red[q][tid].x;
      s.y += red[q][tid].y;
    }
    theta[k] = s;
  }
  if (!focal) return;
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
    if (last) {
      __threadfence();
      *counter = 0u;
    }
  }
  __syncthreads();
  if (!last) return;
  if (K <= SEP_THREADS * 4)
    ofa_focal::iterate_regs<SEP_THREADS, 4>(theta, 1, K, kp, t, w, c, hist, st, weighting,
                                            focal_sh, tid, ofa_focal::BarBlock());
  else if (K <= SEP_THREADS * 16)
    ofa_focal::iterate_regs<SEP_THREADS, 16>(theta, 1, K, kp, t, w, c, hist, st, weighting,
                                             focal_sh, tid, ofa_focal::BarBlock());
  else
    ofa_focal::iterate<SEP_THREADS>(theta, K, kp, t, w, c, hist, st, weighting, focal_sh, tid,
                                    ofa_focal::BarBlock());
}

// Separable form on the tensor cores, Theta from the forward's product G (contraction
// parts [parts][ux][ny], parts <= TCT_MAX_PARTS): warp w of block (ix, g) takes grid row
// iy = 16 g + w and loads its Fy_u row into registers (lane + 32 u: TCT_FV values, the
// rows of one chunk) before it waits for the forward; the block then sums the parts of
// column ix in fixed order into shared memory (chunks of TCT_CHUNK rows, all parts of a
// row loaded before any is added), each warp forms T[iy][ix] = sum_n Fy_u[iy][n] G[n][ix]
// from registers and shared memory (fixed shuffle tree) and writes Theta_k = T at the
// focus of that grid point (every focus sits on one).  The blocks also copy the weights
// to wprev, which the focal step reads while it writes the new ones.
constexpr int TCT_THREADS = 512, TCT_WARPS = TCT_THREADS / 32, TCT_FV = 32;
constexpr int TCT_CHUNK = 32 * TCT_FV;   // rows per chunk (one Fy_u value per lane and u)
constexpr int TCT_MAX_PARTS = 16;
static_assert(TCT_MAX_PARTS >= SEP_TC_MAX_PARTS, "the forward's parts must fit the part sum");
__global__ void __launch_bounds__(TCT_THREADS) sep_tc_theta_kernel(
    const float2* __restrict__ gt, int parts, const float2* __restrict__ fyu,
    const int* __restrict__ gridk, int ny, int ux, int uy, int K, float2* __restrict__ theta,
    const float* __restrict__ w, float* __restrict__ wprev, const int* __restrict__ done) {
  pdl_launch_dependents();
  __shared__ float2 g[TCT_CHUNK];
  __shared__ int skip;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, ix = blockIdx.x;
  const int iy = blockIdx.y * TCT_WARPS + warp;
  const float2* fr = fyu + (size_t)min(iy, uy - 1) * ny;
  auto load_fv = [&](float2 (&fv)[TCT_FV], int n0) {
#pragma unroll
    for (int u = 0; u < TCT_FV; ++u) {
      const int i = n0 + u * 32 + lane;
      fv[u] = iy < uy && i < ny ? __ldg(fr + i) : make_float2(0.f, 0.f);
    }
  };
  float2 fv[TCT_FV];
  load_fv(fv, 0);   // constant over the loop: before the wait
  pdl_wait();
  if (tid == 0) skip = done != nullptr && __ldcg(done);
  __syncthreads();
  if (skip) return;
  if (wprev != nullptr) {
    const int b = blockIdx.y * gridDim.x + blockIdx.x, nb = gridDim.x * gridDim.y;
    for (int k = b * TCT_THREADS + tid; k < K; k += nb * TCT_THREADS) wprev[k] = __ldcg(w + k);
  }
  const size_t slice = (size_t)ux * ny;
  const float2* col = gt + (size_t)ix * ny;
  float2 acc = make_float2(0.f, 0.f);
  for (int n0 = 0; n0 < ny; n0 += TCT_CHUNK) {
    const int nn = min(TCT_CHUNK, ny - n0);
    if (n0 > 0) load_fv(fv, n0);
    __syncthreads();  // the previous chunk is consumed
    for (int i = tid; i < nn; i += TCT_THREADS) {
      float2 v[TCT_MAX_PARTS];
#pragma unroll
      for (int z = 0; z < TCT_MAX_PARTS; ++z)
        v[z] = z < parts ? __ldcg(col + z * slice + n0 + i) : make_float2(0.f, 0.f);
      float2 a = v[0];
#pragma unroll
      for (int z = 1; z < TCT_MAX_PARTS; ++z)
        if (z < parts) {
          a.x += v[z].x;
          a.y += v[z].y;
        }
      g[i] = a;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TCT_FV; ++u) {
      const int i = u * 32 + lane;
      if (i < nn) cmac(acc, fv[u], g[i]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (iy < uy && lane == 0) {
    const int k = gridk[(size_t)iy * ux + ix];
    if (k >= 0) theta[k] = acc;
  }
}

// T for a tile's 32 pixel columns, then E' over the warp's INV_RPW rows and the
// projection.  fys: the tile's Fyu rows [uy][INV_ROWS] (16-byte aligned), fxs: its Fxu
// columns [ux][INV_COLS], cs: C on the grid [uy][ux], all complete in shared memory;
// ts: scratch [uy][INV_COLS]; av: this thread's amplitudes (rows n0 + 16 warp + i,
// column m0 + lane).  Writes phi = arg E' and the next field A E'/|E'| (= A e^{i phi};
// A where E' = 0).  Contains one block barrier.
__device__ __forceinline__ void inv_tile(const float2* fys, const float2* fxs, const float2* cs,
                                         float2* ts, const float (&av)[INV_RPW], int ux, int uy,
                                         int nx, int ny, int m0, int n0, float* __restrict__ phi,
                                         float2* __restrict__ e32, int tid) {
  const int lane = tid & 31, warp = tid >> 5;
  const int nw0 = n0 + warp * INV_RPW;   // this warp's first row
  // T[iy][m0 + lane] for iy = warp, warp + 16, ...: sum over ix in order of
  // C[iy][ix] conj(Fxu[ix][m])
  {
    constexpr int TI = INV_MAX_UY / INV_WARPS;
    float2 ta[TI];
#pragma unroll
    for (int i = 0; i < TI; ++i) ta[i] = make_float2(0.f, 0.f);
    for (int ix = 0; ix < ux; ++ix) {
      const float2 f = fxs[ix * INV_COLS + lane];
#pragma unroll
      for (int i = 0; i < TI; ++i) {
        const int iy = warp + i * INV_WARPS;
        if (iy < uy) cmac_conj(ta[i], f, cs[iy * ux + ix]);
      }
    }
#pragma unroll
    for (int i = 0; i < TI; ++i) {
      const int iy = warp + i * INV_WARPS;
      if (iy < uy) ts[iy * INV_COLS + lane] = ta[i];
    }
  }
  __syncthreads();
  // E'[nw0 + i][m0 + lane] = sum over iy in order of conj(Fyu[iy][n]) T[iy][m]
  float2 acc[INV_RPW];
#pragma unroll
  for (int i = 0; i < INV_RPW; ++i) acc[i] = make_float2(0.f, 0.f);
  for (int iy = 0; iy < uy; ++iy) {
    const float2 tv = ts[iy * INV_COLS + lane];
    const float4* f4 =
        reinterpret_cast<const float4*>(fys + (size_t)iy * INV_ROWS + warp * INV_RPW);
#pragma unroll
    for (int i = 0; i < INV_RPW / 2; ++i) {
      const float4 q = f4[i];
      cmac_conj(acc[2 * i], make_float2(q.x, q.y), tv);
      cmac_conj(acc[2 * i + 1], make_float2(q.z, q.w), tv);
    }
  }
  const int m = m0 + lane;
  if (m >= nx) return;
  // projection; the pixels are independent, so their chains interleave
#pragma unroll
  for (int i = 0; i < INV_RPW; ++i) {
    const float ph = ofa_arg(acc[i].y, acc[i].x);   // arg(0) = 0
    const float r2 = acc[i].x * acc[i].x + acc[i].y * acc[i].y;
    const float sc = r2 > 0.f ? av[i] * rsqrtf(r2) : 0.f;
    const float2 ev = r2 > 0.f ? make_float2(sc * acc[i].x, sc * acc[i].y) : make_float2(av[i], 0.f);
    if (nw0 + i < ny) {
      const size_t o = (size_t)(nw0 + i) * nx + m;
      phi[o] = ph;
      e32[o] = ev;
    }
  }
}

// The tile's constant operands into shared memory, asynchronously (one commit group).
__device__ __forceinline__ void inv_stage_constants(float2* fys, float2* fxs,
                                                    const float2* __restrict__ fyu,
                                                    const float2* __restrict__ fxu, int ux,
                                                    int uy, int nx, int ny, int m0, int n0,
                                                    int tid, int nthreads) {
  for (int i = tid; i < uy * INV_ROWS; i += nthreads) {
    const int iy = i / INV_ROWS, n = n0 + (i - iy * INV_ROWS);
    cp_async8(fys + i, n < ny ? fyu + (size_t)iy * ny + n : fyu, n < ny);
  }
  for (int i = tid; i < ux * INV_COLS; i += nthreads) {
    const int ix = i / INV_COLS, m = m0 + (i - ix * INV_COLS);
    cp_async8(fxs + i, m < nx ? fxu + (size_t)ix * nx + m : fxu, m < nx);
  }
  cp_async_commit();
}

// Shared memory of the inverse: Fyu rows of the tile [uy][INV_ROWS] (first: 16-byte
// aligned for its paired loads), C [uy][ux], Fxu columns of the tile [ux][INV_COLS],
// T [uy][INV_COLS].
__global__ void __launch_bounds__(INV_THREADS, 1) sep_inv_kernel(
    const float2* __restrict__ c, const int* __restrict__ gridk, const float2* __restrict__ fxu,
    const float2* __restrict__ fyu, const float* __restrict__ amp, int nx, int ny, int ux,
    int uy, float* __restrict__ phi, float2* __restrict__ e32, const int* __restrict__ done) {
  pdl_launch_dependents();
  extern __shared__ float4 sep_smem4[];
  float2* fys = reinterpret_cast<float2*>(sep_smem4);
  float2* cs = fys + (size_t)uy * INV_ROWS;
  float2* fxs = cs + (size_t)uy * ux;
  float2* ts = fxs + (size_t)ux * INV_COLS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.x * INV_COLS, n0 = blockIdx.y * INV_ROWS;
  const int nw0 = n0 + warp * INV_RPW;
  inv_stage_constants(fys, fxs, fyu, fxu, ux, uy, nx, ny, m0, n0, tid, INV_THREADS);
  // the grid map (the focus index in the low word until c is known) and the
  // amplitudes of this thread's pixels
  for (int i = tid; i < uy * ux; i += INV_THREADS)
    cs[i] = make_float2(__int_as_float(__ldg(gridk + i)), 0.f);
  const int m = m0 + lane;
  float av[INV_RPW];
#pragma unroll
  for (int i = 0; i < INV_RPW; ++i)
    av[i] = (nw0 + i < ny && m < nx) ? __ldg(amp + (size_t)(nw0 + i) * nx + m) : 0.f;

  pdl_wait();   // c and the stop flag come from the kernel before this one
  const int stop = done != nullptr ? __ldcg(done) : 0;
  // C on the grid: each thread fills the entries it mapped above
  for (int i = tid; i < uy * ux; i += INV_THREADS) {
    const int k = __float_as_int(cs[i].x);
    cs[i] = k >= 0 ? __ldcg(c + k) : make_float2(0.f, 0.f);
  }
  cp_async_wait<0>();
  if (stop) return;
  __syncthreads();
  inv_tile(fys, fxs, cs, ts, av, ux, uy, nx, ny, m0, n0, phi, e32, tid);
}

// ---------------------------------------------------------------- persistent loop
// All iterations of an ofa_iterate call in one cooperative launch.  Block b owns pupil
// rows [b R, b R + R) for both products, and each thread keeps the pupil field E (and A)
// of its pixels in registers across iterations:
//   forward  the block's partial Theta row, as sep_fwd_kernel computes it;
//   barrier; block b sums the partial rows of a slice of the foci (a warp per focus, in
//   fixed order) into Theta; barrier;
//   focal    every block runs the focal step on Theta identically (block 0 alone writes
//            w, c, xi and the state);
//   inverse  the adjoint restricted to the block's rows factors through
//            U[n][ix] = sum_iy C[iy][ix] conj(Fyu[iy][n]) (R x U_x values per block):
//            E'[n][m] = sum_ix U[n][ix] conj(Fxu[ix][m]), with Fxu streamed through the
//            same ring as the forward and no cross-thread reduction; then the next
//            E = A E'/|E'| in registers (phi = arg E' and the stored field are written
//            on the last iteration, or on every one when a threshold can stop the loop).
// Two grid barriers per iteration; every wait gives up after one second
// (OFA_ERRBIT_TIMEOUT) and the block leaves.
constexpr int LOOP_KPR = 5;                       // foci per thread: K <= 2560
constexpr int LOOP_KMAX = LOOP_KPR * FWD_THREADS;

struct LoopLayout {
  size_t ring, red, gs, fs, us, cs, cl, wl, tl, gk, scr, total;
};
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline LoopLayout loop_layout(int R, int ux, int uy) {
  LoopLayout L;
  const int uxp = (ux + 3) & ~3;   // U padded to whole quads of grid columns
  size_t o = 0;
  L.ring = o; o = align16(o + sizeof(float2) * FWD_RING);
  L.red = o;  o = align16(o + sizeof(float) * (size_t)(uxp / 4) * FWD_WARPS * 32);
  L.gs = o;   o = align16(o + sizeof(float2) * (size_t)R * ux);
  L.fs = o;   o = align16(o + sizeof(float2) * (size_t)uy * R);
  L.us = o;   o = align16(o + sizeof(float2) * (size_t)R * uxp);
  L.cs = o;   o = align16(o + sizeof(float2) * (size_t)uy * ux);
  L.cl = o;   o = align16(o + sizeof(float2) * LOOP_KMAX);
  L.wl = o;   o = align16(o + sizeof(float) * LOOP_KMAX);
  L.tl = o;   o = align16(o + sizeof(float) * LOOP_KMAX);
  L.gk = o;   o = align16(o + sizeof(int) * (size_t)uy * ux);
  L.scr = o;  o = align16(o + sizeof(float) * 4 * FWD_WARPS);
  L.total = o;
  return L;
}

struct SepLoopArgs {
  const float2* fxu;
  const float2* fyu;
  const int2* ixy;
  const int* gridk;
  const float* amp;
  float2* e32;
  float* phi;
  float2* part;
  float2* theta;
  float2* c;
  const float* t;
  float* w;
  double* hist;
  OfaDevState* st;
  unsigned* bar;   // two counters, zero at launch
  double threshold;
  int nx, ny, ux, uy, K, kp, R, weighting, n_iter;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* q) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(q) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch: the block's writes are released by thread
// 0 (CTA barrier, then a gpu-scope fence and a release add), and the wait for all
// arrivals (the counter reaching target) is bounded.  Returns false when it gave up.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    int ok = 1;
    if (ld_acquire_gpu(bar) < target) {
      const uint64_t t0 = ofa_ptx::gtimer();
      while (ld_acquire_gpu(bar) < target) {
        __nanosleep(64);
        if (ofa_ptx::gtimer() - t0 > ofa_ptx::WAIT_NS) {
          ok = ld_acquire_gpu(bar) >= target;
          break;
        }
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Sum of one value per thread over the block in a fixed order (warp butterfly, then the
// warp partials in warp order); every thread receives the same bits.
__device__ __forceinline__ float loop_block_sum(float v, float* scr, int tid) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((tid & 31) == 0) scr[tid >> 5] = v;
  __syncthreads();
  float r = scr[0];
#pragma unroll
  for (int w = 1; w < FWD_WARPS; ++w) r += scr[w];
  return r;
}

// Two sums and a max of one value each per thread, in one round of the same fixed order.
__device__ __forceinline__ void loop_block_reduce3(float& s0, float& s1, float& mx, float* scr,
                                                   int tid) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  __syncthreads();
  if ((tid & 31) == 0) {
    scr[tid >> 5] = s0;
    scr[FWD_WARPS + (tid >> 5)] = s1;
    scr[2 * FWD_WARPS + (tid >> 5)] = mx;
  }
  __syncthreads();
  s0 = scr[0];
  s1 = scr[FWD_WARPS];
  mx = scr[2 * FWD_WARPS];
#pragma unroll
  for (int w = 1; w < FWD_WARPS; ++w) {
    s0 += scr[w];
    s1 += scr[FWD_WARPS + w];
    mx = fmaxf(mx, scr[2 * FWD_WARPS + w]);
  }
}

template <int RT>
__global__ void __launch_bounds__(FWD_THREADS, 1) sep_loop_kernel(SepLoopArgs a) {
  extern __shared__ float4 sep_smem4[];
  char* base = reinterpret_cast<char*>(sep_smem4);
  const LoopLayout L = loop_layout(a.R, a.ux, a.uy);
  float2* ring = reinterpret_cast<float2*>(base + L.ring);
  float* red = reinterpret_cast<float*>(base + L.red);
  float2* gs = reinterpret_cast<float2*>(base + L.gs);
  float2* fs = reinterpret_cast<float2*>(base + L.fs);
  float2* us = reinterpret_cast<float2*>(base + L.us);
  float2* cs = reinterpret_cast<float2*>(base + L.cs);
  float2* cl = reinterpret_cast<float2*>(base + L.cl);
  float* wl = reinterpret_cast<float*>(base + L.wl);
  float* tl = reinterpret_cast<float*>(base + L.tl);
  int* gk = reinterpret_cast<int*>(base + L.gk);
  float* scr = reinterpret_cast<float*>(base + L.scr);
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x, G = gridDim.x;
  const int nx = a.nx, ny = a.ny, ux = a.ux, uy = a.uy, K = a.K, R = a.R;
  const int uxp = (ux + 3) & ~3, nquad = uxp >> 2;
  if (tid == 0) s_ok = 1;
  const int g = tid / FWD_GROUP, t = tid % FWD_GROUP;
  const int n0 = b * R, rows = min(R, ny - n0);
  const int rows_g = max(0, min(RT, rows - g * RT));
  const bool writer = b == 0;

  // ---- constants and state, once per launch
#pragma unroll
  for (int q = 0; q < FWD_STAGES - 1; ++q) fwd_issue(ring, a.fxu, ux, nx, q, tid);
  for (int i = tid; i < uy * R; i += FWD_THREADS) {
    const int iy = i / R, r = i - iy * R;
    fs[i] = r < rows ? __ldg(a.fyu + (size_t)iy * ny + n0 + r) : make_float2(0.f, 0.f);
  }
  for (int i = tid; i < uy * ux; i += FWD_THREADS) gk[i] = __ldg(a.gridk + i);
  for (int k = tid; k < LOOP_KMAX; k += FWD_THREADS) {
    tl[k] = k < K ? __ldg(a.t + k) : 0.f;
    wl[k] = k < K ? __ldcg(a.w + k) : 0.f;
  }
  int2 xy[LOOP_KPR];
#pragma unroll
  for (int i = 0; i < LOOP_KPR; ++i) {
    const int k = tid + i * FWD_THREADS;
    xy[i] = k < K ? __ldg(a.ixy + k) : make_int2(0, 0);
  }
  float2 e[RT][FWD_MT];
  float av[RT][FWD_MT];
  fwd_load_e<RT>(e, a.e32, nx, n0, rows, tid);
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int j = 0; j < FWD_MT; ++j) {
      const int m = t + j * FWD_GROUP;
      av[r][j] = (r < rows_g && m < nx) ? __ldg(a.amp + (size_t)(n0 + g * RT + r) * nx + m)
                                        : 0.f;
    }
  const int h0 = __ldcg(&a.st->hist_count), j0 = __ldcg(&a.st->j);
  const int stop0 = __ldcg(&a.st->done);
  __syncthreads();
  if (stop0) {
    cp_async_wait<0>();
    return;
  }
  const bool thr_on = a.threshold > 0.0 && a.threshold < 1.0;
  const int fpb = (K + G - 1) / G;   // foci whose partial rows this block sums

  for (int it = 0; it < a.n_iter; ++it) {
    const unsigned target = (unsigned)(it + 1) * (unsigned)G;
    // ---- forward: this block's partial Theta row
    fwd_g<RT>(e, ring, red, gs, a.fxu, ux, nx, R, tid);
#pragma unroll
    for (int i = 0; i < LOOP_KPR; ++i) {
      const int k = tid + i * FWD_THREADS;
      if (k < a.kp) {
        float2 acc = make_float2(0.f, 0.f);
        if (k < K)
          for (int r = 0; r < R; ++r) cmac(acc, fs[xy[i].y * R + r], gs[r * ux + xy[i].x]);
        a.part[(size_t)b * a.kp + k] = acc;
      }
    }
    // the inverse pass streams the same Fxu quads again
#pragma unroll
    for (int q = 0; q < FWD_STAGES - 1; ++q) fwd_issue(ring, a.fxu, ux, nx, q, tid);
    if (!grid_barrier(a.bar + 0, target, &s_ok)) break;
    // ---- Theta_k for this block's foci: warp per focus, lanes over the rows in order
    for (int kk = warp; kk < fpb; kk += FWD_WARPS) {
      const int k = b * fpb + kk;
      if (k >= K) break;
      float2 acc = make_float2(0.f, 0.f);
      for (int p = lane; p < G; p += 32) {
        const float2 v = __ldcg(a.part + (size_t)p * a.kp + k);
        acc.x += v.x;
        acc.y += v.y;
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) a.theta[k] = acc;
    }
    if (!grid_barrier(a.bar + 1, target, &s_ok)) break;
    // ---- focal step (Algorithm 1), identical in every block
    float2 th[LOOP_KPR];
    float ik[LOOP_KPR], s_part = 0.f;
#pragma unroll
    for (int i = 0; i < LOOP_KPR; ++i) {
      const int k = tid + i * FWD_THREADS;
      th[i] = k < K ? __ldcg(a.theta + k) : make_float2(0.f, 0.f);
      ik[i] = th[i].x * th[i].x + th[i].y * th[i].y;
      s_part += ik[i];
    }
    const float S = loop_block_sum(s_part, scr, tid);
    if (!(S > 0.f) || !isfinite(S)) {
      if (writer && tid == 0) {
        atomicOr(&a.st->err, OFA_ERRBIT_NUMERIC);
        a.st->done = 1;
      }
      break;
    }
    const float inv_s = 1.f / S;
    float wk[LOOP_KPR], sq[LOOP_KPR], r0 = 0.f, r1 = 0.f, mx = 0.f;
#pragma unroll
    for (int i = 0; i < LOOP_KPR; ++i) {
      const int k = tid + i * FWD_THREADS;
      sq[i] = sqrtf(tl[k < LOOP_KMAX ? k : 0]);
      wk[i] = wl[k < LOOP_KMAX ? k : 0];
      if (k >= K) continue;
      const float ih = ik[i] * inv_s, d = tl[k] - ih;
      r0 += d * d;
      r1 += ih * ih;
      if (a.weighting) wk[i] *= sq[i] * rsqrtf(fmaxf(ih, 1e-30f));   // w sqrt(t / Ihat)
      mx = fmaxf(mx, wk[i] * sq[i]);
    }
    loop_block_reduce3(r0, r1, mx, scr, tid);
    const float xi = 1.f - sqrtf(r0 / r1);
    if (writer && tid == 0) {
      a.hist[(h0 + it) % OFA_HIST_CAP] = (double)xi;
      a.st->hist_count = h0 + it + 1;
      a.st->xi = (double)xi;
    }
    if (thr_on && (double)xi > a.threshold) {
      if (writer && tid == 0) a.st->done = 1;
      break;
    }
    int ex = 0;
    frexpf(mx, &ex);
    const float scale = mx > 0.f ? exp2f((float)-ex) : 1.f;
#pragma unroll
    for (int i = 0; i < LOOP_KPR; ++i) {
      const int k = tid + i * FWD_THREADS;
      if (k >= K) continue;
      const float mag = wk[i] * sq[i] * scale;
      float2 ck;
      if (ik[i] > 0.f) {
        const float inv = rsqrtf(ik[i]);
        ck = make_float2(mag * th[i].x * inv, mag * th[i].y * inv);
      } else {
        ck = make_float2(mag, 0.f);   // arg(0) = 0
      }
      cl[k] = ck;
      if (a.weighting) wl[k] = wk[i];
      if (writer) {
        if (a.weighting) a.w[k] = wk[i];
        a.c[k] = ck;
      }
    }
    if (writer && tid == 0) {
      a.st->j = j0 + it + 1;
      a.st->c_scale = scale;
    }
    __syncthreads();
    // ---- inverse for the block's rows: U = (C on the grid) conj(Fyu) restricted to them
    for (int i = tid; i < uy * ux; i += FWD_THREADS) {
      const int k = gk[i];
      cs[i] = k >= 0 ? cl[k] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int i = tid; i < R * uxp; i += FWD_THREADS) {
      const int r = i / uxp, ix = i - r * uxp;
      float2 u = make_float2(0.f, 0.f);
      if (ix < ux)
        for (int iy = 0; iy < uy; ++iy) cmac_conj(u, fs[iy * R + r], cs[iy * ux + ix]);
      us[i] = u;   // U[r][ix] = sum_iy C[iy][ix] conj(Fyu[iy][n0 + r])
    }
    // E'[r][j] = sum_ix U[g RT + r][ix] conj(Fxu[ix][t + 256 j]), quads through the ring
    float2 acc[RT][FWD_MT];
#pragma unroll
    for (int r = 0; r < RT; ++r)
#pragma unroll
      for (int j = 0; j < FWD_MT; ++j) acc[r][j] = make_float2(0.f, 0.f);
    for (int q = 0; q < nquad; ++q) {
      cp_async_wait<FWD_STAGES - 2>();
      __syncthreads();   // quad q landed for everyone (and, at q = 0, U is complete)
      fwd_issue(ring, a.fxu, ux, nx, q + FWD_STAGES - 1, tid);
      const float2* src = ring + (size_t)(q % FWD_STAGES) * FWD_SLOT;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float2 uv[RT];
#pragma unroll
        for (int r = 0; r < RT; ++r) {
          const int row = g * RT + r;   // rows past R (the group's padding) stay zero
          uv[r] = row < R ? us[row * uxp + 4 * q + c] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < FWD_MT; ++j) {
          const float2 fv = src[(c * FWD_MT + j) * FWD_GROUP + t];
#pragma unroll
          for (int r = 0; r < RT; ++r) cmac_conj(acc[r][j], fv, uv[r]);   // U conj(Fxu)
        }
      }
    }
    // the next field E = A E'/|E'| (A at E' = 0); phi and the stored field when the
    // loop may end here
    const bool store = it == a.n_iter - 1 || thr_on;
#pragma unroll
    for (int r = 0; r < RT; ++r)
#pragma unroll
      for (int j = 0; j < FWD_MT; ++j) {
        const float2 z = acc[r][j];
        const float r2 = z.x * z.x + z.y * z.y;
        const float sc = r2 > 0.f ? av[r][j] * rsqrtf(r2) : 0.f;
        e[r][j] = r2 > 0.f ? make_float2(sc * z.x, sc * z.y) : make_float2(av[r][j], 0.f);
        const int m = t + j * FWD_GROUP;
        if (store && r < rows_g && m < nx) {
          const size_t o = (size_t)(n0 + g * RT + r) * nx + m;
          a.phi[o] = ofa_arg(z.y, z.x);   // arg(0) = 0
          a.e32[o] = e[r][j];
        }
      }
    // the next forward's first quads, once every thread is done with the ring
    __syncthreads();
#pragma unroll
    for (int q = 0; q < FWD_STAGES - 1; ++q) fwd_issue(ring, a.fxu, ux, nx, q, tid);
  }
  if (!s_ok && tid == 0) {
    atomicOr(&a.st->err, OFA_ERRBIT_TIMEOUT);
    a.st->done = 1;
  }
  cp_async_wait<0>();
}

size_t fwd_smem(int R, int ux, int uy) {
  return sizeof(float2) * FWD_RING + sizeof(float) * (size_t)((ux + 3) / 4) * FWD_WARPS * 32 +
         sizeof(float2) * ((size_t)R * ux + (size_t)uy * R);
}

// rows of a forward thread group: RT = ceil(R / 2)
template <class F>
void visit_rt(int R, F&& f) {
  switch ((R + 1) / 2) {
    case 1: f(std::integral_constant<int, 1>()); break;
    case 2: f(std::integral_constant<int, 2>()); break;
    case 3: f(std::integral_constant<int, 3>()); break;
    default: f(std::integral_constant<int, 4>()); break;
  }
}

// Launch as a programmatic dependent of the previous kernel in the stream.
template <class... P, class... A>
void launch_pdl(void (*kernel)(P...), dim3 grid, int threads, size_t smem, cudaStream_t s,
                A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

}  // namespace

int sep_rows_per_block(int ny, int sms) {
  const int r = (ny + sms - 1) / sms;
  return r < 1 ? 1 : (r > SEP_MAX_R ? SEP_MAX_R : r);
}

int sep_fwd_blocks(int ny, int sms) {
  const int r = sep_rows_per_block(ny, sms);
  return (ny + r - 1) / r;
}

size_t sep_fwd_smem(int ny, int ux, int uy, int sms) {
  return fwd_smem(sep_rows_per_block(ny, sms), ux, uy);
}

size_t sep_inv_smem(int ux, int uy) {
  return sizeof(float2) * ((size_t)uy * INV_ROWS + (size_t)uy * ux + (size_t)ux * INV_COLS +
                           (size_t)uy * INV_COLS);
}

bool sep_fast_shape(int nx, int uy) { return nx <= FWD_MT * FWD_GROUP && uy <= INV_MAX_UY; }

size_t sep_smem_limit() { return SEP_SMEM_LIMIT; }

// The attribute is per function, shared by every plan of the process: it is set to
// the fixed ceiling the fast path admits, never to one plan's own size (a later plan
// with a smaller grid would otherwise lower it under an earlier plan's launches).
cudaError_t sep_prepare() {
  cudaError_t e = cudaSuccess;
  for (int r = 1; r <= SEP_MAX_R && e == cudaSuccess; ++r)
    visit_rt(r, [&](auto rc) {
      e = cudaFuncSetAttribute(sep_fwd_kernel<decltype(rc)::value>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SEP_SMEM_LIMIT);
    });
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sep_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SEP_SMEM_LIMIT);
}

bool sep_fwd_fuses_focal(int ny, int K, int sms) {
  const size_t staged = (size_t)sep_fwd_blocks(ny, sms) * (size_t)((K + 1) / 2) * 2;
  return K <= FWD_THREADS && staged <= FWD_RING;
}

void launch_sep_fwd(const float2* e32, const float2* fxu, const float2* fyu, const int2* ixy,
                    int nx, int ny, int ux, int uy, int K, int kp, int sms, float2* part,
                    const FocalTail& f, const int* done, cudaStream_t s) {
  const int R = sep_rows_per_block(ny, sms);
  const size_t smem = fwd_smem(R, ux, uy);
  const int blocks = sep_fwd_blocks(ny, sms);
  FocalTail fk = f;
  fk.on = f.on && sep_fwd_fuses_focal(ny, K, sms);
  visit_rt(R, [&](auto rc) {
    launch_pdl(sep_fwd_kernel<decltype(rc)::value>, dim3(blocks), FWD_THREADS, smem, s, e32, fxu,
               fyu, ixy, nx, ny, ux, uy, K, kp, R, part, done, fk);
  });
}

void launch_sep_sum_focal(const float2* part, int nb, int K, int kp, float2* theta, int focal,
                          const float* t, float* w, float2* c, double* hist, OfaDevState* st,
                          int weighting, unsigned* counter, const int* done, cudaStream_t s) {
  launch_pdl(sep_sum_focal_kernel, dim3((K + 31) / 32), SEP_THREADS, 0, s, part, nb, K, kp, theta,
             focal, t, w, c, hist, st, weighting, counter, done);
}

void launch_sep_tc_theta(const float2* gt, int parts, const float2* fyu, const int* gridk, int ny,
                         int ux, int uy, int K, float2* theta, const float* w, float* wprev,
                         const int* done, cudaStream_t s) {
  const dim3 grid((unsigned)ux, (unsigned)((uy + TCT_WARPS - 1) / TCT_WARPS));
  launch_pdl(sep_tc_theta_kernel, grid, TCT_THREADS, 0, s, gt, parts, fyu, gridk, ny, ux, uy, K,
             theta, w, wprev, done);
}

void launch_sep_inverse(const float2* c, const int* gridk, const float2* fxu, const float2* fyu,
                        const float* amp, int nx, int ny, int ux, int uy, float* phi,
                        float2* e32, const int* done, cudaStream_t s) {
  dim3 grid((nx + INV_COLS - 1) / INV_COLS, (ny + INV_ROWS - 1) / INV_ROWS);
  launch_pdl(sep_inv_kernel, grid, INV_THREADS, sep_inv_smem(ux, uy), s, c, gridk, fxu, fyu, amp,
             nx, ny, ux, uy, phi, e32, done);
}

// ---------------------------------------------------------------- persistent loop host
constexpr size_t SEP_LOOP_SMEM_LIMIT = 220 * 1024;

bool sep_loop_shape(int nx, int ny, int ux, int uy, int K, int sms, size_t* smem, int* grid) {
  const int R = sep_rows_per_block(ny, sms);
  const int G = sep_fwd_blocks(ny, sms);
  const size_t bytes = loop_layout(R, ux, uy).total;
  if (!sep_fast_shape(nx, uy) || K > LOOP_KMAX || G > sms || bytes > SEP_LOOP_SMEM_LIMIT)
    return false;
  if (smem) *smem = bytes;
  if (grid) *grid = G;
  return true;
}

cudaError_t sep_loop_prepare(int ny, int sms, int* resident) {
  cudaError_t e = cudaSuccess;
  int per_sm = 0;
  visit_rt(sep_rows_per_block(ny, sms), [&](auto rc) {
    auto kern = sep_loop_kernel<decltype(rc)::value>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SEP_LOOP_SMEM_LIMIT);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FWD_THREADS,
                                                        SEP_LOOP_SMEM_LIMIT);
  });
  if (resident) *resident = e == cudaSuccess ? per_sm : 0;
  return e;
}

cudaError_t launch_sep_loop(ofa_plan* p, int n_iter, double threshold, cudaStream_t s) {
  if (n_iter <= 0) return cudaSuccess;
  constexpr int CHUNK = 1 << 20;   // a barrier counter reaches iterations x blocks
  if (n_iter > CHUNK) {
    for (int left = n_iter; left > 0; left -= CHUNK) {
      cudaError_t e = launch_sep_loop(p, left < CHUNK ? left : CHUNK, threshold, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  size_t smem = 0;
  int G = 0;
  if (!sep_loop_shape(p->nx, p->ny, p->ux, p->uy, p->K, p->sm_count, &smem, &G))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(p->loop_bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  SepLoopArgs a;
  a.fxu = p->fxu; a.fyu = p->fyu; a.ixy = p->ixy; a.gridk = p->sep_gridk; a.amp = p->amp;
  a.e32 = p->e32; a.phi = p->phi; a.part = p->part; a.theta = p->theta; a.c = p->c;
  a.t = p->t; a.w = p->w; a.hist = p->hist; a.st = p->st; a.bar = p->loop_bar;
  a.threshold = threshold;
  a.nx = p->nx; a.ny = p->ny; a.ux = p->ux; a.uy = p->uy; a.K = p->K; a.kp = p->kp;
  a.R = sep_rows_per_block(p->ny, p->sm_count);
  a.weighting = p->weighting;
  a.n_iter = n_iter;
  visit_rt(a.R, [&](auto rc) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(FWD_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, sep_loop_kernel<decltype(rc)::value>, a);
  });
  return e;
}
