// FP32 CUDA-core form of the two MTP products (kernels (b) and (d), OFA_PREC_FP32).
//
// Forward (Eq. 2 at the foci): G[n,k] = sum_m E[n,m] Fx[k,m] over the pupil field
// E = A exp(i phi) kept as complex planes (written by the inverse's epilogue, or by
// field_f32_kernel for a given phase), then the per-focus dot
// Theta_k = sum_n Fy[k,n] G[n,k] reduced inside the tile; each 64-row tile writes
// one deterministic partial Theta.
//
// Inverse (Algorithm 1, inverse propagation read as the adjoint of Eq. 2):
// E'[n,m] = sum_k conj(Fy[k,n]) c_k conj(Fx[k,m]), fused with the phase-only
// projection phi = arg(E') and the next field A exp(i phi) (or, for the
// gradient, 2 Im(conj(E) E')).
//
// Both products are 64 x 64 complex tiles computed by 128 threads (four warps of
// 32 x 32), each thread holding 8 x 4 complex outputs, by one loop (tile_product)
// over operands stored row-major with the contraction contiguous: E and Fx for
// the forward; conj(Fy)^T c and conj(Fx)^T for the inverse (conj(Fx)^T and Fy^T
// are formed once per plan, conj(Fy)^T c once per iteration).  Stages of 16 contraction
// steps are copied global -> shared by cp.async (two buffers, one barrier per
// stage).  The shape is set by shared-memory bandwidth, the limit of these
// products on sm_103a: a 16-byte shared load costs a warp 4 SM cycles, or 2 when
// it reads at most four distinct addresses, so every lane of a quarter warp
// reads the same row operand and the per-thread tile is 8 rows by 4 columns, 16
// shared-load cycles for 32 FMA cycles per contraction step.  Both products
// split their contraction over up to four blocks per tile (more resident warps
// per SM and an even spread of blocks over the SMs) and sum the parts in fixed
// order, so results do not depend on timing: in the forward the last block of a
// tile to arrive sums the per-focus partial dots; in the inverse the parts of a
// tile form a thread-block cluster and reduce through distributed shared memory.
#include <cooperative_groups.h>

#include <algorithm>

#include "ofa_focal.cuh"
#include "ofa_internal.cuh"
#include "ofa_math.cuh"

namespace {

constexpr int T64 = 64;
constexpr int TS = 16;
constexpr int SIMT_THREADS = 128;
constexpr int SP = TS + 2;   // padded row pitch (complex) of the forward's staged tiles

// Pairs of contraction steps unrolled in the inner loop.
#ifndef OFA_SIMT_UNROLL
#define OFA_SIMT_UNROLL 1
#endif
constexpr int UNROLL = OFA_SIMT_UNROLL;

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// 8-byte global -> shared asynchronous copy; zero-fills the destination when !ok
// (src is then not read).
__device__ __forceinline__ void cp_async8(float2* dst, const float2* src, bool ok) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
               "r"(ok ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// E = A exp(i phi), complex planes [ny][nx] (accurate sincosf: the FP32 form keeps
// full FP32 accuracy).
__global__ void field_f32_kernel(const float* __restrict__ phi, const float* __restrict__ amp,
                                 size_t n, float2* __restrict__ e) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float s, c;
    sincosf(phi[i], &s, &c);
    const float a = amp[i];
    e[i] = make_float2(a * c, a * s);
  }
}

// Shared staging of one 64 x 64 tile product: two buffers of 64 rows x 16
// contraction steps for each operand, padded pitch.
struct TileSmem {
  float2 a[2][T64][SP];
  float2 b[2][T64][SP];
};

// acc[i][j] += sum_t A[r0 + r_i][t] B[c0 + c_j][t] over t in [t_begin, t_end).
// A and B are row-major with the contraction contiguous
// (leading dimensions lda, ldb; rows >= a_rows / b_rows read as zero) and are
// staged in that layout, so that one 16-byte load gives a row's two consecutive
// contraction steps.  Thread (warp w, lane l): rows r_i = (w>>1)*32 + (l>>3) + 4i,
// i < 8 (one row per quarter warp: the same address across its lanes), columns
// c_j = (w&1)*32 + (l&7) + 8j, j < 4 (eight consecutive padded rows per quarter:
// distinct banks).  t_begin is a multiple of 16; t_end is one too or the end of
// the contraction.
__device__ __forceinline__ void tile_product(TileSmem& sm, const float2* __restrict__ A, int lda,
                                             int a_rows, const float2* __restrict__ B, int ldb,
                                             int b_rows, int r0, int c0, int t_begin, int t_end,
                                             float2 (&acc)[8][4]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lr = lane >> 3, lc = lane & 7, wr = warp >> 1, wc = warp & 1;
  // element q of a stage: row (tid + 128 q) / 16, step (tid + 128 q) % 16
  auto issue = [&](int b, int t0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + SIMT_THREADS * q, r = e >> 4, tt = e & 15, t = t0 + tt;
      const bool okA = r0 + r < a_rows && t < t_end, okB = c0 + r < b_rows && t < t_end;
      cp_async8(&sm.a[b][r][tt], okA ? A + (size_t)(r0 + r) * lda + t : A, okA);
      cp_async8(&sm.b[b][r][tt], okB ? B + (size_t)(c0 + r) * ldb + t : B, okB);
    }
    cp_async_commit();
  };

  if (t_begin < t_end) issue(0, t_begin);
  int b = 0;
  for (int t0 = t_begin; t0 < t_end; t0 += TS) {
    cp_async_wait_all();
    __syncthreads();  // stage b complete; every thread is done with stage b ^ 1
    if (t0 + TS < t_end) issue(b ^ 1, t0 + TS);
#pragma unroll UNROLL
    for (int tt = 0; tt < TS; tt += 2) {
      float4 fq[4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        fq[j] = *reinterpret_cast<const float4*>(&sm.b[b][wc * 32 + lc + 8 * j][tt]);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float4 aq = *reinterpret_cast<const float4*>(&sm.a[b][wr * 32 + lr + 4 * i][tt]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          cmac(acc[i][j], make_float2(aq.x, aq.y), make_float2(fq[j].x, fq[j].y));
          cmac(acc[i][j], make_float2(aq.z, aq.w), make_float2(fq[j].z, fq[j].w));
        }
      }
    }
    b ^= 1;
  }
}

// Contraction part z of gridDim.z: whole 16-deep steps [begin, end) of len.
__device__ __forceinline__ int2 part_range(int len) {
  const int steps = (len + TS - 1) / TS;
  return make_int2((int)(blockIdx.z * steps / gridDim.z) * TS,
                   min(len, (int)((blockIdx.z + 1) * steps / gridDim.z) * TS));
}

// Forward tile: rows n (E rows), columns k (foci), contraction m.
// STORE: instead of the per-focus dot, write the product itself transposed,
// gt[k][n] = G[n][k] (the separable grid form's first product).
// With f.on (K <= 2048): the last row tile of each focus column to finish sums that
// column's partial rows in order into row 0 (the order the focal kernel sums them), and
// the last column to finish runs the focal step (f.counter: one counter per column
// tile, then one for the columns).
template <bool STORE>
__global__ void __launch_bounds__(SIMT_THREADS, 4) fwd_simt_kernel(
    const float2* __restrict__ e32, const float2* __restrict__ fx, const float2* __restrict__ fy,
    int nx, int ny, int K, int kp, float2* __restrict__ part, const int* __restrict__ done,
    float2* __restrict__ fws, unsigned* __restrict__ cnt, FocalTail f) {
  if (done != nullptr && *done) return;
  __shared__ __align__(16) TileSmem sm;
  __shared__ float2 red[2][T64];
  __shared__ int last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lr = lane >> 3, lc = lane & 7, wr = warp >> 1, wc = warp & 1;
  const int n0 = blockIdx.y * T64, k0 = blockIdx.x * T64;

  float2 acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  const int2 range = part_range(nx);
  tile_product(sm, e32, nx, ny, fx, nx, K, n0, k0, range.x, range.y, acc);

  if constexpr (STORE) {
    float2* g = part + (size_t)blockIdx.z * K * ny;   // slice of this contraction part
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + wc * 32 + lc + 8 * j;
      if (k >= K) continue;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int n = n0 + wr * 32 + lr + 4 * i;
        if (n < ny) g[(size_t)k * ny + n] = acc[i][j];
      }
    }
  } else {
    // Per-focus dot with the Fy rows over the tile's 64 rows, reduced in fixed order:
    // the thread's 8 rows, the four quarter warps (shuffles), the two row warps.
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + wc * 32 + lc + 8 * j;
      float2 s = make_float2(0.f, 0.f);
      if (k < K) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int n = n0 + wr * 32 + lr + 4 * i;
          if (n < ny) cmac(s, fy[(size_t)k * ny + n], acc[i][j]);
        }
      }
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 8);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 8);
      s.x += __shfl_xor_sync(0xffffffffu, s.x, 16);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, 16);
      if (lr == 0) red[wr][wc * 32 + lc + 8 * j] = s;
    }
    __syncthreads();
    const int k = k0 + tid;
    float2 mine = make_float2(0.f, 0.f);
    if (tid < T64) mine = make_float2(red[0][tid].x + red[1][tid].x, red[0][tid].y + red[1][tid].y);
    if (gridDim.z == 1) {
      if (tid < T64 && k < kp) part[(size_t)blockIdx.y * kp + k] = mine;
    } else {
      // contraction parts: the last block of this tile sums them in order z = 0, 1, ...
      const int tile = blockIdx.y * gridDim.x + blockIdx.x;
      float2* ws = fws + (size_t)tile * gridDim.z * T64;
      if (tid < T64) ws[blockIdx.z * T64 + tid] = mine;
      __threadfence();
      __syncthreads();
      if (tid == 0) last = atomicAdd(&cnt[tile], 1u) == gridDim.z - 1;
      __syncthreads();
      if (!last) return;
      __threadfence();
      if (tid < T64) {
        float2 a = make_float2(0.f, 0.f);
        for (int z = 0; z < (int)gridDim.z; ++z) {
          const float2 v = z == (int)blockIdx.z ? mine : __ldcg(&ws[z * T64 + tid]);
          a.x += v.x;
          a.y += v.y;
        }
        if (k < kp) part[(size_t)blockIdx.y * kp + k] = a;
      }
      if (tid == 0) cnt[tile] = 0;
    }
    if (!f.on) return;

    // this focus column's partial rows (one per row tile) summed in order into row 0
    __shared__ int tail_last;
    __shared__ float focal_sh[4 * 33 + 4];
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      tail_last = atomicAdd(&f.counter[blockIdx.x], 1u) == gridDim.y - 1;
      if (tail_last) {
        __threadfence();
        f.counter[blockIdx.x] = 0u;
      }
    }
    __syncthreads();
    if (!tail_last) return;
    if (tid < T64 && k < kp) {
      constexpr int RB = 8;   // rows of loads in flight
      float2 a = make_float2(0.f, 0.f);
      for (int y0 = 0; y0 < (int)gridDim.y; y0 += RB) {
        float2 v[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u)
          v[u] = y0 + u < (int)gridDim.y ? __ldcg(part + (size_t)(y0 + u) * kp + k)
                                         : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < RB; ++u)
          if (y0 + u < (int)gridDim.y) {
            a.x += v[u].x;
            a.y += v[u].y;
          }
      }
      part[k] = a;
    }
    // the last column runs the focal step on Theta
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      tail_last = atomicAdd(&f.counter[gridDim.x], 1u) == gridDim.x - 1;
      if (tail_last) {
        __threadfence();
        f.counter[gridDim.x] = 0u;
      }
    }
    __syncthreads();
    if (!tail_last) return;
    if (K <= SIMT_THREADS * 4)
      ofa_focal::iterate_regs<SIMT_THREADS, 4>(part, 1, K, kp, f.t, f.w, f.c, f.hist, f.st,
                                               f.weighting, focal_sh, tid,
                                               ofa_focal::BarBlock());
    else
      ofa_focal::iterate_regs<SIMT_THREADS, 16>(part, 1, K, kp, f.t, f.w, f.c, f.hist, f.st,
                                                f.weighting, focal_sh, tid,
                                                ofa_focal::BarBlock());
  }
}

// pT[n][k] = conj(FyT[n][k]) c_k: the inverse's left operand, rows n, contraction
// k < K, row pitch ldk (a multiple of 16; the padding columns are zero).  Each
// thread handles four consecutive k of one row (two 16-byte loads and stores).
__global__ void scale_conj_kernel(const float2* __restrict__ fyT, const float2* __restrict__ c,
                                  int K, int ldk, int ny, float2* __restrict__ pT,
                                  const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int q = ldk / 4;   // quads per row
  const size_t n_quads = (size_t)q * ny;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n_quads;
       i += (size_t)gridDim.x * blockDim.x) {
    const int k0 = (int)(i % q) * 4;
    const float4* src = reinterpret_cast<const float4*>(fyT) + 2 * i;
    float4* dst = reinterpret_cast<float4*>(pT) + 2 * i;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float4 a = src[h];
      const int k = k0 + 2 * h;
      const float2 c0 = k < K ? c[k] : make_float2(0.f, 0.f);
      const float2 c1 = k + 1 < K ? c[k + 1] : make_float2(0.f, 0.f);
      dst[h] = make_float4(a.x * c0.x + a.y * c0.y, a.x * c0.y - a.y * c0.x,
                           a.z * c1.x + a.w * c1.y, a.z * c1.y - a.w * c1.x);
    }
  }
}

// Inverse tile: rows n, columns m, contraction k over this block's part of it:
// E'[n][m] = sum_k pT[n][k] fxT[m][k], fxT = conj(Fx)^T (both with row pitch ldk).
// With the contraction split (gridDim.z > 1) the z parts of a tile run as one
// thread-block cluster: each keeps its partial tile in its shared memory, and
// after a cluster barrier part z sums outputs [32z/Z, 32(z+1)/Z) of every thread
// over the parts in order 0, 1, ... (distributed shared memory) and finishes them.
// EPI 0: phi = arg(E') (atan2(0,0) = 0) and the next field A exp(i phi), formed
// exactly as field_f32_kernel forms it from a stored phi.
// EPI 1: grad = f 2 A (cos phi Im B - sin phi Re B).
template <int EPI>
__global__ void __launch_bounds__(SIMT_THREADS, 4) bwd_simt_kernel(
    const float2* __restrict__ pT, const float2* __restrict__ fxT, int nx, int ny, int K, int ldk,
    float* __restrict__ out, float2* __restrict__ e_out, const float* __restrict__ phi_in,
    const float* __restrict__ amp, float amp_factor, const OfaDevState* __restrict__ st,
    const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  __shared__ __align__(16) TileSmem sm;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lr = lane >> 3, lc = lane & 7, wr = warp >> 1, wc = warp & 1;
  const int n0 = blockIdx.y * T64, m0 = blockIdx.x * T64;

  float2 acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  const int2 range = part_range(K);
  tile_product(sm, pT, ldk, ny, fxT, ldk, nx, n0, m0, range.x, range.y, acc);

  const float factor = EPI == 1 ? 2.f * amp_factor / st->c_scale : 0.f;
  // output (i, j) of this thread: row n0 + (w>>1)*32 + (l>>3) + 4i, column
  // m0 + (w&1)*32 + (l&7) + 8j
  auto finish = [&](int i, int j, float2 z) {
    const int n = n0 + wr * 32 + lr + 4 * i, m = m0 + wc * 32 + lc + 8 * j;
    if (n >= ny || m >= nx) return;
    const size_t o = (size_t)n * nx + m;
    if (EPI == 0) {
      const float ph = ofa_arg(z.y, z.x);
      float sn, cs;
      sincosf(ph, &sn, &cs);
      const float a = amp[o];
      out[o] = ph;
      e_out[o] = make_float2(a * cs, a * sn);
    } else {
      float sn, cs;
      sincosf(phi_in[o], &sn, &cs);
      out[o] = factor * amp[o] * (cs * z.y - sn * z.x);
    }
  };

  if (gridDim.z == 1) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) finish(i, j, acc[i][j]);
    return;
  }
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  float2* part = &sm.a[0][0][0];   // 32 x 128 partial outputs (fits in the stages)
  __syncthreads();                 // every warp is done with the stages
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) part[(i * 4 + j) * SIMT_THREADS + tid] = acc[i][j];
  cluster.sync();
  const int Z = (int)gridDim.z, z = (int)blockIdx.z;
  for (int idx = z * 32 / Z; idx < (z + 1) * 32 / Z; ++idx) {
    float2 v = make_float2(0.f, 0.f);
    for (int r = 0; r < Z; ++r) {
      const float2 t = cluster.map_shared_rank(part, r)[idx * SIMT_THREADS + tid];
      v.x += t.x;
      v.y += t.y;
    }
    finish(idx >> 2, idx & 3, v);
  }
  cluster.sync();   // the other parts still read this block's shared memory
}

// Separable grid form, focal step of the forward: Theta_k = sum_n Fyu[iy_k][n] G[n][ix_k]
// (one warp per focus, fixed-order shuffle tree), written as the single partial row.
// The first product's contraction slices [parts][ux][ny] summed in order into slice 0.
__global__ void sep_reduce_kernel(float2* __restrict__ gt, size_t slice, int parts) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < slice;
       i += (size_t)gridDim.x * blockDim.x) {
    float2 a = gt[i];
    for (int z = 1; z < parts; ++z) {
      const float2 v = gt[z * slice + i];
      a.x += v.x;
      a.y += v.y;
    }
    gt[i] = a;
  }
}

// One 256-thread block per focus; fixed-order shuffle and shared-memory tree.
__global__ void __launch_bounds__(256) sep_theta_kernel(const float2* __restrict__ gt,
                                                        const float2* __restrict__ fyu,
                                                        const int2* __restrict__ ixy, int ny,
                                                        float2* __restrict__ part) {
  __shared__ float2 red[8];
  const int k = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int2 q = ixy[k];
  const float2* g = gt + (size_t)q.x * ny;
  const float2* f = fyu + (size_t)q.y * ny;
  float2 a = make_float2(0.f, 0.f);
  for (int n = threadIdx.x; n < ny; n += 256) cmac(a, f[n], g[n]);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
  }
  if (lane == 0) red[warp] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 t = red[0];
    for (int w = 1; w < 8; ++w) {
      t.x += red[w].x;
      t.y += red[w].y;
    }
    part[k] = t;
  }
}

// Separable grid form, first product of the inverse: for row iy of the grid,
// T[iy][m] = sum over the foci of that row (in fixed order) of c_k conj(Fxu[ix_k][m]);
// stored conjugated, as the inverse product conjugates its right operand.  Block
// (column chunk, iy); the row's (c_k, ix_k) are staged in shared memory.
constexpr int SEP_T_ROW = 256;   // foci of a row staged per pass
__global__ void __launch_bounds__(256) sep_t_kernel(
    const float2* __restrict__ c, const float2* __restrict__ fxu, const int2* __restrict__ ixy,
    const int* __restrict__ row_ptr, const int* __restrict__ row_foci, int nx,
    float2* __restrict__ tconj) {
  __shared__ float2 cs[SEP_T_ROW];
  __shared__ int xs[SEP_T_ROW];
  const int iy = blockIdx.y, m = blockIdx.x * 256 + threadIdx.x;
  const int r0 = row_ptr[iy], r1 = row_ptr[iy + 1];
  float2 a = make_float2(0.f, 0.f);
  for (int rb = r0; rb < r1; rb += SEP_T_ROW) {
    const int nr = min(SEP_T_ROW, r1 - rb);
    __syncthreads();
    if ((int)threadIdx.x < nr) {
      const int k = row_foci[rb + threadIdx.x];
      cs[threadIdx.x] = c[k];
      xs[threadIdx.x] = ixy[k].x;
    }
    __syncthreads();
    if (m < nx)
      for (int r = 0; r < nr; ++r) {
        const float2 f = fxu[(size_t)xs[r] * nx + m];
        cmac(a, cs[r], make_float2(f.x, -f.y));
      }
  }
  if (m < nx) tconj[(size_t)iy * nx + m] = make_float2(a.x, -a.y);
}

}  // namespace

// Contraction parts (grid z) of the two products, at most: more, shorter blocks
// fill the SMs with resident warps and even out the blocks per SM.  A part keeps
// at least four 16-deep stages.
#ifndef OFA_SIMT_FWD_SPLIT
#define OFA_SIMT_FWD_SPLIT 4
#endif
#ifndef OFA_SIMT_BWD_SPLIT
#define OFA_SIMT_BWD_SPLIT 4
#endif
constexpr int FWD_SPLIT = OFA_SIMT_FWD_SPLIT;
constexpr int BWD_SPLIT = OFA_SIMT_BWD_SPLIT;

int split_parts(int len, int max_parts) {
  const int stages = (len + TS - 1) / TS;
  return std::max(1, std::min(max_parts, stages / 4));
}

int tiles_of(int n) { return (n + T64 - 1) / T64; }

int simt_fwd_tiles(int ny) { return tiles_of(ny); }

int simt_ldk(int K) { return (K + TS - 1) / TS * TS; }

SimtSizes simt_sizes(int nx, int ny, int K, int rows) {
  SimtSizes z;
  z.fwd_tiles = tiles_of(K) * tiles_of(ny);
  const size_t ldk = simt_ldk(std::max(rows, K));
  z.p32 = ldk * ny;
  z.fxT = ldk * nx;
  z.fyT = ldk * ny;
  z.fws = (size_t)z.fwd_tiles * FWD_SPLIT * T64;
  z.cnt = (size_t)z.fwd_tiles + tiles_of(K) + 1;   // tiles, focus columns, all columns
  return z;
}

void launch_field_f32(const float* phi, const float* amp, int nx, int ny, float2* e,
                      cudaStream_t s) {
  const size_t n = (size_t)nx * ny;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  field_f32_kernel<<<(unsigned)blocks, 256, 0, s>>>(phi, amp, n, e);
}

bool simt_fwd_fuses_focal(int K) { return K <= SIMT_THREADS * 16; }

void launch_fwd_simt(const float2* e32, const float2* fx, const float2* fy, int nx, int ny, int K,
                     int kp, float2* part, const int* done, const SimtWork& w, cudaStream_t s,
                     const FocalTail* f) {
  dim3 grid(tiles_of(K), tiles_of(ny), split_parts(nx, FWD_SPLIT));
  FocalTail tail = {};
  if (f && f->on && simt_fwd_fuses_focal(K)) {
    tail = *f;
    tail.counter = w.cnt + (size_t)tiles_of(K) * tiles_of(ny);   // after the tile counters
  }
  fwd_simt_kernel<false><<<grid, SIMT_THREADS, 0, s>>>(e32, fx, fy, nx, ny, K, kp, part, done,
                                                       w.fws, w.cnt, tail);
}

int sep_parts(int nx, int ny, int ux, int sms) {
  const int tiles = ((ux + T64 - 1) / T64) * ((ny + T64 - 1) / T64);
  const int steps = (nx + TS - 1) / TS;
  int parts = (2 * sms + tiles - 1) / tiles;   // about two blocks per SM
  if (parts > steps) parts = steps;
  if (parts > 32) parts = 32;
  return parts < 1 ? 1 : parts;
}

void launch_sep_forward(const float2* e32, const float2* fxu, int nx, int ny, int ux, int parts,
                        float2* gt, cudaStream_t s) {
  dim3 grid((ux + T64 - 1) / T64, (ny + T64 - 1) / T64, parts);
  fwd_simt_kernel<true><<<grid, SIMT_THREADS, 0, s>>>(e32, fxu, nullptr, nx, ny, ux, ux, gt,
                                                      nullptr, nullptr, nullptr, FocalTail{});
}

void launch_sep_theta(float2* gt, const float2* fyu, const int2* ixy, int K, int ny, int ux,
                      int parts, float2* part, cudaStream_t s) {
  if (parts > 1) {
    const size_t slice = (size_t)ux * ny;
    size_t blocks = (slice + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    sep_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(gt, slice, parts);
  }
  sep_theta_kernel<<<K, 256, 0, s>>>(gt, fyu, ixy, ny, part);
}

void launch_sep_t(const float2* c, const float2* fxu, const int2* ixy, const int* row_ptr,
                  const int* row_foci, int uy, int nx, float2* tconj, cudaStream_t s) {
  dim3 grid((nx + 255) / 256, uy);
  sep_t_kernel<<<grid, 256, 0, s>>>(c, fxu, ixy, row_ptr, row_foci, nx, tconj);
}

void launch_scale_conj(const float2* c, const float2* fyT, int ny, int K, float2* pT,
                       const int* done, cudaStream_t s) {
  const int ldk = simt_ldk(K);
  const size_t quads = (size_t)(ldk / 4) * ny;
  size_t blocks = (quads + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  scale_conj_kernel<<<(unsigned)blocks, 256, 0, s>>>(fyT, c, K, ldk, ny, pT, done);
}

// The inverse product; its contraction parts (grid z) form one cluster per tile.
template <int EPI>
void launch_bwd_kernel(const float2* pT, const float2* fxT, int nx, int ny, int K, float* out,
                       float2* e_out, const float* phi_in, const float* amp, float amp_factor,
                       const OfaDevState* st, const int* done, cudaStream_t s) {
  const int z = split_parts(K, BWD_SPLIT);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles_of(nx), tiles_of(ny), z);
  cfg.blockDim = dim3(SIMT_THREADS);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = z;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, bwd_simt_kernel<EPI>, pT, fxT, nx, ny, K, simt_ldk(K), out, e_out,
                     phi_in, amp, amp_factor, st, done);
}

void launch_bwd_simt_product(const float2* fxT, int nx, int ny, int K, const float* amp,
                             float* phi, float2* e32, const int* done, const SimtWork& w,
                             cudaStream_t s) {
  launch_bwd_kernel<0>(w.p32, fxT, nx, ny, K, phi, e32, nullptr, amp, 0.f, nullptr, done, s);
}

void launch_bwd_simt(const float2* c, const float2* fxT, const float2* fyT, int nx, int ny, int K,
                     const float* amp, float* phi, float2* e32, const int* done,
                     const SimtWork& w, cudaStream_t s) {
  launch_scale_conj(c, fyT, ny, K, w.p32, done, s);
  launch_bwd_simt_product(fxT, nx, ny, K, amp, phi, e32, done, w, s);
}

void launch_grad_simt(const float2* c, const float2* fxT, const float2* fyT, int nx, int ny,
                      int K, const float* phi, const float* amp, float amp_factor,
                      const OfaDevState* st, float* grad, const SimtWork& w, cudaStream_t s) {
  launch_scale_conj(c, fyT, ny, K, w.p32, nullptr, s);
  launch_bwd_kernel<1>(w.p32, fxT, nx, ny, K, grad, nullptr, phi, amp, amp_factor, st, nullptr,
                       s);
}
