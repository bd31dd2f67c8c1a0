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
// Both are 64 x 64 complex tiles, 256 threads, 4 x 4 complex accumulators per
// thread, 16-deep steps through double-buffered shared memory (one barrier per
// step) with the next step's global loads in flight during the current one.
#include "ofa_internal.cuh"
#include "ofa_math.cuh"

namespace {

constexpr int T64 = 64;
constexpr int TS = 16;

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// 16 steps of the 4 x 4 complex outer products of one shared-memory stage:
// rows a[.][ty*4 ..], columns b[.][tx*4 ..].
// UNROLL: steps unrolled (the forward runs best with 4, the inverse with 16).
template <int UNROLL>
__device__ __forceinline__ void mma_stage(const float2 (*a)[T64], const float2 (*b)[T64], int ty,
                                          int tx, float2 (&acc)[4][4]) {
#pragma unroll UNROLL
  for (int mm = 0; mm < TS; ++mm) {
    const float4 a01 = *reinterpret_cast<const float4*>(&a[mm][ty * 4]);
    const float4 a23 = *reinterpret_cast<const float4*>(&a[mm][ty * 4 + 2]);
    const float4 b01 = *reinterpret_cast<const float4*>(&b[mm][tx * 4]);
    const float4 b23 = *reinterpret_cast<const float4*>(&b[mm][tx * 4 + 2]);
    const float2 e[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w),
                         make_float2(a23.x, a23.y), make_float2(a23.z, a23.w)};
    const float2 f[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w),
                         make_float2(b23.x, b23.y), make_float2(b23.z, b23.w)};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) cmac(acc[i][j], e[i], f[j]);
  }
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

// STORE: instead of the per-focus dot, write the product itself transposed,
// gt[k][n] = G[n][k] (the separable grid form's first product).
template <bool STORE>
__global__ void __launch_bounds__(256) fwd_simt_kernel(
    const float2* __restrict__ e32, const float2* __restrict__ fx, const float2* __restrict__ fy,
    int nx, int ny, int K, int kp, float2* __restrict__ part, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  __shared__ __align__(16) float2 Es[2][TS][T64];
  __shared__ __align__(16) float2 Fs[2][TS][T64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int n0 = blockIdx.y * T64, k0 = blockIdx.x * T64;
  const int lr = tid >> 2, lc = (tid & 3) * 4;
  // this block's share of the contraction: whole TS-deep steps [m_begin, m_end)
  const int steps = (nx + TS - 1) / TS;
  const int m_begin = (int)(blockIdx.z * steps / gridDim.z) * TS;
  const int m_end = min(nx, (int)((blockIdx.z + 1) * steps / gridDim.z) * TS);

  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

  float2 ev[4], fv[4];
  auto gload = [&](int m0) {
    const int n = n0 + lr, k = k0 + lr;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = m0 + lc + q;
      ev[q] = (n < ny && m < nx) ? e32[(size_t)n * nx + m] : make_float2(0.f, 0.f);
      fv[q] = (k < K && m < nx) ? fx[(size_t)k * nx + m] : make_float2(0.f, 0.f);
    }
  };
  auto sstore = [&](int b) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Es[b][lc + q][lr] = ev[q];
      Fs[b][lc + q][lr] = fv[q];
    }
  };
  gload(m_begin);
  sstore(0);
  __syncthreads();
  int b = 0;
  for (int m0 = m_begin; m0 < m_end; m0 += TS) {
    const bool more = m0 + TS < m_end;
    if (more) gload(m0 + TS);
    mma_stage<4>(Es[b], Fs[b], ty, tx, acc);
    if (more) sstore(b ^ 1);  // its readers finished before the previous barrier
    __syncthreads();
    b ^= 1;
  }

  if (STORE) {
    float2* g = part + (size_t)blockIdx.z * K * ny;   // slice of this contraction part
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + tx * 4 + j;
      if (k >= K) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int n = n0 + ty * 4 + i;
        if (n < ny) g[(size_t)k * ny + n] = acc[i][j];
      }
    }
    return;
  }
  // Per-focus dot with the Fy rows, reduced over the tile's 64 rows in fixed order.
  float2* red = &Es[0][0][0];  // 16 x 64 float2
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = k0 + tx * 4 + j;
    float2 s = make_float2(0.f, 0.f);
    if (k < K) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int n = n0 + ty * 4 + i;
        if (n < ny) cmac(s, fy[(size_t)k * ny + n], acc[i][j]);
      }
    }
    red[ty * T64 + tx * 4 + j] = s;
  }
  __syncthreads();
  if (tid < T64) {
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const float2 v = red[t * T64 + tid];
      a.x += v.x;
      a.y += v.y;
    }
    const int k = k0 + tid;
    if (k < kp) part[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * kp + k] = a;
  }
}

// EPI 0: phi = arg(E') (atan2(0,0) = 0) and the next field A exp(i phi), formed
// exactly as field_f32_kernel forms it from a stored phi.
// EPI 1: grad = f 2 A (cos phi Im B - sin phi Re B).
template <int EPI>
__global__ void __launch_bounds__(256) bwd_simt_kernel(
    const float2* __restrict__ c, const float2* __restrict__ fx, const float2* __restrict__ fy,
    int nx, int ny, int K, float* __restrict__ out, float2* __restrict__ e_out,
    const float* __restrict__ phi_in, const float* __restrict__ amp, float amp_factor,
    const OfaDevState* __restrict__ st, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  __shared__ __align__(16) float2 Ps[2][TS][T64];
  __shared__ __align__(16) float2 Qs[2][TS][T64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int n0 = blockIdx.y * T64, m0 = blockIdx.x * T64;
  const int lk = tid >> 4, lc = (tid & 15) * 4;

  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

  float2 pv[4], qv[4];
  auto gload = [&](int k0) {
    const int k = k0 + lk;
    const float2 ck = k < K ? c[k] : make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = n0 + lc + q, m = m0 + lc + q;
      const float2 a = (k < K && n < ny) ? fy[(size_t)k * ny + n] : make_float2(0.f, 0.f);
      const float2 b = (k < K && m < nx) ? fx[(size_t)k * nx + m] : make_float2(0.f, 0.f);
      // conj(Fy[k,n]) c_k
      pv[q] = make_float2(a.x * ck.x + a.y * ck.y, a.x * ck.y - a.y * ck.x);
      qv[q] = make_float2(b.x, -b.y);  // conj(Fx[k,m])
    }
  };
  auto sstore = [&](int b) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Ps[b][lk][lc + q] = pv[q];
      Qs[b][lk][lc + q] = qv[q];
    }
  };
  gload(0);
  sstore(0);
  __syncthreads();
  int b = 0;
  for (int k0 = 0; k0 < K; k0 += TS) {
    const bool more = k0 + TS < K;
    if (more) gload(k0 + TS);
    mma_stage<16>(Ps[b], Qs[b], ty, tx, acc);
    if (more) sstore(b ^ 1);
    __syncthreads();
    b ^= 1;
  }

  float factor = 0.f;
  if (EPI == 1) factor = 2.f * amp_factor / st->c_scale;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n = n0 + ty * 4 + i;
    if (n >= ny) continue;
    float v[4];
    float2 ev[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + tx * 4 + j;
      if (EPI == 0) {
        v[j] = ofa_arg(acc[i][j].y, acc[i][j].x);
        float s, cs;
        sincosf(v[j], &s, &cs);
        const float a = m < nx ? amp[(size_t)n * nx + m] : 0.f;
        ev[j] = make_float2(a * cs, a * s);
      } else if (m < nx) {
        float s, cs;
        sincosf(phi_in[(size_t)n * nx + m], &s, &cs);
        v[j] = factor * amp[(size_t)n * nx + m] * (cs * acc[i][j].y - s * acc[i][j].x);
      } else {
        v[j] = 0.f;
      }
    }
    const int m = m0 + tx * 4;
    float* dst = out + (size_t)n * nx + m;
    if ((nx & 3) == 0 && m + 3 < nx) {
      *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
      if (EPI == 0) {
        float4* ed = reinterpret_cast<float4*>(e_out + (size_t)n * nx + m);
        ed[0] = make_float4(ev[0].x, ev[0].y, ev[1].x, ev[1].y);
        ed[1] = make_float4(ev[2].x, ev[2].y, ev[3].x, ev[3].y);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (m + j < nx) {
          dst[j] = v[j];
          if (EPI == 0) e_out[(size_t)n * nx + m + j] = ev[j];
        }
    }
  }
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

constexpr int FWD_SPLIT = 1;  // contraction parts of the forward (grid z)

int simt_fwd_tiles(int ny) { return FWD_SPLIT * ((ny + T64 - 1) / T64); }

void launch_field_f32(const float* phi, const float* amp, int nx, int ny, float2* e,
                      cudaStream_t s) {
  const size_t n = (size_t)nx * ny;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  field_f32_kernel<<<(unsigned)blocks, 256, 0, s>>>(phi, amp, n, e);
}

void launch_fwd_simt(const float2* e32, const float2* fx, const float2* fy, int nx, int ny, int K,
                     int kp, float2* part, const int* done, cudaStream_t s) {
  dim3 grid((K + T64 - 1) / T64, (ny + T64 - 1) / T64, FWD_SPLIT);
  fwd_simt_kernel<false><<<grid, 256, 0, s>>>(e32, fx, fy, nx, ny, K, kp, part, done);
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
  fwd_simt_kernel<true><<<grid, 256, 0, s>>>(e32, fxu, nullptr, nx, ny, ux, ux, gt, nullptr);
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

void launch_bwd_simt(const float2* c, const float2* fx, const float2* fy, int nx, int ny, int K,
                     const float* amp, float* phi, float2* e32, const int* done, cudaStream_t s) {
  dim3 grid((nx + T64 - 1) / T64, (ny + T64 - 1) / T64);
  bwd_simt_kernel<0><<<grid, 256, 0, s>>>(c, fx, fy, nx, ny, K, phi, e32, nullptr, amp, 0.f,
                                          nullptr, done);
}

void launch_grad_simt(const float2* c, const float2* fx, const float2* fy, int nx, int ny, int K,
                      const float* phi, const float* amp, float amp_factor,
                      const OfaDevState* st, float* grad, cudaStream_t s) {
  dim3 grid((nx + T64 - 1) / T64, (ny + T64 - 1) / T64);
  bwd_simt_kernel<1><<<grid, 256, 0, s>>>(c, fx, fy, nx, ny, K, grad, nullptr, phi, amp,
                                          amp_factor, st, nullptr);
}
