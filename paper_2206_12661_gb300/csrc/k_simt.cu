// FP32 CUDA-core form of the two MTP products (kernels (b) and (d), OFA_PREC_FP32).
//
// Forward (Eq. 2 at the foci): G[n,k] = sum_m E[n,m] Fx[k,m] with the pupil
// field E = A exp(i phi) formed on the fly from phi and A (fused phase->field
// prologue), then the per-focus dot Theta_k = sum_n Fy[k,n] G[n,k] reduced
// inside the tile; each 64-row tile writes one deterministic partial Theta.
//
// Inverse (Algorithm 1, inverse propagation read as the adjoint of Eq. 2):
// E'[n,m] = sum_k conj(Fy[k,n]) c_k conj(Fx[k,m]), fused with the phase-only
// projection phi = arg(E') (or, for the gradient, 2 Im(conj(E) E')).
//
// Both are 64 x 64 complex tiles, 256 threads, 4 x 4 complex accumulators per
// thread, 16-deep steps staged through shared memory with register prefetch.
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

__global__ void __launch_bounds__(256) fwd_simt_kernel(
    const float* __restrict__ phi, const float* __restrict__ amp, const float2* __restrict__ fx,
    const float2* __restrict__ fy, int nx, int ny, int K, int kp, float2* __restrict__ part,
    const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  __shared__ __align__(16) float2 Es[TS][T64];
  __shared__ __align__(16) float2 Fs[TS][T64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int n0 = blockIdx.y * T64, k0 = blockIdx.x * T64;
  const int lr = tid >> 2, lc = (tid & 3) * 4;

  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

  float pv[4], av[4];
  float2 fv[4];
  auto gload = [&](int m0) {
    const int n = n0 + lr, k = k0 + lr;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = m0 + lc + q;
      const bool ok_e = n < ny && m < nx;
      pv[q] = ok_e ? phi[(size_t)n * nx + m] : 0.f;
      av[q] = ok_e ? amp[(size_t)n * nx + m] : 0.f;
      fv[q] = (k < K && m < nx) ? fx[(size_t)k * nx + m] : make_float2(0.f, 0.f);
    }
  };
  gload(0);
  for (int m0 = 0; m0 < nx; m0 += TS) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float s, c;
      sincosf(pv[q], &s, &c);
      Es[lc + q][lr] = make_float2(av[q] * c, av[q] * s);   // E = A exp(i phi)
      Fs[lc + q][lr] = fv[q];
    }
    __syncthreads();
    if (m0 + TS < nx) gload(m0 + TS);
#pragma unroll
    for (int mm = 0; mm < TS; ++mm) {
      const float4 e01 = *reinterpret_cast<const float4*>(&Es[mm][ty * 4]);
      const float4 e23 = *reinterpret_cast<const float4*>(&Es[mm][ty * 4 + 2]);
      const float4 f01 = *reinterpret_cast<const float4*>(&Fs[mm][tx * 4]);
      const float4 f23 = *reinterpret_cast<const float4*>(&Fs[mm][tx * 4 + 2]);
      const float2 e[4] = {make_float2(e01.x, e01.y), make_float2(e01.z, e01.w),
                           make_float2(e23.x, e23.y), make_float2(e23.z, e23.w)};
      const float2 f[4] = {make_float2(f01.x, f01.y), make_float2(f01.z, f01.w),
                           make_float2(f23.x, f23.y), make_float2(f23.z, f23.w)};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cmac(acc[i][j], e[i], f[j]);
    }
  }

  // Per-focus dot with the Fy rows, reduced over the tile's 64 rows in fixed order.
  __syncthreads();
  float2* red = &Es[0][0];  // 16 x 64 float2
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
    if (k < kp) part[(size_t)blockIdx.y * kp + k] = a;
  }
}

// EPI 0: phi = atan2(Im E', Re E').  EPI 1: grad = f 2 A (cos phi Im B - sin phi Re B).
template <int EPI>
__global__ void __launch_bounds__(256) bwd_simt_kernel(
    const float2* __restrict__ c, const float2* __restrict__ fx, const float2* __restrict__ fy,
    int nx, int ny, int K, float* __restrict__ out, const float* __restrict__ phi_in,
    const float* __restrict__ amp, float amp_factor, const OfaDevState* __restrict__ st,
    const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  __shared__ __align__(16) float2 Ps[TS][T64];
  __shared__ __align__(16) float2 Qs[TS][T64];
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
  gload(0);
  for (int k0 = 0; k0 < K; k0 += TS) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Ps[lk][lc + q] = pv[q];
      Qs[lk][lc + q] = qv[q];
    }
    __syncthreads();
    if (k0 + TS < K) gload(k0 + TS);
#pragma unroll
    for (int kk = 0; kk < TS; ++kk) {
      const float4 p01 = *reinterpret_cast<const float4*>(&Ps[kk][ty * 4]);
      const float4 p23 = *reinterpret_cast<const float4*>(&Ps[kk][ty * 4 + 2]);
      const float4 q01 = *reinterpret_cast<const float4*>(&Qs[kk][tx * 4]);
      const float4 q23 = *reinterpret_cast<const float4*>(&Qs[kk][tx * 4 + 2]);
      const float2 p[4] = {make_float2(p01.x, p01.y), make_float2(p01.z, p01.w),
                           make_float2(p23.x, p23.y), make_float2(p23.z, p23.w)};
      const float2 qq[4] = {make_float2(q01.x, q01.y), make_float2(q01.z, q01.w),
                            make_float2(q23.x, q23.y), make_float2(q23.z, q23.w)};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cmac(acc[i][j], p[i], qq[j]);
    }
  }

  float factor = 0.f;
  if (EPI == 1) factor = 2.f * amp_factor / st->c_scale;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n = n0 + ty * 4 + i;
    if (n >= ny) continue;
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + tx * 4 + j;
      if (EPI == 0) {
        v[j] = ofa_arg(acc[i][j].y, acc[i][j].x);
      } else if (m < nx) {
        float s, cc;
        sincosf(phi_in[(size_t)n * nx + m], &s, &cc);
        v[j] = factor * amp[(size_t)n * nx + m] * (cc * acc[i][j].y - s * acc[i][j].x);
      } else {
        v[j] = 0.f;
      }
    }
    const int m = m0 + tx * 4;
    float* dst = out + (size_t)n * nx + m;
    if ((nx & 3) == 0 && m + 3 < nx) {
      *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (m + j < nx) dst[j] = v[j];
    }
  }
}

}  // namespace

int simt_fwd_tiles(int ny) { return (ny + T64 - 1) / T64; }

void launch_fwd_simt(const float* phi, const float* amp, const float2* fx, const float2* fy,
                     int nx, int ny, int K, int kp, float2* part, const int* done,
                     cudaStream_t s) {
  dim3 grid((K + T64 - 1) / T64, (ny + T64 - 1) / T64);
  fwd_simt_kernel<<<grid, 256, 0, s>>>(phi, amp, fx, fy, nx, ny, K, kp, part, done);
}

void launch_bwd_simt(const float2* c, const float2* fx, const float2* fy, int nx, int ny, int K,
                     float* phi, const int* done, cudaStream_t s) {
  dim3 grid((nx + T64 - 1) / T64, (ny + T64 - 1) / T64);
  bwd_simt_kernel<0><<<grid, 256, 0, s>>>(c, fx, fy, nx, ny, K, phi, nullptr, nullptr, 0.f,
                                          nullptr, done);
}

void launch_grad_simt(const float2* c, const float2* fx, const float2* fy, int nx, int ny, int K,
                      const float* phi, const float* amp, float amp_factor,
                      const OfaDevState* st, float* grad, cudaStream_t s) {
  dim3 grid((nx + T64 - 1) / T64, (ny + T64 - 1) / T64);
  bwd_simt_kernel<1><<<grid, 256, 0, s>>>(c, fx, fy, nx, ny, K, grad, phi, amp, amp_factor, st,
                                          nullptr);
}
