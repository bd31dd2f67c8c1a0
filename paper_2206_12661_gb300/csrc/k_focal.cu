// Kernel (c): focal-plane statistics and the generalized weighting update of
// Algorithm 1, plus the per-iteration left operand of the inverse product.
//
// One CTA of 1024 threads sums the per-tile partials of Theta in a fixed order,
// forms I_k = |Theta_k|^2, S = sum I, the intensity accuracy
//   xi = 1 - ||t - Ihat|| / ||Ihat||,  Ihat = I / S,  t = I~ / sum I~
// (fixed-order shuffle-tree reductions, so every run is bitwise reproducible;
// FP32 inside the loop, FP64 for the reported statistic), records xi, applies
// the loop's break test, then updates
//   w_k <- w_k sqrt(t_k / Ihat_k)                       (generalized weighting)
//   c_k  = w_k sqrt(t_k) exp(i arg Theta_k) * 2^s       (focused field)
// where 2^s is the power of two that brings max |c| into [1/2, 1): arg() of
// the inverse product does not see a positive scale, and the tensor-core
// operand formats want bounded magnitudes.
#include <math_constants.h>

#include "ofa_internal.cuh"
#include "ofa_focal.cuh"
#include "ofa_split.cuh"

namespace {

constexpr int FT = 1024;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  return r;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = sh[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = fmax(r, sh[i]);
  return r;
}

// Fixed-order FP32 block reductions (every lane of every warp ends with the same
// bits: xor-butterfly in registers, then warp partials summed in warp order).
template <int N>
__device__ __forceinline__ void block_sum_f(float (&v)[N], float* sh) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < N; ++i) sh[i * 32 + (threadIdx.x >> 5)] = v[i];
  __syncthreads();
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float r = 0.f;
    for (int w = 0; w < nw; ++w) r += sh[i * 32 + w];
    v[i] = r;
  }
}

__device__ __forceinline__ float block_max_f(float v, float* sh) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = sh[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, sh[w]);
  return r;
}

// Per-focus work of one loop iteration runs in FP32; the statistics of mode 1
// (the reported intensity accuracy and uniformity) are reduced in FP64.
__global__ void __launch_bounds__(FT) focal_kernel(
    const float2* __restrict__ part, int n_part, int kp, int K, const float* __restrict__ t,
    float* __restrict__ w, float2* __restrict__ theta, float* __restrict__ inten,
    float2* __restrict__ c, double* __restrict__ hist, OfaDevState* __restrict__ st, int mode,
    int weighting, float out_scale, double energy) {
  __shared__ float shf[4 * 32];
  __shared__ double sh[32];
  if (mode == 0 && st->done) return;
  const int tid = threadIdx.x;

  // Theta_k = sum over tiles in fixed order; I_k = |Theta_k|^2.
  float r1[1] = {0.f};
  double s_i = 0.0;
  for (int k = tid; k < K; k += FT) {
    float2 a = make_float2(0.f, 0.f);
    for (int p = 0; p < n_part; ++p) {
      const float2 v = part[(size_t)p * kp + k];
      a.x += v.x;
      a.y += v.y;
    }
    const float ik = a.x * a.x + a.y * a.y;
    if (mode == 2) {
      theta[k] = make_float2(a.x * out_scale, a.y * out_scale);
      inten[k] = ik * out_scale * out_scale;
    } else {
      theta[k] = a;
      inten[k] = ik;
    }
    r1[0] += ik;
    if (mode == 1) s_i += ik;
  }
  if (mode == 2) return;

  if (mode == 1) {
    const double S = block_sum(s_i, sh);
    if (!(S > 0.0) || !isfinite(S)) {
      if (tid == 0) atomicOr(&st->err, OFA_ERRBIT_NUMERIC);
      return;
    }
    double d2 = 0.0, n2 = 0.0, rmin = CUDART_INF, rmax = 0.0;
    for (int k = tid; k < K; k += FT) {
      const double ih = (double)inten[k] / S;
      const double tk = (double)t[k];
      d2 += (tk - ih) * (tk - ih);
      n2 += ih * ih;
      if (tk > 0.0) {
        const double r = ih / tk;
        rmin = fmin(rmin, r);
        rmax = fmax(rmax, r);
      }
    }
    d2 = block_sum(d2, sh);
    n2 = block_sum(n2, sh);
    rmax = block_max(rmax, sh);
    rmin = -block_max(-rmin, sh);
    if (tid == 0) {
      const double s2 = (double)out_scale * out_scale;
      st->xi = 1.0 - sqrt(d2 / n2);
      st->uniformity = 1.0 - (rmax - rmin) / (rmax + rmin);
      st->sum_i = S * s2;
      st->energy_fraction = energy > 0.0 ? S * s2 / energy : 0.0;
    }
    return;
  }

  // mode 0: one loop iteration of Algorithm 1.
  block_sum_f(r1, shf);
  const float S = r1[0];
  if (!(S > 0.f) || !isfinite(S)) {
    if (tid == 0) {
      atomicOr(&st->err, OFA_ERRBIT_NUMERIC);
      st->done = 1;
    }
    return;
  }
  const float inv_s = 1.f / S;
  // xi terms and the largest new focused-field magnitude, one reduction round
  float r2[2] = {0.f, 0.f};
  float mx = 0.f;
  for (int k = tid; k < K; k += FT) {
    const float ih = inten[k] * inv_s;
    const float tk = t[k];
    const float d = tk - ih;
    r2[0] += d * d;
    r2[1] += ih * ih;
    float wk = w[k];
    const float stk = sqrtf(tk);
    if (weighting) wk *= stk * rsqrtf(fmaxf(ih, 1e-30f));  // w sqrt(t / Ihat)
    mx = fmaxf(mx, wk * stk);
  }
  block_sum_f(r2, shf + 32);
  mx = block_max_f(mx, shf + 96);
  const double xi = 1.0 - sqrt((double)r2[0] / (double)r2[1]);
  if (tid == 0) {
    const int h = st->hist_count;
    hist[h % OFA_HIST_CAP] = xi;
    st->hist_count = h + 1;
    st->xi = xi;
  }
  const double thr = st->threshold;
  if (thr > 0.0 && thr < 1.0 && xi > thr) {
    if (tid == 0) st->done = 1;
    return;
  }
  int e = 0;
  frexpf(mx, &e);
  const float scale = mx > 0.f ? exp2f((float)-e) : 1.f;
  for (int k = tid; k < kp; k += FT) {
    float2 ck = make_float2(0.f, 0.f);
    if (k < K) {
      const float tk = t[k];
      float wk = w[k];
      if (weighting) {
        wk *= sqrtf(tk) * rsqrtf(fmaxf(inten[k] * inv_s, 1e-30f));  // w_j = w_{j-1} sqrt(t / Ihat)
        w[k] = wk;
      }
      const float mag = wk * sqrtf(tk) * scale;
      const float2 th = theta[k];
      const float rr = th.x * th.x + th.y * th.y;
      if (rr > 0.f) {
        const float inv = rsqrtf(rr);
        ck = make_float2(mag * th.x * inv, mag * th.y * inv);
      } else {
        ck = make_float2(mag, 0.f);  // arg(0) = 0
      }
    }
    c[k] = ck;
  }
  if (tid == 0) {
    st->j += 1;
    st->c_scale = scale;
  }
}

// One loop iteration (mode 0): Theta_k from the per-tile partials (fixed order),
// then the shared focal routine of ofa_focal.cuh on 1024 threads.
__global__ void __launch_bounds__(FT) focal_iter_kernel(
    const float2* __restrict__ part, int n_part, int kp, int K, const float* __restrict__ t,
    float* __restrict__ w, float2* __restrict__ theta, float2* __restrict__ c,
    double* __restrict__ hist, OfaDevState* __restrict__ st, int weighting) {
  __shared__ float sh[4 * 33];
  if (st->done) return;
  for (int k = threadIdx.x; k < K; k += FT) {
    float2 a = make_float2(0.f, 0.f);
    for (int p = 0; p < n_part; ++p) {
      const float2 v = part[(size_t)p * kp + k];
      a.x += v.x;
      a.y += v.y;
    }
    theta[k] = a;
  }
  __syncthreads();
  ofa_focal::iterate<FT>(theta, K, kp, t, w, c, hist, st, weighting, sh, (int)threadIdx.x,
                         ofa_focal::BarBlock());
}

// The loop's focal step with captured intensities (camera in the loop).
__global__ void __launch_bounds__(FT) focal_measured_kernel(
    const float2* __restrict__ part, int n_part, int kp, int K, const float* __restrict__ t,
    float* __restrict__ w, float2* __restrict__ theta, float2* __restrict__ c,
    double* __restrict__ hist, OfaDevState* __restrict__ st, int weighting,
    const float* __restrict__ meas) {
  __shared__ float sh[4 * 33];
  if (st->done) return;
  for (int k = threadIdx.x; k < K; k += FT) {
    float2 a = make_float2(0.f, 0.f);
    for (int p = 0; p < n_part; ++p) {
      const float2 v = part[(size_t)p * kp + k];
      a.x += v.x;
      a.y += v.y;
    }
    theta[k] = a;
  }
  __syncthreads();
  ofa_focal::iterate<FT>(theta, K, kp, t, w, c, hist, st, weighting, sh, (int)threadIdx.x,
                         ofa_focal::BarBlock(), meas);
}

// Mode 0 for K <= 4096: everything from registers (ofa_focal::iterate_regs).
__global__ void __launch_bounds__(FT) focal_regs_kernel(
    const float2* __restrict__ part, int n_part, int kp, int K, const float* __restrict__ t,
    float* __restrict__ w, float2* __restrict__ c, double* __restrict__ hist,
    OfaDevState* __restrict__ st, int weighting) {
  __shared__ float sh[4 * 33];
  if (st->done) return;
  ofa_focal::iterate_regs<FT, 4>(part, n_part, K, kp, t, w, c, hist, st, weighting, sh,
                                 (int)threadIdx.x, ofa_focal::BarBlock());
}

__global__ void control_kernel(OfaDevState* st, double thr, int reset_done) {
  st->threshold = thr;
  if (reset_done) st->done = 0;
}

__global__ void set_j_kernel(OfaDevState* st, int j, int reset_hist) {
  st->j = j;
  st->done = 0;
  if (reset_hist) st->hist_count = 0;
}

// c_k = g_k Theta_k (gradient of a loss of the intensities), power-of-two scaled.
__global__ void __launch_bounds__(FT) grad_c_kernel(const float2* __restrict__ theta,
                                                    const float* __restrict__ g, int K, int kp,
                                                    float in_scale, float2* __restrict__ c,
                                                    OfaDevState* __restrict__ st) {
  __shared__ double sh[32];
  double mx = 0.0;
  for (int k = threadIdx.x; k < K; k += FT) {
    const float2 th = theta[k];
    const double a = fabs((double)g[k]) * sqrt((double)th.x * th.x + (double)th.y * th.y);
    mx = fmax(mx, a * in_scale);
  }
  mx = block_max(mx, sh);
  int e = 0;
  frexp(mx, &e);
  const float scale = mx > 0.0 ? (float)ldexp(1.0, -e) : 1.f;
  for (int k = threadIdx.x; k < kp; k += FT) {
    float2 ck = make_float2(0.f, 0.f);
    if (k < K) {
      const float f = g[k] * in_scale * scale;
      ck = make_float2(f * theta[k].x, f * theta[k].y);
    }
    c[k] = ck;
  }
  if (threadIdx.x == 0) st->c_scale = scale;
}

// The intensity loss of the differentiable form and the start of its adjoint, one
// block: I_k = |Theta_k|^2, S = sum I, Ihat = I / S, d = Ihat - t,
//   L = sum_k d_k^2,   g_k = dL/dI_k = (2 / S) (d_k - sum_j d_j Ihat_j),
// then c_k = g_k Theta_k scaled by the power of two that brings max |c| into [1/2, 1)
// (recorded in st->c_scale; the gradient epilogue divides it out).  S, L and the inner
// sum are reduced in FP64.  loss_hist[*step] (or [0] without a step counter) = L when
// that index lies in [0, loss_cap).
__global__ void __launch_bounds__(FT) loss_grad_c_kernel(const float2* __restrict__ theta,
                                                         const float* __restrict__ t, int K,
                                                         int kp, float2* __restrict__ c,
                                                         OfaDevState* __restrict__ st,
                                                         float* __restrict__ loss_hist,
                                                         int loss_cap,
                                                         const int* __restrict__ step) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < K; k += FT) {
    const float2 a = theta[k];
    s += (double)a.x * a.x + (double)a.y * a.y;
  }
  const double S = block_sum(s, sh);
  const double inv_s = S > 0.0 ? 1.0 / S : 0.0;
  double l = 0.0, dsum = 0.0;
  for (int k = threadIdx.x; k < K; k += FT) {
    const float2 a = theta[k];
    const double ih = ((double)a.x * a.x + (double)a.y * a.y) * inv_s;
    const double d = ih - (double)t[k];
    l += d * d;
    dsum += d * ih;
  }
  const double L = block_sum(l, sh);
  const double D = block_sum(dsum, sh);
  double mx = 0.0;
  for (int k = threadIdx.x; k < K; k += FT) {
    const float2 a = theta[k];
    const double ih = ((double)a.x * a.x + (double)a.y * a.y) * inv_s;
    const double g = 2.0 * inv_s * ((ih - (double)t[k]) - D);
    mx = fmax(mx, fabs(g) * sqrt((double)a.x * a.x + (double)a.y * a.y));
  }
  mx = block_max(mx, sh);
  int e = 0;
  frexp(mx, &e);
  const double scale = mx > 0.0 ? ldexp(1.0, -e) : 1.0;
  for (int k = threadIdx.x; k < kp; k += FT) {
    float2 ck = make_float2(0.f, 0.f);
    if (k < K) {
      const float2 a = theta[k];
      const double ih = ((double)a.x * a.x + (double)a.y * a.y) * inv_s;
      const double g = 2.0 * inv_s * ((ih - (double)t[k]) - D) * scale;
      ck = make_float2((float)(g * a.x), (float)(g * a.y));
    }
    c[k] = ck;
  }
  if (threadIdx.x == 0) {
    st->c_scale = (float)scale;
    const int i = step ? *step : 0;
    if (loss_hist && i >= 0 && i < loss_cap) loss_hist[i] = (float)L;
  }
}

// The loss adjoint for K <= 256 KPR foci, each thread's foci held in registers, 256
// threads.  The same quantities as loss_grad_c_kernel; the FP64 work is what carries
// the cancellation: d_k = Ihat_k - t_k is formed in FP64 from the FP32 Theta (then
// rounded), and the cross-warp partial sums are added in FP64.  Per-element products
// and the in-warp sums are FP32.
constexpr int LT = 256;
template <int KPR>
__global__ void __launch_bounds__(LT) loss_grad_c_regs_kernel(
    const float2* __restrict__ theta, const float* __restrict__ t, int K, int kp,
    float2* __restrict__ c, OfaDevState* __restrict__ st, float* __restrict__ loss_hist,
    int loss_cap, const int* __restrict__ step) {
  __shared__ double shd[3 * (LT / 32) + 4];
  __shared__ float shm[LT / 32 + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // sum over the block: in-warp FP32 butterfly, then thread 0 adds the warp partials
  // in FP64 in warp order and every thread reads the result
  auto block_sum_fd = [&](float (&v)[2], int n, double (&out)[2]) {
    for (int i = 0; i < n; ++i)
#pragma unroll
      for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    __syncthreads();
    if (lane == 0)
      for (int i = 0; i < n; ++i) shd[i * (LT / 32) + warp] = (double)v[i];
    __syncthreads();
    if (tid == 0)
      for (int i = 0; i < n; ++i) {
        double r = 0.0;
#pragma unroll
        for (int w = 0; w < LT / 32; ++w) r += shd[i * (LT / 32) + w];
        shd[3 * (LT / 32) + i] = r;
        if (i == 0 && n == 1) shd[3 * (LT / 32) + 1] = r > 0.0 ? 1.0 / r : 0.0;
      }
    __syncthreads();
    for (int i = 0; i < 2; ++i) out[i] = shd[3 * (LT / 32) + i];
  };
  float2 a[KPR];
  float tk[KPR];
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    const int k = tid + i * LT;
    a[i] = k < K ? theta[k] : make_float2(0.f, 0.f);
    tk[i] = k < K ? t[k] : 0.f;
  }
  float v[2] = {0.f, 0.f};
  double r[2];
#pragma unroll
  for (int i = 0; i < KPR; ++i) v[0] += fmaf(a[i].x, a[i].x, a[i].y * a[i].y);
  block_sum_fd(v, 1, r);   // r = {S, 1 / S}
  const double inv_s = r[1];
  const float inv_sf = (float)inv_s;
  float df[KPR];
  v[0] = v[1] = 0.f;
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    const double ih = ((double)a[i].x * a[i].x + (double)a[i].y * a[i].y) * inv_s;
    df[i] = tid + i * LT < K ? (float)(ih - (double)tk[i]) : 0.f;
    v[0] += df[i] * df[i];
    v[1] += df[i] * (float)ih;
  }
  block_sum_fd(v, 2, r);
  const double L = r[0];
  const float Df = (float)r[1];
  float g[KPR], mx = 0.f;
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    g[i] = 2.f * inv_sf * (df[i] - Df);
    mx = fmaxf(mx, fabsf(g[i]) * sqrtf(fmaf(a[i].x, a[i].x, a[i].y * a[i].y)));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) shm[warp] = mx;
  __syncthreads();
  mx = shm[0];
#pragma unroll
  for (int w = 1; w < LT / 32; ++w) mx = fmaxf(mx, shm[w]);
  int e = 0;
  frexpf(mx, &e);
  const float scale = mx > 0.f ? ldexpf(1.f, -e) : 1.f;
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    const int k = tid + i * LT;
    if (k >= kp) break;
    const float gs = g[i] * scale;
    c[k] = k < K ? make_float2(gs * a[i].x, gs * a[i].y) : make_float2(0.f, 0.f);
  }
  if (tid == 0) {
    st->c_scale = scale;
    const int i = step ? *step : 0;
    if (loss_hist && i >= 0 && i < loss_cap) loss_hist[i] = (float)L;
  }
}

// One Adam update of n parameters (the published algorithm with torch's defaults for
// the order of operations): t = *step + 1, m <- b1 m + (1 - b1) g,
// v <- b2 v + (1 - b2) g^2, x <- x - lr / (1 - b1^t) m / (sqrt(v) / sqrt(1 - b2^t) + eps).
// adam_prepare_kernel advances the step and forms the two bias corrections once (one
// thread); adam_kernel applies the update, four parameters per thread when the
// four arrays are 16-byte aligned.
// 1 - b^t = -expm1(t log(b)), log(b) = log1p(-(1 - b)): accurate to a few FP32 ulps
// relative also where b^t is close to 1 (b2 = 0.999 early on), where 1 - powf(b, t)
// would cancel.  1 - b is exact in FP32 for b in [1/2, 1].
__device__ __forceinline__ float one_minus_pow(float b, float t) {
  return -expm1f(t * log1pf(-(1.f - b)));
}

__global__ void adam_prepare_kernel(int* __restrict__ step, OfaDevState* __restrict__ st,
                                    float lr, float b1, float b2) {
  const int t = *step + 1;
  *step = t;
  st->adam_step_size = lr / one_minus_pow(b1, (float)t);
  st->adam_bc2_sqrt = sqrtf(one_minus_pow(b2, (float)t));
}

__device__ __forceinline__ void adam_one(float& x, float g, float& m, float& v, float b1,
                                         float b2, float eps, float step_size,
                                         float bc2_sqrt) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  x -= step_size * (m / (sqrtf(v) / bc2_sqrt + eps));
}

template <bool VEC>
__global__ void adam_kernel(float* __restrict__ x, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v,
                            const OfaDevState* __restrict__ st, size_t n, float b1, float b2,
                            float eps) {
  const float step_size = st->adam_step_size, bc2_sqrt = st->adam_bc2_sqrt;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (VEC) {
    if (4 * i + 3 < n) {
      float4 xv = reinterpret_cast<float4*>(x)[i];
      const float4 gv = reinterpret_cast<const float4*>(g)[i];
      float4 mv = reinterpret_cast<float4*>(m)[i];
      float4 vv = reinterpret_cast<float4*>(v)[i];
      adam_one(xv.x, gv.x, mv.x, vv.x, b1, b2, eps, step_size, bc2_sqrt);
      adam_one(xv.y, gv.y, mv.y, vv.y, b1, b2, eps, step_size, bc2_sqrt);
      adam_one(xv.z, gv.z, mv.z, vv.z, b1, b2, eps, step_size, bc2_sqrt);
      adam_one(xv.w, gv.w, mv.w, vv.w, b1, b2, eps, step_size, bc2_sqrt);
      reinterpret_cast<float4*>(x)[i] = xv;
      reinterpret_cast<float4*>(m)[i] = mv;
      reinterpret_cast<float4*>(v)[i] = vv;
    } else {
      for (size_t j = 4 * i; j < n; ++j) adam_one(x[j], g[j], m[j], v[j], b1, b2, eps,
                                                   step_size, bc2_sqrt);
    }
  } else if (i < n) {
    adam_one(x[i], g[i], m[i], v[i], b1, b2, eps, step_size, bc2_sqrt);
  }
}

// P[n][2k..2k+1] = conj(Fy[k,n]) c_k in the operand format of the precision;
// four foci per thread (kp is a multiple of 128): 16-byte loads and stores.
__global__ void build_p_kernel(const float2* __restrict__ fyT, const float2* __restrict__ c,
                               const int* __restrict__ done, int nyp, int kp, int prec, void* hi,
                               void* lo) {
  // programmatic dependent launch: schedule the inverse product now, then wait
  // for the forward kernel (which produced c) to complete
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (done != nullptr && *done) return;
  const size_t quads = (size_t)nyp * kp / 4;
  const bool wide = prec == OFA_PREC_TF32;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < quads;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t e0 = 4 * i;                 // first complex element
    const int k0 = (int)(e0 % kp);
    const float4 f01 = __ldg(reinterpret_cast<const float4*>(fyT + e0));
    const float4 f23 = __ldg(reinterpret_cast<const float4*>(fyT + e0) + 1);
    const float4 c01 = __ldg(reinterpret_cast<const float4*>(c + k0));
    const float4 c23 = __ldg(reinterpret_cast<const float4*>(c + k0) + 1);
    const float fr[4] = {f01.x, f01.z, f23.x, f23.z}, fi[4] = {f01.y, f01.w, f23.y, f23.w};
    const float cr[4] = {c01.x, c01.z, c23.x, c23.z}, ci[4] = {c01.y, c01.w, c23.y, c23.w};
    uint2 h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      split_pack(prec, fr[j] * cr[j] + fi[j] * ci[j], fr[j] * ci[j] - fi[j] * cr[j], h[j], l[j]);
    if (wide) {
      uint4* dst = reinterpret_cast<uint4*>(static_cast<float*>(hi) + 2 * e0);
      dst[0] = make_uint4(h[0].x, h[0].y, h[1].x, h[1].y);
      dst[1] = make_uint4(h[2].x, h[2].y, h[3].x, h[3].y);
    } else {
      reinterpret_cast<uint4*>(static_cast<uint16_t*>(hi) + 2 * e0)[0] =
          make_uint4(h[0].x, h[1].x, h[2].x, h[3].x);
      if (lo != nullptr)
        reinterpret_cast<uint4*>(static_cast<uint16_t*>(lo) + 2 * e0)[0] =
            make_uint4(l[0].x, l[1].x, l[2].x, l[3].x);
    }
  }
}

// The same operand build over many plans: block b converts quads
// [chunks[b].y, chunks[b].z) of plan chunks[b].x.
__global__ void build_p_group_kernel(const BpGroupItem* __restrict__ items,
                                     const int4* __restrict__ chunks, int prec) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int4 ch = chunks[blockIdx.x];
  const BpGroupItem it = items[ch.x];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const bool wide = prec == OFA_PREC_TF32;
  for (int i = ch.y + (int)threadIdx.x; i < ch.z; i += blockDim.x) {
    const size_t e0 = 4 * (size_t)i;
    const int k0 = (int)(e0 % it.kp);
    const float4 f01 = __ldg(reinterpret_cast<const float4*>(it.fyT + e0));
    const float4 f23 = __ldg(reinterpret_cast<const float4*>(it.fyT + e0) + 1);
    const float4 c01 = __ldg(reinterpret_cast<const float4*>(it.c + k0));
    const float4 c23 = __ldg(reinterpret_cast<const float4*>(it.c + k0) + 1);
    const float fr[4] = {f01.x, f01.z, f23.x, f23.z}, fi[4] = {f01.y, f01.w, f23.y, f23.w};
    const float cr[4] = {c01.x, c01.z, c23.x, c23.z}, ci[4] = {c01.y, c01.w, c23.y, c23.w};
    uint2 h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      split_pack(prec, fr[j] * cr[j] + fi[j] * ci[j], fr[j] * ci[j] - fi[j] * cr[j], h[j], l[j]);
    if (wide) {
      uint4* dst = reinterpret_cast<uint4*>(static_cast<float*>(it.hi) + 2 * e0);
      dst[0] = make_uint4(h[0].x, h[0].y, h[1].x, h[1].y);
      dst[1] = make_uint4(h[2].x, h[2].y, h[3].x, h[3].y);
    } else {
      reinterpret_cast<uint4*>(static_cast<uint16_t*>(it.hi) + 2 * e0)[0] =
          make_uint4(h[0].x, h[1].x, h[2].x, h[3].x);
      if (it.lo != nullptr)
        reinterpret_cast<uint4*>(static_cast<uint16_t*>(it.lo) + 2 * e0)[0] =
            make_uint4(l[0].x, l[1].x, l[2].x, l[3].x);
    }
  }
}

}  // namespace

void launch_build_p_group(const BpGroupItem* items, const int4* chunks, int n_chunks, int prec,
                          cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)n_chunks);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, build_p_group_kernel, items, chunks, prec);
}

void launch_focal(const float2* part, int n_part, int kp, int K, const float* t, float* w,
                  float2* theta, float* inten, float2* c, double* hist, OfaDevState* st, int mode,
                  int weighting, float out_scale, double energy, cudaStream_t s) {
  if (mode == 0 && K <= 4 * FT) {
    focal_regs_kernel<<<1, FT, 0, s>>>(reinterpret_cast<const float2*>(part), n_part, kp, K, t,
                                       w, c, hist, st, weighting);
    return;
  }
  if (mode == 0) {
    focal_iter_kernel<<<1, FT, 0, s>>>(part, n_part, kp, K, t, w, theta, c, hist, st, weighting);
    return;
  }
  focal_kernel<<<1, FT, 0, s>>>(part, n_part, kp, K, t, w, theta, inten, c, hist, st, mode,
                                weighting, out_scale, energy);
}

void launch_focal_measured(const float2* part, int n_part, int kp, int K, const float* t,
                           float* w, float2* theta, float2* c, double* hist, OfaDevState* st,
                           int weighting, const float* meas, cudaStream_t s) {
  focal_measured_kernel<<<1, FT, 0, s>>>(part, n_part, kp, K, t, w, theta, c, hist, st,
                                         weighting, meas);
}

void launch_control(OfaDevState* st, double threshold, int reset_done, cudaStream_t s) {
  control_kernel<<<1, 1, 0, s>>>(st, threshold, reset_done);
}

void launch_set_j(OfaDevState* st, int j, int reset_hist, cudaStream_t s) {
  set_j_kernel<<<1, 1, 0, s>>>(st, j, reset_hist);
}

void launch_grad_c(const float2* theta, const float* g, int K, int kp, float in_scale, float2* c,
                   OfaDevState* st, cudaStream_t s) {
  grad_c_kernel<<<1, FT, 0, s>>>(theta, g, K, kp, in_scale, c, st);
}

void launch_loss_grad_c(const float2* theta, const float* t, int K, int kp, float2* c,
                        OfaDevState* st, float* loss_hist, int loss_cap, const int* step,
                        cudaStream_t s) {
  if (K <= 2 * LT)
    loss_grad_c_regs_kernel<2><<<1, LT, 0, s>>>(theta, t, K, kp, c, st, loss_hist, loss_cap,
                                                step);
  else if (K <= 16 * LT)
    loss_grad_c_regs_kernel<16><<<1, LT, 0, s>>>(theta, t, K, kp, c, st, loss_hist, loss_cap,
                                                 step);
  else
    loss_grad_c_kernel<<<1, FT, 0, s>>>(theta, t, K, kp, c, st, loss_hist, loss_cap, step);
}

void launch_adam(float* x, const float* g, float* m, float* v, int* step, OfaDevState* st,
                 size_t n, float lr, float b1, float b2, float eps, cudaStream_t s) {
  adam_prepare_kernel<<<1, 1, 0, s>>>(step, st, lr, b1, b2);
  const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(g) |
                     reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) & 15) == 0;
  if (vec) {
    const size_t threads = (n + 3) / 4;
    adam_kernel<true><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(x, g, m, v, st, n, b1,
                                                                         b2, eps);
  } else {
    adam_kernel<false><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, g, m, v, st, n, b1, b2,
                                                                    eps);
  }
}

namespace {

// Separable grid form on the tensor cores: the focal step of the loop and the inverse's
// left operand in one launch.  Every block runs the focal step on Theta (the same
// fixed-order reductions over the same inputs, so every block holds the same bits; the
// weights are read from wprev, a copy taken before this launch, because block 0 alone
// writes the new w, c, the xi history and the loop state), places c_k at the grid
// point of focus k in shared memory (C, zero where no focus sits), and forms
// U[n][ix] = sum over the grid rows iy (in order) of conj(Fyu[iy][n]) C[iy][ix] for its
// eight rows n (one per warp; lane + 32 r = column ix, ux <= 128) into the operand
// planes [nyp][2 kpad] (columns ix >= ux and rows n >= ny are never written and stay
// zero).  The focal arithmetic is that of ofa_focal::iterate_regs.
constexpr int SEP_U_THREADS = 256, SEP_U_ROWS = 8, SEP_U_MAXY = 128;
constexpr size_t SEP_U_SMEM_MAX = 96 * 1024;   // the C grid, [uy][pitch] complex
template <int KPR>
__global__ void __launch_bounds__(SEP_U_THREADS) sep_focal_u_kernel(
    const float2* __restrict__ theta, const float* __restrict__ t,
    const float* __restrict__ wprev, float* __restrict__ w, float2* __restrict__ c,
    double* __restrict__ hist, OfaDevState* __restrict__ st, int weighting,
    const int2* __restrict__ ixy, int K, const float2* __restrict__ fyu,
    const int* __restrict__ done, int ny, int ux, int uy, int pitch, int kpad, int prec,
    void* hi, void* lo) {
  constexpr int NT = SEP_U_THREADS;
  extern __shared__ float2 cg[];                  // [uy][pitch]
  __shared__ float2 fy[SEP_U_MAXY][SEP_U_ROWS];   // conj(Fyu) of the block's rows
  __shared__ float sh[4 * 33 + 4];
  __shared__ int skip;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n0 = blockIdx.x * SEP_U_ROWS;
  const bool writer = blockIdx.x == 0;
  // what does not change over the loop, before the wait: the block's conj(Fyu), the
  // focus positions and targets, and the zero grid
  for (int e = tid; e < uy * SEP_U_ROWS; e += NT) {
    const int i = e / SEP_U_ROWS, r = e % SEP_U_ROWS, n = n0 + r;
    float2 v = make_float2(0.f, 0.f);
    if (n < ny) {
      const float2 f = __ldg(fyu + (size_t)i * ny + n);
      v = make_float2(f.x, -f.y);
    }
    fy[i][r] = v;
  }
  int2 q[KPR];
  float tk[KPR];
  bool in[KPR];
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    const int k = tid + i * NT;
    in[i] = k < K;
    q[i] = in[i] ? __ldg(ixy + k) : make_int2(0, 0);
    tk[i] = in[i] ? __ldg(t + k) : 0.f;
  }
  for (int e = tid; e < uy * pitch; e += NT) cg[e] = make_float2(0.f, 0.f);
  // programmatic dependent launch: schedule the inverse product now, then wait for
  // Theta and the weights' copy
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (tid == 0) skip = done != nullptr && __ldcg(done);   // one decision per block
  __syncthreads();
  if (skip) return;
  const double thr = st->threshold;
  float2 th[KPR];
  float wk[KPR], ik[KPR];
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    const int k = tid + i * NT;
    th[i] = in[i] ? __ldcg(theta + k) : make_float2(0.f, 0.f);
    wk[i] = in[i] ? __ldcg(wprev + k) : 0.f;
  }
  float r1[1] = {0.f};
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    ik[i] = th[i].x * th[i].x + th[i].y * th[i].y;
    r1[0] += ik[i];
  }
  ofa_focal::block_sum<NT>(r1, sh, tid, ofa_focal::BarBlock());
  const float S = r1[0];
  if (!(S > 0.f) || !isfinite(S)) {
    if (writer && tid == 0) {
      atomicOr(&st->err, OFA_ERRBIT_NUMERIC);
      st->done = 1;
    }
    return;
  }
  const float inv_s = 1.f / S;
  float r2[2] = {0.f, 0.f};
  float mx = 0.f;
  float sq[KPR];
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    sq[i] = sqrtf(tk[i]);
    if (!in[i]) continue;
    const float ih = ik[i] * inv_s;
    const float d = tk[i] - ih;
    r2[0] += d * d;
    r2[1] += ih * ih;
    if (weighting) wk[i] *= sq[i] * rsqrtf(fmaxf(ih, 1e-30f));  // w_j = w_{j-1} sqrt(t / Ihat)
    mx = fmaxf(mx, wk[i] * sq[i]);
  }
  ofa_focal::block_sum2_max<NT>(r2, mx, sh + 33, tid, ofa_focal::BarBlock());
  const float xi = 1.f - sqrtf(r2[0] / r2[1]);
  if (writer && tid == 0) {
    const int hcount = st->hist_count;
    hist[hcount % OFA_HIST_CAP] = (double)xi;
    st->hist_count = hcount + 1;
    st->xi = (double)xi;
  }
  if (thr > 0.0 && thr < 1.0 && (double)xi > thr) {
    if (writer && tid == 0) st->done = 1;
    return;
  }
  int e2 = 0;
  frexpf(mx, &e2);
  const float scale = mx > 0.f ? exp2f((float)-e2) : 1.f;
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    if (!in[i]) continue;
    const int k = tid + i * NT;
    const float mag = wk[i] * sq[i] * scale;
    float2 ck;
    if (ik[i] > 0.f) {
      const float inv = rsqrtf(ik[i]);
      ck = make_float2(mag * th[i].x * inv, mag * th[i].y * inv);
    } else {
      ck = make_float2(mag, 0.f);  // arg(0) = 0
    }
    cg[q[i].y * pitch + q[i].x] = ck;
    if (writer) {
      if (weighting) w[k] = wk[i];
      c[k] = ck;
    }
  }
  if (writer && tid == 0) {
    st->j = st->j + 1;
    st->c_scale = scale;
  }
  __syncthreads();
  // two accumulators per column (even and odd grid rows, added at the end): twice the
  // independent FMA chains
  float2 acc[4], acc2[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) acc[r] = acc2[r] = make_float2(0.f, 0.f);
  const int R = pitch / 32;
  auto cmac_u = [](float2& a, float2 g, float2 v) {
    a.x = fmaf(g.x, v.x, a.x);
    a.x = fmaf(-g.y, v.y, a.x);
    a.y = fmaf(g.x, v.y, a.y);
    a.y = fmaf(g.y, v.x, a.y);
  };
  int iy = 0;
  for (; iy + 1 < uy; iy += 2) {
    const float2 g0 = fy[iy][warp], g1 = fy[iy + 1][warp];
    const float2* row = cg + iy * pitch + lane;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (r >= R) break;
      cmac_u(acc[r], g0, row[32 * r]);
      cmac_u(acc2[r], g1, row[pitch + 32 * r]);
    }
  }
  if (iy < uy) {
    const float2 g0 = fy[iy][warp];
    const float2* row = cg + iy * pitch + lane;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (r >= R) break;
      cmac_u(acc[r], g0, row[32 * r]);
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    acc[r].x += acc2[r].x;
    acc[r].y += acc2[r].y;
  }
  const int n = n0 + warp;
  if (n >= ny) return;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int ix = lane + 32 * r;
    if (ix < ux) split_store2(prec, hi, lo, ((size_t)n * kpad + ix) * 2, acc[r].x, acc[r].y);
  }
}

}  // namespace

size_t sep_focal_u_smem(int ux, int uy) {
  return (size_t)uy * (size_t)((ux + 31) / 32 * 32) * sizeof(float2);
}

cudaError_t sep_focal_u_prepare() {
  cudaError_t e = cudaFuncSetAttribute(sep_focal_u_kernel<4>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SEP_U_SMEM_MAX);
  const cudaError_t e2 = cudaFuncSetAttribute(sep_focal_u_kernel<16>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)SEP_U_SMEM_MAX);
  return e != cudaSuccess ? e : e2;
}

bool sep_focal_u_fits(int ux, int uy, int K) {
  return ux <= 128 && uy <= SEP_U_MAXY && K <= 16 * SEP_U_THREADS &&
         sep_focal_u_smem(ux, uy) <= SEP_U_SMEM_MAX;
}

void launch_sep_focal_u(const float2* theta, const float* t, const float* wprev, float* w,
                        float2* c, double* hist, OfaDevState* st, int weighting, const int2* ixy,
                        int K, const float2* fyu, const int* done, int ny, int ux, int uy,
                        int kpad, int prec, void* hi, void* lo, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((ny + SEP_U_ROWS - 1) / SEP_U_ROWS));
  cfg.blockDim = dim3(SEP_U_THREADS);
  cfg.dynamicSmemBytes = sep_focal_u_smem(ux, uy);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int pitch = (ux + 31) / 32 * 32;
  if (K <= 4 * SEP_U_THREADS)
    cudaLaunchKernelEx(&cfg, sep_focal_u_kernel<4>, theta, t, wprev, w, c, hist, st, weighting,
                       ixy, K, fyu, done, ny, ux, uy, pitch, kpad, prec, hi, lo);
  else
    cudaLaunchKernelEx(&cfg, sep_focal_u_kernel<16>, theta, t, wprev, w, c, hist, st, weighting,
                       ixy, K, fyu, done, ny, ux, uy, pitch, kpad, prec, hi, lo);
}

void launch_build_p(const float2* fyT, const float2* c, const int* done, int nyp, int kp,
                    int prec, void* hi, void* lo, cudaStream_t s) {
  const size_t total = (size_t)nyp * kp / 4;
  size_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, build_p_kernel, fyT, c, done, nyp, kp, prec, hi, lo);
}
