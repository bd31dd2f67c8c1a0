// One iteration of the focal-plane update of Algorithm 1, as a device routine
// run by NT threads of one block (thread ids 0..NT-1, NT a multiple of 32 up to
// 1024) that synchronise through the barrier functor `bar`:
//   I_k = |Theta_k|^2, S = sum I, Ihat = I / S, xi = 1 - ||t - Ihat|| / ||Ihat||,
//   break if xi > threshold (before the update),
//   w_k <- w_k sqrt(t_k / Ihat_k)           (generalized weighting)
//   c_k  = w_k sqrt(t_k) exp(i arg Theta_k) 2^s   (focused field)
// with 2^s the power of two that brings max |c| into [1/2, 1) (arg() of the
// inverse product does not see a positive scale; the tensor-core operand
// formats want bounded magnitudes).  Reductions are fixed-order shuffle trees,
// so the result is bitwise reproducible for a given block size.
#pragma once
#include "ofa_internal.cuh"


namespace ofa_focal {

struct BarBlock {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Sum of N values over NT threads; every thread receives the same bits.
// sh must hold 33 * N floats.
template <int NT, int N, class Bar>
__device__ __forceinline__ void block_sum(float (&v)[N], float* sh, int tid, Bar bar) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  const int w = tid >> 5, lane = tid & 31;
  bar();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < N; ++i) sh[i * 32 + w] = v[i];
  bar();
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float x = lane < NT / 32 ? sh[i * 32 + lane] : 0.f;
#pragma unroll
      for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) sh[32 * N + i] = x;
    }
  }
  bar();
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = sh[32 * N + i];
}

template <int NT, class Bar>
__device__ __forceinline__ float block_max(float v, float* sh, int tid, Bar bar) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = tid >> 5, lane = tid & 31;
  bar();
  if (lane == 0) sh[w] = v;
  bar();
  if (w == 0) {
    float x = lane < NT / 32 ? sh[lane] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) sh[32] = x;
  }
  bar();
  return sh[32];
}

// Two sums and one max over NT threads in one round; sh must hold 100 floats.
template <int NT, class Bar>
__device__ __forceinline__ void block_sum2_max(float (&v)[2], float& mx, float* sh, int tid,
                                               Bar bar) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    v[1] += __shfl_xor_sync(0xffffffffu, v[1], o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int w = tid >> 5, lane = tid & 31;
  bar();
  if (lane == 0) {
    sh[w] = v[0];
    sh[32 + w] = v[1];
    sh[64 + w] = mx;
  }
  bar();
  if (w == 0) {
    float a = lane < NT / 32 ? sh[lane] : 0.f;
    float b = lane < NT / 32 ? sh[32 + lane] : 0.f;
    float m = lane < NT / 32 ? sh[64 + lane] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
      sh[96] = a;
      sh[97] = b;
      sh[98] = m;
    }
  }
  bar();
  v[0] = sh[96];
  v[1] = sh[97];
  mx = sh[98];
}

// theta: the final Theta_k (K values, written by other threads or blocks of this
// launch: read through L2); sh: >= 4 * 33 floats of shared memory.
// meas (nullable): captured intensities that replace the calculated |Theta_k|^2 in
// xi and the weight update (camera in the loop); the focused field keeps the
// phase of the calculated Theta.
template <int NT, class Bar>
__device__ inline void iterate(const float2* theta, int K, int kp, const float* __restrict__ t,
                               float* __restrict__ w, float2* __restrict__ c,
                               double* __restrict__ hist, OfaDevState* __restrict__ st,
                               int weighting, float* sh, int tid, Bar bar,
                               const float* __restrict__ meas = nullptr) {
  constexpr int nt = NT;
  const double thr = st->threshold;
  float r1[1] = {0.f};
  for (int k = tid; k < K; k += nt) {
    const float2 a = __ldcg(theta + k);
    r1[0] += meas ? meas[k] : a.x * a.x + a.y * a.y;
  }
  block_sum<NT>(r1, sh, tid, bar);
  const float S = r1[0];
  if (!(S > 0.f) || !isfinite(S)) {
    if (tid == 0) {
      atomicOr(&st->err, OFA_ERRBIT_NUMERIC);
      st->done = 1;
    }
    return;
  }
  const float inv_s = 1.f / S;
  float r2[2] = {0.f, 0.f};
  float mx = 0.f;
  for (int k = tid; k < K; k += nt) {
    const float2 a = __ldcg(theta + k);
    const float ih = (meas ? meas[k] : a.x * a.x + a.y * a.y) * inv_s;
    const float tk = t[k];
    const float d = tk - ih;
    r2[0] += d * d;
    r2[1] += ih * ih;
    float wk = w[k];
    const float stk = sqrtf(tk);
    if (weighting) wk *= stk * rsqrtf(fmaxf(ih, 1e-30f));  // w sqrt(t / Ihat)
    mx = fmaxf(mx, wk * stk);
  }
  block_sum<NT>(r2, sh + 33, tid, bar);
  mx = block_max<NT>(mx, sh + 99, tid, bar);
  const double xi = 1.0 - sqrt((double)r2[0] / (double)r2[1]);
  if (tid == 0) {
    const int h = st->hist_count;
    hist[h % OFA_HIST_CAP] = xi;
    st->hist_count = h + 1;
    st->xi = xi;
  }
  if (thr > 0.0 && thr < 1.0 && xi > thr) {
    if (tid == 0) st->done = 1;
    return;
  }
  int e = 0;
  frexpf(mx, &e);
  const float scale = mx > 0.f ? exp2f((float)-e) : 1.f;
  for (int k = tid; k < kp; k += nt) {
    float2 ck = make_float2(0.f, 0.f);
    if (k < K) {
      const float2 a = __ldcg(theta + k);
      const float rr = a.x * a.x + a.y * a.y;
      const float tk = t[k];
      float wk = w[k];
      if (weighting) {
        const float iu = meas ? meas[k] : rr;
        wk *= sqrtf(tk) * rsqrtf(fmaxf(iu * inv_s, 1e-30f));  // w_j = w_{j-1} sqrt(t / Ihat)
        w[k] = wk;
      }
      const float mag = wk * sqrtf(tk) * scale;
      if (rr > 0.f) {
        const float inv = rsqrtf(rr);
        ck = make_float2(mag * a.x * inv, mag * a.y * inv);
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

// The same update from the per-tile partials, with each thread's foci held in
// registers (KPR foci per thread, K <= NT * KPR): the partials, targets and
// weights are loaded with all independent loads in flight; the rest runs from
// registers in two reduction rounds.  part is [n_part][kp] complex, written
// earlier in this launch (read through L2).  sh: >= 133 floats.
template <int NT, int KPR, class Bar>
__device__ inline void iterate_regs(const float2* part, int n_part, int K, int kp,
                                    const float* __restrict__ t, float* __restrict__ w,
                                    float2* __restrict__ c, double* __restrict__ hist,
                                    OfaDevState* __restrict__ st, int weighting, float* sh,
                                    int tid, Bar bar) {
  const double thr = st->threshold;
  const int hcount = st->hist_count;
  const int j0 = st->j;
  float2 th[KPR];
  float tk[KPR], wk[KPR], ik[KPR];
  bool in[KPR];
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    const int k = tid + i * NT;
    in[i] = k < K;
    th[i] = make_float2(0.f, 0.f);
    tk[i] = in[i] ? t[k] : 0.f;
    wk[i] = in[i] ? w[k] : 0.f;
  }
  // partials in fixed order p = 0, 1, ...; the loads of RB rows (RB x KPR values)
  // are issued together, then summed, so a round costs one L2 latency
  constexpr int RB = KPR <= 4 ? 8 : 2;
  for (int p0 = 0; p0 < n_part; p0 += RB) {
    float2 v[RB][KPR];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int i = 0; i < KPR; ++i)
        v[r][i] = (in[i] && p0 + r < n_part)
                      ? __ldcg(part + (size_t)(p0 + r) * kp + tid + i * NT)
                      : make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int i = 0; i < KPR; ++i) {
        th[i].x += v[r][i].x;
        th[i].y += v[r][i].y;
      }
  }
  float r1[1] = {0.f};
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    ik[i] = th[i].x * th[i].x + th[i].y * th[i].y;
    r1[0] += ik[i];
  }
  block_sum<NT>(r1, sh, tid, bar);
  const float S = r1[0];
  if (!(S > 0.f) || !isfinite(S)) {
    if (tid == 0) {
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
  block_sum2_max<NT>(r2, mx, sh + 33, tid, bar);
  const float xi = 1.f - sqrtf(r2[0] / r2[1]);
  if (tid == 0) {
    hist[hcount % OFA_HIST_CAP] = (double)xi;
    st->hist_count = hcount + 1;
    st->xi = (double)xi;
  }
  if (thr > 0.0 && thr < 1.0 && (double)xi > thr) {
    if (tid == 0) st->done = 1;
    return;
  }
  int e = 0;
  frexpf(mx, &e);
  const float scale = mx > 0.f ? exp2f((float)-e) : 1.f;
#pragma unroll
  for (int i = 0; i < KPR; ++i) {
    const int k = tid + i * NT;
    if (k >= K) continue;
    if (weighting) w[k] = wk[i];
    const float mag = wk[i] * sq[i] * scale;
    float2 ck;
    if (ik[i] > 0.f) {
      const float inv = rsqrtf(ik[i]);
      ck = make_float2(mag * th[i].x * inv, mag * th[i].y * inv);
    } else {
      ck = make_float2(mag, 0.f);  // arg(0) = 0
    }
    c[k] = ck;
  }
  if (tid == 0) {
    st->j = j0 + 1;
    st->c_scale = scale;
  }
}

}  // namespace ofa_focal
