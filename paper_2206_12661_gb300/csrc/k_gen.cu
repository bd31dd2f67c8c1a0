// Kernel (a): DFT-matrix generator and operand packing.
//
// Eq. 2 writes propagation with arbitrarily sampled DFT matrices
// Omega_x = exp(-i 2 pi K_x^T X); restricted to the foci, row k of the x factor
// is Fx[k][m] = exp(-i 2 pi x_k u_m / (lambda f)).  The phase argument
// x_k u_m / (lambda f) (in turns, up to thousands of turns for wide arrays) is
// reduced modulo one turn exactly, in 64-bit fixed point, and only the reduced
// angle goes to the FP32 sincos.
#include "ofa_internal.cuh"
#include "ofa_split.cuh"

namespace {

// Fx[k][m] = exp(-i 2 pi (x_k u_m / (lambda f) + z_k u_m^2 / (2 lambda f^2))): the
// DFT row of Eq. 2 and, for a 3D focus (focus_z non-NULL), the separable Fresnel
// defocus phase of the pupil function that moves the focus z_k off the focal plane.
// Pupil sample m sits at u_m = (m - origin) pitch with 2 origin = o2 an integer
// (o2 = n - 1 centres a whole pupil; a shard of rows passes the axis position of the
// whole pupil), so with j = 2m - o2 the phase is j b_k + j^2 d_k turns,
// b_k = x_k pitch / (2 lambda f) and d_k = z_k pitch^2 / (8 lambda f^2).  Each row's
// b_k and d_k are formed once in FP64, reduced to [-1/2, 1/2] and held as multiples
// of 2^-64 turn; the products with j and j^2 then wrap modulo 2^64, which is the
// reduction modulo one turn, exact for every m.  The only rounding is that of b_k
// and d_k (about 2^-53 of each), the same as forming the turns in FP64.
constexpr int DFT_THREADS = 256, DFT_ROWS = 16;

__device__ __forceinline__ unsigned long long turns_fixed(double t) {
  const double f = t - rint(t);  // [-1/2, 1/2], exact
  // f 2^62 fits an int64 with room for f = 1/2; the shift by two wraps to 2^-64 units
  return (unsigned long long)__double2ll_rn(f * 0x1p62) << 2;
}

__global__ void __launch_bounds__(DFT_THREADS)
    dft_rows_kernel(const double* __restrict__ focus_xy, const double* __restrict__ focus_z,
                    int coord, int K, int n, int o2, double cb, double cd,
                    float2* __restrict__ out) {
  __shared__ unsigned long long sb[DFT_ROWS], sd[DFT_ROWS];
  const int k0 = blockIdx.x * DFT_ROWS;
  const int rows = min(DFT_ROWS, K - k0);
  if (threadIdx.x < rows) {
    const int k = k0 + threadIdx.x;
    sb[threadIdx.x] = turns_fixed(focus_xy[2 * (size_t)k + coord] * cb);
    sd[threadIdx.x] = focus_z != nullptr ? turns_fixed(focus_z[k] * cd) : 0ull;
  }
  __syncthreads();
  const int m = blockIdx.y * DFT_THREADS + threadIdx.x;
  if (m >= n) return;
  const long long j = 2 * (long long)m - o2;
  const unsigned long long uj = (unsigned long long)j, uj2 = (unsigned long long)(j * j);
  for (int r = 0; r < rows; ++r) {
    const long long ph = (long long)(uj * sb[r] + uj2 * sd[r]);  // 2^-64 turns, [-1/2, 1/2)
    float s, c;
    sincospif(__ll2float_rn(ph) * 0x1p-63f, &s, &c);           // angle pi (2 ph 2^-64)
    out[(size_t)(k0 + r) * n + m] = make_float2(c, -s);         // exp(-i 2 pi ph 2^-64)
  }
}

__global__ void default_amplitude_kernel(float* __restrict__ amp, int nx, int ny, int row0,
                                         int ny_total, double px, double py, double wf) {
  size_t total = (size_t)nx * ny;
  double wx = wf * nx * px, wy = wf * ny_total * py;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    int n = (int)(i / nx), m = (int)(i % nx);
    double u = ((double)m - 0.5 * (nx - 1)) * px;
    double v = ((double)(n + row0) - 0.5 * (ny_total - 1)) * py;
    amp[i] = (float)exp(-(u * u / (wx * wx) + v * v / (wy * wy)));
  }
}

// splitmix64 (Steele, Lea and Flood 2014): output i of the stream seeded with
// `seed` mixes seed + (i + 1) * gamma.
__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void default_phase_kernel(float* __restrict__ phi, size_t total, size_t index0,
                                     uint64_t seed) {
  const uint64_t gamma = 0x9E3779B97F4A7C15ull;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    uint64_t v = splitmix64_mix(seed + (uint64_t)(i + index0 + 1) * gamma);
    double u01 = (double)(v >> 11) * (1.0 / 9007199254740992.0);
    phi[i] = (float)(u01 * 6.283185307179586 - 3.141592653589793);
  }
}

// Peak, energy (sum of squares, FP64) and validity of the pupil amplitude.  Each of
// the AMP_STAT_BLOCKS blocks reduces a fixed strided share of the pixels (four at a
// time, one 16-byte load per thread and step) by a fixed shuffle tree; the last block
// to finish reduces the block results by the same fixed tree, so the result is the
// same on every run.  The peak then fixes the exponent ex with peak 2^-ex in
// (1/2, 1] (an exact power of two maps to 1), which the scale below applies.
constexpr int AMP_STAT_THREADS = 256;

struct AmpStat {
  double e;   // sum of squares
  float m;    // peak
  int bad;    // a value was negative, infinite or NaN
};

__device__ __forceinline__ void amp_stat_add(AmpStat& s, float v) {
  s.bad |= !(v >= 0.f) || isinf(v);
  s.m = fmaxf(s.m, v);
  s.e += (double)v * v;  // exact square: 48 significant bits
}

__device__ __forceinline__ void amp_stat_merge(AmpStat& s, const AmpStat& o) {
  s.e += o.e;
  s.m = fmaxf(s.m, o.m);
  s.bad |= o.bad;
}

// Block-wide fixed-order reduction; thread 0 holds the result.
__device__ __forceinline__ AmpStat amp_stat_block(AmpStat s, AmpStat* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    AmpStat t;
    t.e = __shfl_xor_sync(0xffffffffu, s.e, o);
    t.m = __shfl_xor_sync(0xffffffffu, s.m, o);
    t.bad = __shfl_xor_sync(0xffffffffu, s.bad, o);
    amp_stat_merge(s, t);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < AMP_STAT_THREADS / 32; ++w) amp_stat_merge(s, sh[w]);
  return s;
}

__global__ void __launch_bounds__(AMP_STAT_THREADS)
    amp_stats_kernel(const float* __restrict__ a, size_t n, double* __restrict__ part,
                     unsigned* __restrict__ count, OfaDevState* __restrict__ st) {
  __shared__ AmpStat sh[AMP_STAT_THREADS / 32];
  __shared__ bool last;
  AmpStat s = {0.0, 0.f, 0};
  const size_t n4 = n / 4;  // the amplitude buffer starts on a 256-byte boundary
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 v = a4[i];
    amp_stat_add(s, v.x);
    amp_stat_add(s, v.y);
    amp_stat_add(s, v.z);
    amp_stat_add(s, v.w);
  }
  const size_t tail = 4 * n4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (tail < n) amp_stat_add(s, a[tail]);
  s = amp_stat_block(s, sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = s.e;
    part[3 * blockIdx.x + 1] = s.m;
    part[3 * blockIdx.x + 2] = s.bad;
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block: thread t merges blocks t, t + 256, ... in order, then the tree
  AmpStat r = {0.0, 0.f, 0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += AMP_STAT_THREADS) {
    const AmpStat o = {__ldcg(part + 3 * b), (float)__ldcg(part + 3 * b + 1),
                       __ldcg(part + 3 * b + 2) != 0.0 ? 1 : 0};
    amp_stat_merge(r, o);
  }
  __syncthreads();  // sh is reused
  r = amp_stat_block(r, sh);
  if (threadIdx.x != 0) return;
  const double mt = r.m;
  int ex = 0;
  if (!r.bad && mt > 0.0) {
    frexp(mt, &ex);                              // mt = f 2^ex, f in [1/2, 1)
    if (mt == ldexp(1.0, ex - 1)) ex -= 1;       // an exact power of two maps to 1
  }
  st->amp_max = mt;
  st->amp_energy = r.e;
  st->amp_bad = r.bad;
  st->amp_exp = ex;
  *count = 0;
}

// x *= 2^-ex with ex from amp_stats_kernel.  The product is formed in FP64 (exact)
// and rounded once to FP32, so a peak that is subnormal or near the FP32 maximum
// scales as exactly as any other.
__global__ void scale_pow2_kernel(float* __restrict__ x, size_t n,
                                  const OfaDevState* __restrict__ st) {
  const int ex = st->amp_exp;
  if (ex == 0) return;
  const double f = ldexp(1.0, -ex);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    x[i] = (float)((double)x[i] * f);
}

// fyT[n][k] = fy[k][n] (conjugated when conj; zero outside K x ny), [nyp][kp]
__global__ void transpose_fy_kernel(const float2* __restrict__ fy, int K, int ny, int kp,
                                    int nyp, int conj, float2* __restrict__ fyT) {
  __shared__ float2 tile[32][33];
  int k0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int k = k0 + r, n = n0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && n < ny) ? fy[(size_t)k * ny + n] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int n = n0 + r, k = k0 + threadIdx.x;
    const float2 v = tile[threadIdx.x][r];
    if (n < nyp && k < kp) fyT[(size_t)n * kp + k] = make_float2(v.x, conj ? -v.y : v.y);
  }
}

// Real block form of the complex factor.  Thread (a, b) reads one complex entry and
// writes the 2 x 2 real block it becomes, as two pairs of adjacent elements:
//  forward (inverse == 0): B[2k+h][2m+g], rows give Re/Im of G = E Fx^T:
//     h=0: ( Fr, -Fi )   h=1: ( Fi,  Fr )
//  inverse (inverse == 1): Q[2m+h][2k+g], rows give Re/Im of E' = P conj(Fx):
//     h=0: ( Fr,  Fi )   h=1: (-Fi,  Fr )
// a runs along the rows of the block form (m for the forward, k for the inverse), b over
// its row pairs; entries beyond K foci or nx samples give zeros.
__global__ void pack_fx_kernel(const float2* __restrict__ fx, int K, int nx, int kp, int nxp,
                               int inverse, int prec, void* hi, void* lo) {
  const int A = inverse ? kp : nxp;   // complex columns of a row pair
  const int B = inverse ? nxp : kp;   // row pairs
  const size_t cols = 2 * (size_t)A;
  for (int b = blockIdx.y; b < B; b += gridDim.y)
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < A; a += gridDim.x * blockDim.x) {
      const int k = inverse ? a : b, m = inverse ? b : a;
      const float2 f = k < K && m < nx ? fx[(size_t)k * nx + m] : make_float2(0.f, 0.f);
      const size_t e = 2 * (size_t)b * cols + 2 * (size_t)a;   // element (2b, 2a)
      if (!inverse) {
        split_store2(prec, hi, lo, e, f.x, -f.y);
        split_store2(prec, hi, lo, e + cols, f.y, f.x);
      } else {
        split_store2(prec, hi, lo, e, f.x, f.y);
        split_store2(prec, hi, lo, e + cols, -f.y, f.x);
      }
    }
}

// E = A exp(i phi) as interleaved operand planes [nyp][2 nxp] (padding untouched).
__global__ void field_planes_kernel(const float* __restrict__ phi, const float* __restrict__ amp,
                                    int nx, int ny, int nxp, int prec, void* hi, void* lo) {
  size_t total = (size_t)nx * ny;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    int n = (int)(i / nx), m = (int)(i % nx);
    float s, c;
    __sincosf(phi[i], &s, &c);  // same intrinsic as the inverse epilogue: resume is bitwise
    float a = amp[i];
    split_store2(prec, hi, lo, ((size_t)n * nxp + m) * 2, a * c, a * s);
  }
}

inline int grid_for(size_t n, int threads = 256) {
  size_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

void launch_dft_rows(const double* focus_xy, const double* focus_z, int coord, int K, int n,
                     double pitch, double origin, double lam_f, double lam_f2, float2* out,
                     cudaStream_t s) {
  if (K < 1 || n < 1) return;
  const int o2 = (int)llrint(2.0 * origin);
  const double cb = pitch / (2.0 * lam_f), cd = pitch * pitch / (8.0 * lam_f2);
  const dim3 grid((unsigned)((K + DFT_ROWS - 1) / DFT_ROWS),
                  (unsigned)((n + DFT_THREADS - 1) / DFT_THREADS));
  dft_rows_kernel<<<grid, DFT_THREADS, 0, s>>>(focus_xy, focus_z, coord, K, n, o2, cb, cd, out);
}

void launch_default_amplitude(float* amp, int nx, int ny, int row0, int ny_total, double px,
                              double py, double wf, cudaStream_t s) {
  default_amplitude_kernel<<<grid_for((size_t)nx * ny), 256, 0, s>>>(amp, nx, ny, row0, ny_total,
                                                                      px, py, wf);
}

void launch_default_phase(float* phi, int nx, int ny, int row0, uint64_t seed, cudaStream_t s) {
  default_phase_kernel<<<grid_for((size_t)nx * ny), 256, 0, s>>>(phi, (size_t)nx * ny,
                                                                  (size_t)row0 * nx, seed);
}

void launch_amp_stats(const float* amp, size_t n, double* part, unsigned* count,
                      OfaDevState* st, cudaStream_t s) {
  amp_stats_kernel<<<AMP_STAT_BLOCKS, AMP_STAT_THREADS, 0, s>>>(amp, n, part, count, st);
}

void launch_scale_pow2(float* x, size_t n, const OfaDevState* st, cudaStream_t s) {
  scale_pow2_kernel<<<grid_for(n), 256, 0, s>>>(x, n, st);
}

void launch_transpose_fy(const float2* fy, int K, int ny, int kp, int nyp, float2* fyT,
                         cudaStream_t s, bool conj) {
  dim3 grid((kp + 31) / 32, (nyp + 31) / 32);
  transpose_fy_kernel<<<grid, dim3(32, 8), 0, s>>>(fy, K, ny, kp, nyp, conj ? 1 : 0, fyT);
}

void launch_pack_fx(const float2* fx, int K, int nx, int kp, int nxp, int inverse, int prec,
                    void* hi, void* lo, cudaStream_t s) {
  const int A = inverse ? kp : nxp, B = inverse ? nxp : kp;
  const dim3 grid((unsigned)((A + 255) / 256), (unsigned)(B < 65535 ? B : 65535));
  pack_fx_kernel<<<grid, 256, 0, s>>>(fx, K, nx, kp, nxp, inverse, prec, hi, lo);
}

void launch_field_planes(const float* phi, const float* amp, int nx, int ny, int nxp, int prec,
                         void* hi, void* lo, cudaStream_t s) {
  field_planes_kernel<<<grid_for((size_t)nx * ny), 256, 0, s>>>(phi, amp, nx, ny, nxp, prec, hi,
                                                                  lo);
}
