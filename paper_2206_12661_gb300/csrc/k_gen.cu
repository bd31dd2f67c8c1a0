// Kernel (a): DFT-matrix generator and operand packing.
//
// Eq. 2 writes propagation with arbitrarily sampled DFT matrices
// Omega_x = exp(-i 2 pi K_x^T X); restricted to the foci, row k of the x factor
// is Fx[k][m] = exp(-i 2 pi x_k u_m / (lambda f)).  The phase argument
// x_k u_m / (lambda f) (in turns, up to tens of turns for wide arrays) is
// formed and reduced to [-1/2, 1/2] in FP64; only the reduced angle goes to the
// FP32 sincos.
#include "ofa_internal.cuh"
#include "ofa_split.cuh"

namespace {

// Fx[k][m] = exp(-i 2 pi (x_k u_m / (lambda f) + z_k u_m^2 / (2 lambda f^2))): the
// DFT row of Eq. 2 and, for a 3D focus (focus_z non-NULL), the separable Fresnel
// defocus phase of the pupil function that moves the focus z_k off the focal plane.
// Pupil sample m sits at u_m = (m - origin) pitch: origin = (n - 1) / 2 centres a
// whole pupil; a shard of rows passes the axis position of the whole pupil.
__global__ void dft_rows_kernel(const double* __restrict__ focus_xy,
                                const double* __restrict__ focus_z, int coord, int K, int n,
                                double pitch, double origin, double lam_f, double lam_f2,
                                float2* __restrict__ out) {
  size_t total = (size_t)K * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    int k = (int)(i / n);
    int m = (int)(i % n);
    double u = ((double)m - origin) * pitch;
    double turns = focus_xy[2 * (size_t)k + coord] * u / lam_f;
    if (focus_z != nullptr) turns += focus_z[k] * u * u / (2.0 * lam_f2);
    double r = turns - rint(turns);                 // FP64 reduction to [-1/2, 1/2]
    float s, c;
    sincospif((float)(2.0 * r), &s, &c);
    out[i] = make_float2(c, -s);                    // exp(-i 2 pi r)
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

__global__ void scale_kernel(float* x, size_t n, float f) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    x[i] *= f;
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

// Real block form of the complex factor, one output element per thread.
//  forward (inverse == 0): B[2k+h][2m+g], rows give Re/Im of G = E Fx^T:
//     h=0: ( Fr, -Fi )   h=1: ( Fi,  Fr )
//  inverse (inverse == 1): Q[2m+h][2k+g], rows give Re/Im of E' = P conj(Fx):
//     h=0: ( Fr,  Fi )   h=1: (-Fi,  Fr )
__global__ void pack_fx_kernel(const float2* __restrict__ fx, int K, int nx, int kp, int nxp,
                               int inverse, int prec, void* hi, void* lo) {
  size_t rows = inverse ? 2 * (size_t)nxp : 2 * (size_t)kp;
  size_t cols = inverse ? 2 * (size_t)kp : 2 * (size_t)nxp;
  size_t total = rows * cols;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    size_t r = i / cols, cidx = i % cols;
    int h = (int)(r & 1), g = (int)(cidx & 1);
    int k = inverse ? (int)(cidx >> 1) : (int)(r >> 1);
    int m = inverse ? (int)(r >> 1) : (int)(cidx >> 1);
    float v = 0.f;
    if (k < K && m < nx) {
      float2 f = fx[(size_t)k * nx + m];
      if (!inverse) v = h == 0 ? (g == 0 ? f.x : -f.y) : (g == 0 ? f.y : f.x);
      else          v = h == 0 ? (g == 0 ? f.x : f.y) : (g == 0 ? -f.y : f.x);
    }
    split_store(prec, hi, lo, i, v);
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
  dft_rows_kernel<<<grid_for((size_t)K * n), 256, 0, s>>>(focus_xy, focus_z, coord, K, n, pitch,
                                                           origin, lam_f, lam_f2, out);
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

void launch_scale(float* x, size_t n, float f, cudaStream_t s) {
  scale_kernel<<<grid_for(n), 256, 0, s>>>(x, n, f);
}

void launch_transpose_fy(const float2* fy, int K, int ny, int kp, int nyp, float2* fyT,
                         cudaStream_t s, bool conj) {
  dim3 grid((kp + 31) / 32, (nyp + 31) / 32);
  transpose_fy_kernel<<<grid, dim3(32, 8), 0, s>>>(fy, K, ny, kp, nyp, conj ? 1 : 0, fyT);
}

void launch_pack_fx(const float2* fx, int K, int nx, int kp, int nxp, int inverse, int prec,
                    void* hi, void* lo, cudaStream_t s) {
  size_t total = 4 * (size_t)kp * nxp;
  pack_fx_kernel<<<grid_for(total), 256, 0, s>>>(fx, K, nx, kp, nxp, inverse, prec, hi, lo);
}

void launch_field_planes(const float* phi, const float* amp, int nx, int ny, int nxp, int prec,
                         void* hi, void* lo, cudaStream_t s) {
  field_planes_kernel<<<grid_for((size_t)nx * ny), 256, 0, s>>>(phi, amp, nx, ny, nxp, prec, hi,
                                                                  lo);
}
