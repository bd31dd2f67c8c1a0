// ofa_forward_noalloc: focal field at the foci without any device allocation.
//
// Some callers cannot allocate device memory at the time they need a forward
// propagation: a real-time loop that refreshes an SLM hologram and must not see
// the latency spikes or failures of cudaMalloc once it runs, or an application
// whose device memory is entirely reserved up front by a framework allocator.
// This entry point needs no plan: it takes the pupil field (phi, A) and the focus
// positions, generates the DFT rows on the fly (phase arguments reduced in FP64)
// and keeps its only scratch, one partial focal field per 64-row tile, in a
// file-scope static device array that every GPU loading the library holds until
// the process exits.  Callers still pass their inputs and outputs.
//
// The array is shared by every call: each call overwrites all entries it later
// reads, but calls that overlap on the GPU (different streams, or host threads
// racing) race on it and must be serialised by the caller.
#include <cudaTypedefs.h>

#include <mutex>

#include "ofa_internal.cuh"

#define OFA_NOALLOC_MAX_ROW_TILES 32    // ny <= 32 * 64 = 2048
#define OFA_NOALLOC_MAX_FOCI 8192
#define OFA_NOALLOC_MAX_NX 32768

// 32 x 8192 complex floats = 2 MiB of scratch.
static __device__ __align__(256) float2 g_noalloc_part[OFA_NOALLOC_MAX_ROW_TILES *
                                                       OFA_NOALLOC_MAX_FOCI];

namespace {

constexpr int T64 = 64;
constexpr int TS = 16;

// Device address of g_noalloc_part, looked up once per device (the symbol name
// is a host-side stand-in, not a device address), together with the context it
// was looked up in: after a device reset the runtime loads the module into a new
// context, where the array may sit elsewhere, so a changed context looks it up
// again.
std::mutex g_noalloc_mu;
float2* g_noalloc_addr[64] = {};
CUcontext g_noalloc_ctx[64] = {};

CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
  });
  CUcontext c = nullptr;
  if (fn == nullptr || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// exp(-i 2 pi (a m + b)) with the turns a m + b formed and reduced in FP64.
__device__ __forceinline__ float2 dft_factor(double a, double b, int m) {
  const double turns = fma(a, (double)m, b);
  const double r = turns - rint(turns);
  float s, c;
  sincospif((float)(2.0 * r), &s, &c);
  return make_float2(c, -s);
}

// Same tiling as the FP32 forward (64 rows x 64 foci, 256 threads, 4 x 4 complex
// accumulators), with Fx and Fy generated in shared memory instead of read.
__global__ void __launch_bounds__(256) fwd_noalloc_kernel(
    const float* __restrict__ phi, const float* __restrict__ amp,
    const double* __restrict__ focus_xy, int nx, int ny, int K, double px, double py,
    double lam_f, float2* __restrict__ part) {
  __shared__ __align__(16) float2 Es[TS][T64];
  __shared__ __align__(16) float2 Fs[TS][T64];
  __shared__ double ax[T64], bx[T64], ay[T64], by[T64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int n0 = blockIdx.y * T64, k0 = blockIdx.x * T64;
  const int lr = tid >> 2, lc = (tid & 3) * 4;
  if (tid < T64) {
    const int k = k0 + tid;
    const double x = k < K ? focus_xy[2 * (size_t)k] : 0.0;
    const double y = k < K ? focus_xy[2 * (size_t)k + 1] : 0.0;
    // x u_m / (lambda f) with u_m = (m - (nx-1)/2) px: a m + b
    ax[tid] = x * px / lam_f;
    bx[tid] = -x * px * 0.5 * (double)(nx - 1) / lam_f;
    ay[tid] = y * py / lam_f;
    by[tid] = -y * py * 0.5 * (double)(ny - 1) / lam_f;
  }
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int m0 = 0; m0 < nx; m0 += TS) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = m0 + lc + q, n = n0 + lr, k = k0 + lr;
      float2 e = make_float2(0.f, 0.f);
      if (n < ny && m < nx) {
        float s, c;
        sincosf(phi[(size_t)n * nx + m], &s, &c);
        const float a = amp[(size_t)n * nx + m];
        e = make_float2(a * c, a * s);   // E = A exp(i phi)
      }
      Es[lc + q][lr] = e;
      Fs[lc + q][lr] = (k < K && m < nx) ? dft_factor(ax[lr], bx[lr], m) : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int mm = 0; mm < TS; ++mm) {
      float2 e[4], f[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        e[i] = Es[mm][ty * 4 + i];
        f[i] = Fs[mm][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cmac(acc[i][j], e[i], f[j]);
    }
  }
  // Theta partial of this row tile: sum_n Fy[k,n] G[n,k], fixed order.
  __syncthreads();
  float2* red = &Es[0][0];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int kl = tx * 4 + j, k = k0 + kl;
    float2 s = make_float2(0.f, 0.f);
    if (k < K) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int n = n0 + ty * 4 + i;
        if (n < ny) cmac(s, dft_factor(ay[kl], by[kl], n), acc[i][j]);
      }
    }
    red[ty * T64 + kl] = s;
  }
  __syncthreads();
  if (tid < T64 && k0 + tid < K) {
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      a.x += red[t * T64 + tid].x;
      a.y += red[t * T64 + tid].y;
    }
    part[(size_t)blockIdx.y * OFA_NOALLOC_MAX_FOCI + k0 + tid] = a;
  }
}

__global__ void reduce_noalloc_kernel(const float2* __restrict__ part, int n_part, int K,
                                      float2* __restrict__ theta, float* __restrict__ inten) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    float2 a = make_float2(0.f, 0.f);
    for (int p = 0; p < n_part; ++p) {
      const float2 v = part[(size_t)p * OFA_NOALLOC_MAX_FOCI + k];
      a.x += v.x;
      a.y += v.y;
    }
    if (theta) theta[k] = a;
    if (inten) inten[k] = a.x * a.x + a.y * a.y;
  }
}

bool finite_pos(double v) { return v > 0.0 && v < 1e300; }

}  // namespace

extern "C" ofa_status ofa_forward_noalloc(int nx, int ny, double pitch_x, double pitch_y,
                                          double wavelength, double focal_length, int n_foci,
                                          const double* focus_xy, const float* phi,
                                          const float* amplitude, float* theta, float* intensity,
                                          void* cuda_stream) {
  if (nx < 1 || ny < 1 || n_foci < 1 || !focus_xy || !phi || !amplitude ||
      (!theta && !intensity)) {
    ofa_set_thread_error("ofa_forward_noalloc: sizes must be >= 1, inputs non-NULL and at "
                         "least one output given");
    return OFA_ERR_INVALID_ARG;
  }
  if (!finite_pos(pitch_x) || !finite_pos(pitch_y) || !finite_pos(wavelength) ||
      !finite_pos(focal_length)) {
    ofa_set_thread_error("ofa_forward_noalloc: pitch, wavelength and focal length must be > 0");
    return OFA_ERR_INVALID_ARG;
  }
  const int row_tiles = (ny + T64 - 1) / T64;
  if (row_tiles > OFA_NOALLOC_MAX_ROW_TILES || n_foci > OFA_NOALLOC_MAX_FOCI ||
      nx > OFA_NOALLOC_MAX_NX) {
    ofa_set_thread_error("ofa_forward_noalloc: sizes beyond the static scratch (ny <= 2048, "
                         "n_foci <= 8192, nx <= 32768)");
    return OFA_ERR_INVALID_ARG;
  }
  // An error left pending by earlier, unrelated work is reported as such (and
  // cleared), not mistaken for a failure of this call's launches.
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ofa_set_thread_error(std::string("ofa_forward_noalloc: a CUDA error from earlier work was "
                                     "pending on entry (nothing was launched): ") +
                         cudaGetErrorString(e));
    return OFA_ERR_CUDA;
  }
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    ofa_set_thread_error("ofa_forward_noalloc: no usable current CUDA device");
    return OFA_ERR_CUDA;
  }
  float2* part = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    const CUcontext ctx = current_context();
    if (!g_noalloc_addr[dev] || ctx != g_noalloc_ctx[dev]) {
      // first call on this device (or in a new context): resolve the scratch
      // array's device address with this device current
      void* a = nullptr;
      e = cudaGetSymbolAddress(&a, g_noalloc_part);
      if (e != cudaSuccess || a == nullptr) {
        ofa_set_thread_error("ofa_forward_noalloc: cudaGetSymbolAddress of the static scratch "
                             "failed");
        return OFA_ERR_CUDA;
      }
      g_noalloc_addr[dev] = static_cast<float2*>(a);
      g_noalloc_ctx[dev] = current_context();
    }
    part = g_noalloc_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const double lam_f = wavelength * focal_length;
  dim3 grid((n_foci + T64 - 1) / T64, row_tiles);
  fwd_noalloc_kernel<<<grid, 256, 0, s>>>(phi, amplitude, focus_xy, nx, ny, n_foci, pitch_x,
                                          pitch_y, lam_f, part);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    reduce_noalloc_kernel<<<(n_foci + 255) / 256, 256, 0, s>>>(
        part, row_tiles, n_foci, reinterpret_cast<float2*>(theta), intensity);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    ofa_set_thread_error(std::string("ofa_forward_noalloc: kernel launch failed: ") +
                         cudaGetErrorString(e));
    return OFA_ERR_CUDA;
  }
  return OFA_OK;
}
