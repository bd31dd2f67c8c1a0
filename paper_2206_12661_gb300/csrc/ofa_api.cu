// Host side of the C ABI declared in include/ofa.h.
//
// A plan owns its device buffers, a private capture stream and two CUDA graphs
// (a chunk of iterations and a single iteration) built on first use; every
// launch of the loop replays a graph on the plan's stream.  One iteration is
//   FP32 form:        forward (fused phi->field)  ->  focal  ->  inverse (+arg)
//   tensor-core form: forward (TMA/tcgen05, dot epilogue) -> focal -> P build
//                     -> inverse (TMA/tcgen05, arg + next field epilogue)
// The threshold test of Algorithm 1 runs on the device (focal kernel sets a
// flag that makes the rest of a launch skip); the host checks it between
// chunks only when a threshold is set.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ofa_host.h"
#include "ofa_internal.cuh"

namespace {

thread_local std::string g_thread_error;

const char* kStatusNames[] = {"OFA_OK",          "OFA_ERR_INVALID_ARG", "OFA_ERR_OUT_OF_RANGE",
                              "OFA_ERR_CUDA",    "OFA_ERR_OOM",         "OFA_ERR_NUMERIC",
                              "OFA_ERR_TIMEOUT", "OFA_ERR_UNSUPPORTED"};

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Host-side fault injection for the error paths of plan creation: with
// OFA_FAULT_ALLOC=N in the environment, the N-th device allocation of an
// ofa_plan_create call fails as if the device were out of memory.
thread_local int g_fault_alloc_countdown = 0;

// While a plan is being created its buffers are only reserved (slot, bytes) and
// then carved out of one zero-filled device allocation (arena_commit): one
// cudaMalloc and one memset instead of one pair per buffer.
struct ArenaReq {
  void** slot;
  size_t bytes;
};
thread_local std::vector<ArenaReq>* g_arena = nullptr;

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (g_fault_alloc_countdown > 0 && --g_fault_alloc_countdown == 0)
    return cudaErrorMemoryAllocation;
  if (g_arena) {
    g_arena->push_back({reinterpret_cast<void**>(p), count * sizeof(T)});
    return cudaSuccess;
  }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e == cudaSuccess) e = cudaMemset(*p, 0, count * sizeof(T));
  return e;
}

// Per-device reuse of what plan creation and destruction cost most on the host:
// the device attributes, the kernels' shared-memory opt-in (once per precision),
// one plan arena, one pinned state mirror, a few idle streams and the iteration
// graphs' executables of destroyed plans.  A process that creates and destroys plans
// in a loop then calls cudaMalloc / cudaMallocHost / cudaStreamCreate once and
// refreshes a graph executable instead of instantiating one; ofa_trim releases what
// is cached.
constexpr int OFA_CACHED_STREAMS = 8;
constexpr int OFA_CACHED_EXECS = 8;
// What fixes an iteration graph's nodes, kernels and launch attributes: only an
// executable of the same key is refreshed for another plan (whose graph then differs
// in kernel arguments alone).
using ExecKey = std::array<int, 24>;
struct CachedExec {
  cudaGraphExec_t exec;
  ExecKey key;
};
struct DeviceCache {
  bool attrs = false;
  int cc = 0, sms = 0;
  unsigned prepared = 0;   // bit per precision: kernel attributes set
  void* arena = nullptr;
  size_t arena_bytes = 0;
  OfaDevState* st_host = nullptr;
  cudaStream_t streams[OFA_CACHED_STREAMS] = {};
  int n_streams = 0;
  CachedExec execs[OFA_CACHED_EXECS] = {};
  int n_execs = 0;
};
constexpr int OFA_MAX_DEVICES = 64;
std::mutex g_cache_mu;
DeviceCache g_cache[OFA_MAX_DEVICES];

cudaError_t device_attrs(int dev, int* cc, int* sms) {
  if (dev >= 0 && dev < OFA_MAX_DEVICES) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (g_cache[dev].attrs) {
      *cc = g_cache[dev].cc;
      *sms = g_cache[dev].sms;
      return cudaSuccess;
    }
  }
  int major = 0, minor = 0;
  cudaError_t e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  *cc = major * 10 + minor;
  if (dev >= 0 && dev < OFA_MAX_DEVICES) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache[dev].attrs = true;
    g_cache[dev].cc = *cc;
    g_cache[dev].sms = *sms;
  }
  return cudaSuccess;
}

cudaError_t prepare_precision(int dev, int prec) {
  const bool cacheable = dev >= 0 && dev < OFA_MAX_DEVICES && prec >= 0 && prec < 32;
  if (cacheable) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (g_cache[dev].prepared & (1u << prec)) return cudaSuccess;
  }
  cudaError_t e = tc_prepare(prec);
  if (e == cudaSuccess && cacheable) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache[dev].prepared |= 1u << prec;
  }
  return e;
}

// A cached arena of at least `bytes` (and not more than four times that), or null.
void* take_cached_arena(int dev, size_t bytes, size_t* got) {
  if (dev < 0 || dev >= OFA_MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  DeviceCache& c = g_cache[dev];
  if (!c.arena || c.arena_bytes < bytes || c.arena_bytes / 4 > bytes) return nullptr;
  void* a = c.arena;
  *got = c.arena_bytes;
  c.arena = nullptr;
  c.arena_bytes = 0;
  return a;
}

// Keep a destroyed plan's arena for the next plan (the larger of it and the one
// already kept); free the other.  The plan's stream has been synchronised.
void give_back_arena(int dev, void* arena, size_t bytes) {
  void* drop = arena;
  if (dev >= 0 && dev < OFA_MAX_DEVICES) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    DeviceCache& c = g_cache[dev];
    if (!c.arena || c.arena_bytes < bytes) {
      drop = c.arena;
      c.arena = arena;
      c.arena_bytes = bytes;
    }
  }
  if (drop) cudaFree(drop);
}

// An idle non-blocking stream of the device: a cached one, else a new one.
cudaError_t take_stream(int dev, cudaStream_t* s) {
  if (dev >= 0 && dev < OFA_MAX_DEVICES) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    DeviceCache& c = g_cache[dev];
    if (c.n_streams > 0) {
      *s = c.streams[--c.n_streams];
      return cudaSuccess;
    }
  }
  return cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
}

// Keep a stream with no work pending for the next plan, or destroy it.
void give_back_stream(int dev, cudaStream_t s) {
  if (!s) return;
  if (dev >= 0 && dev < OFA_MAX_DEVICES) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    DeviceCache& c = g_cache[dev];
    if (c.n_streams < OFA_CACHED_STREAMS) {
      c.streams[c.n_streams++] = s;
      return;
    }
  }
  cudaStreamDestroy(s);
}

// A cached graph executable of this key (the most recently kept), or null.
cudaGraphExec_t take_cached_exec(int dev, const ExecKey& key) {
  if (dev < 0 || dev >= OFA_MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  DeviceCache& c = g_cache[dev];
  for (int i = c.n_execs - 1; i >= 0; --i)
    if (c.execs[i].key == key) {
      const cudaGraphExec_t x = c.execs[i].exec;
      for (int j = i; j + 1 < c.n_execs; ++j) c.execs[j] = c.execs[j + 1];
      --c.n_execs;
      return x;
    }
  return nullptr;
}

// Keep the executable of a destroyed plan (its stream has been synchronised), or
// destroy it when the cache is full.
void give_back_exec(int dev, cudaGraphExec_t x, const ExecKey& key) {
  if (!x) return;
  if (dev >= 0 && dev < OFA_MAX_DEVICES) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    DeviceCache& c = g_cache[dev];
    if (c.n_execs < OFA_CACHED_EXECS) {
      c.execs[c.n_execs++] = {x, key};
      return;
    }
  }
  cudaGraphExecDestroy(x);
}

OfaDevState* take_cached_st_host(int dev) {
  if (dev < 0 || dev >= OFA_MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  OfaDevState* h = g_cache[dev].st_host;
  g_cache[dev].st_host = nullptr;
  return h;
}

void give_back_st_host(int dev, OfaDevState* h) {
  if (dev >= 0 && dev < OFA_MAX_DEVICES) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (!g_cache[dev].st_host) {
      g_cache[dev].st_host = h;
      return;
    }
  }
  cudaFreeHost(h);
}

cudaError_t arena_commit(ofa_plan* p, const std::vector<ArenaReq>& reqs) {
  std::vector<size_t> off(reqs.size());
  size_t total = 0;
  for (size_t i = 0; i < reqs.size(); ++i) {
    total = (total + 255) & ~(size_t)255;
    off[i] = total;
    total += reqs[i].bytes;
  }
  if (total == 0) total = 256;
  size_t bytes = 0;
  void* base = take_cached_arena(p->device, total, &bytes);
  if (!base) {
    cudaError_t e = cudaMalloc(&base, total);
    if (e != cudaSuccess) return e;
    bytes = total;
  }
  p->arena = base;
  p->arena_bytes = bytes;
  for (size_t i = 0; i < reqs.size(); ++i) {
    *reqs[i].slot = static_cast<uint8_t*>(base) + off[i];
    p->arena_slots.push_back(reqs[i].slot);
  }
  // every later set-up copy and kernel runs on the plan's stream, after the fill
  return cudaMemsetAsync(base, 0, total, p->stream);
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

// The tensor-core products run unless the plan uses the separable grid form (whose
// products are small and run on the CUDA cores in FP32).
inline bool use_tc(const ofa_plan* p) { return prec_is_tc(p->precision) && !p->sep; }

cudaMemcpyKind kind_from(int mem_space) {
  return mem_space == OFA_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}

void free_tc(TcOperands& t) {
  dfree(t.e_hi);
  dfree(t.e_lo);
  dfree(t.bx_hi);
  dfree(t.bx_lo);
  dfree(t.p_hi);
  dfree(t.p_lo);
  dfree(t.q_hi);
  dfree(t.q_lo);
  t = TcOperands();
}

// Tile choice for the two products (cost model: waves x per-CTA MMA work).
void choose_tiles(ofa_plan* p, TcOperands& t, int sms) {
  const int tiles_m = p->nyp / 128;
  const int kb_fwd = (2 * p->nxp * t.elem_bytes) / t.fwd_rb;
  double best = 1e30;
  for (int bn : {256, 128}) {
    for (int split = 1; split <= 8; split *= 2) {
      if (kb_fwd / split < 4) break;
      const long ctas = (long)tiles_m * (2 * t.kp / bn) * split;
      const long waves = (ctas + sms - 1) / sms;
      const double cost = (double)waves * ((double)kb_fwd / split) * bn * t.npass +
                          0.02 * split * tiles_m * 2.0 * t.kp;
      if (cost < best - 1e-9) {
        best = cost;
        t.fwd_bn = bn;
        t.fwd_split = split;
      }
    }
  }
  best = 1e30;
  for (int bn : {256, 128}) {
    const long ctas = (long)tiles_m * (2 * p->nxp / bn);
    const long waves = (ctas + sms - 1) / sms;
    const double cost = (double)waves * bn;
    if (cost < best - 1e-9) {
      best = cost;
      t.bwd_bn = bn;
    }
  }
}

// Separable form on the tensor cores: the forward's tiles and contraction parts (about
// one CTA per SM, at least two k-blocks per part), the inverse as choose_tiles has it.
int sep_tc_split(const ofa_plan* p, const TcOperands& t, int sms) {
  const int tiles = (p->nyp / 128) * (2 * t.kp / t.fwd_bn);
  const int kb_fwd = (2 * p->nxp * t.elem_bytes) / t.fwd_rb;
  int split = 1;
  while (split < SEP_TC_MAX_PARTS && tiles * split * 2 <= sms && kb_fwd / (split * 2) >= 2)
    split *= 2;
  return split;
}

ofa_status alloc_tc(ofa_plan* p, TcOperands& t, bool with_static) {
  const int eb = prec_elem_bytes(p->precision);
  t.elem_bytes = eb;
  t.npass = prec_npass(p->precision);
  // the planes' focus dimension: the foci, or the separable form's distinct x
  t.kp = p->sep_tc ? round_up(p->ux, 64) : p->kp;
  const size_t e_n = (size_t)p->nyp * 2 * p->nxp;
  const size_t bx_n = (size_t)2 * t.kp * 2 * p->nxp;
  const size_t pp_n = (size_t)p->nyp * 2 * t.kp;
  // reserve or allocate straight into the operand's own slot (an arena commit
  // writes the final address there later)
  auto A = [&](void** ptr, size_t n) -> bool {
    return dalloc(reinterpret_cast<uint8_t**>(ptr), n * eb) == cudaSuccess;
  };
  bool ok = A(&t.e_hi, e_n) && (t.npass == 1 || A(&t.e_lo, e_n));
  if (with_static) {
    ok = ok && A(&t.bx_hi, bx_n) && (t.npass == 1 || A(&t.bx_lo, bx_n));
    ok = ok && A(&t.p_hi, pp_n) && (t.npass == 1 || A(&t.p_lo, pp_n));
    ok = ok && A(&t.q_hi, bx_n) && (t.npass == 1 || A(&t.q_lo, bx_n));
  }
  return ok ? OFA_OK : OFA_ERR_OOM;
}

// The key of a plan's graph of `iters` iterations: sizes, form, precision and tiles.
ExecKey exec_key(const ofa_plan* p, int iters) {
  const TcOperands& t = p->tc;
  return {iters,       p->precision, p->nx,      p->ny,      p->K,        p->kp,
          p->nxp,      p->nyp,       p->sep,     p->sep_fast, p->sep_tc,  p->ux,
          p->uy,       p->weighting, p->sm_count, t.kp,     t.fwd_bn,    t.fwd_split,
          t.fwd_cg,    t.bwd_bn,     t.bwd_cg,  t.fwd_rb,   t.bwd_rb,    t.npass};
}

void destroy_graphs(ofa_plan* p) {
  give_back_exec(p->device, p->chunk_exec, exec_key(p, p->chunk_iters));
  give_back_exec(p->device, p->one_exec, exec_key(p, 1));
  p->chunk_exec = p->one_exec = nullptr;
}

int* done_ptr(ofa_plan* p) { return &p->st->done; }

// One iteration of Algorithm 1 on stream s.
// Separable grid form: the forward through the distinct x (G = E Fxu^T, then
// Theta_k = Fyu[iy_k] . G[:, ix_k]) into the single partial row.
// FP32 inverse operand of the separable form: the conjugate of the first inverse
// product, transposed, into p->simt.fxT [nx][ldk] (Fyu^T is formed once per plan).
void sep_transpose_t(ofa_plan* p, cudaStream_t s) {
  launch_transpose_fy(p->tconj, p->uy, p->nx, simt_ldk(p->uy), p->nx, p->simt.fxT, s, true);
}

// Separable form, the inverse from c: T by grid rows, then the second inverse product
// fused with the phase projection (one launch forming T per tile when it fits).
void enqueue_sep_inverse(ofa_plan* p, const int* done, cudaStream_t s) {
  if (p->sep_fast) {
    launch_sep_inverse(p->c, p->sep_gridk, p->fxu, p->fyu, p->amp, p->nx, p->ny, p->ux, p->uy,
                       p->phi, p->e32, done, s);
    return;
  }
  launch_sep_t(p->c, p->fxu, p->ixy, p->row_ptr, p->row_foci, p->uy, p->nx, p->tconj, s);
  sep_transpose_t(p, s);
  launch_bwd_simt(p->ones, p->simt.fxT, p->simt.fyT, p->nx, p->ny, p->uy, p->amp, p->phi, p->e32,
                  done, p->simt, s);
}

// Separable form, forward at the foci for the field e32: Theta in partial row 0.
void enqueue_sep_forward(ofa_plan* p, const float2* e32, cudaStream_t s) {
  if (p->sep_fast) {
    const FocalTail off = {};
    launch_sep_fwd(e32, p->fxu, p->fyu, p->ixy, p->nx, p->ny, p->ux, p->uy, p->K, p->kp,
                   p->sm_count, p->part, off, nullptr, s);
    launch_sep_sum_focal(p->part, sep_fwd_blocks(p->ny, p->sm_count), p->K, p->kp, p->part, 0,
                         p->t, p->w, p->c, p->hist, p->st, p->weighting, p->counters, nullptr, s);
    return;
  }
  launch_sep_forward(e32, p->fxu, p->nx, p->ny, p->ux, p->sep_parts, p->gt, s);
  launch_sep_theta(p->gt, p->fyu, p->ixy, p->K, p->ny, p->ux, p->sep_parts, p->part, s);
}

// The iteration takes no amplitude statistic (the energy enters only the statistics
// of mode 1), so plan creation captures it before the statistics are read back.
void enqueue_iteration(ofa_plan* p, cudaStream_t s) {
  const int* done = done_ptr(p);
  if (p->sep_tc) {
    // separable form on the tensor cores: G per contraction part, Theta from G, the
    // focal step with U = conj(Fy_u)^T C, then E' = U conj(Fx_u) with the phase projection
    launch_fwd_sep_tc(p, p->tc, done, s);
    launch_sep_tc_theta(p->gt, p->tc.fwd_split, p->fyu, p->sep_gridk, p->ny, p->ux, p->uy, p->K,
                        p->part, p->w, p->sep_wprev, done, s);
    launch_sep_focal_u(p->part, p->t, p->sep_wprev, p->w, p->c, p->hist, p->st, p->weighting,
                       p->ixy, p->K, p->fyu, done, p->ny, p->ux, p->uy, p->tc.kp, p->precision,
                       p->tc.p_hi, p->tc.p_lo, s);
    launch_bwd_tc(p, p->tc, done, s);
  } else if (p->sep && p->sep_fast) {
    const FocalTail f = {p->t, p->w, p->c, p->hist, p->st, p->weighting, p->counters, 1};
    launch_sep_fwd(p->e32, p->fxu, p->fyu, p->ixy, p->nx, p->ny, p->ux, p->uy, p->K, p->kp,
                   p->sm_count, p->part, f, done, s);
    if (!sep_fwd_fuses_focal(p->ny, p->K, p->sm_count))
      launch_sep_sum_focal(p->part, sep_fwd_blocks(p->ny, p->sm_count), p->K, p->kp, p->part, 1,
                           p->t, p->w, p->c, p->hist, p->st, p->weighting, p->counters, done, s);
    enqueue_sep_inverse(p, done, s);
  } else if (p->sep) {
    enqueue_sep_forward(p, p->e32, s);
    launch_focal(p->part, 1, p->kp, p->K, p->t, p->w, p->theta, p->inten, p->c, p->hist, p->st,
                 0, p->weighting, 1.f, 0.0, s);
    enqueue_sep_inverse(p, done, s);
  } else if (!use_tc(p)) {
    const FocalTail f = {p->t, p->w, p->c, p->hist, p->st, p->weighting, nullptr, 1};
    launch_fwd_simt(p->e32, p->fx, p->fy, p->nx, p->ny, p->K, p->kp, p->part, done, p->simt, s,
                    &f);
    if (!simt_fwd_fuses_focal(p->K))
      launch_focal(p->part, simt_fwd_tiles(p->ny), p->kp, p->K, p->t, p->w, p->theta, p->inten,
                   p->c, p->hist, p->st, 0, p->weighting, 1.f, 0.0, s);
    launch_bwd_simt(p->c, p->simt.fxT, p->simt.fyT, p->nx, p->ny, p->K, p->amp, p->phi, p->e32,
                    done, p->simt, s);
  } else {
    // up to 4096 foci the focal step runs in the forward kernel's last CTA
    const bool fuse = p->K <= 4096;
    launch_fwd_tc(p, p->tc, done, s, fuse);
    if (!fuse)
      launch_focal(p->part, fwd_n_part(p->nyp, p->tc), p->kp, p->K, p->t, p->w, p->theta,
                   p->inten, p->c, p->hist, p->st, 0, p->weighting, 1.f, 0.0, s);
    launch_build_p(p->fyT, p->c, done, p->nyp, p->kp, p->precision, p->tc.p_hi, p->tc.p_lo, s);
    launch_bwd_tc(p, p->tc, done, s);
  }
}

// The separable form on the tensor cores iterates on the operand planes; its FP32
// entry points take the field of the current phase from this.
void sep_tc_refresh_e32(ofa_plan* p, cudaStream_t s) {
  if (p->sep_tc) launch_field_f32(p->phi, p->amp, p->nx, p->ny, p->e32, s);
}

// ... and after an FP32 step has moved the phase, the iteration's planes follow it.
void sep_tc_refresh_planes(ofa_plan* p, cudaStream_t s) {
  if (p->sep_tc)
    launch_field_planes(p->phi, p->amp, p->nx, p->ny, p->nxp, p->precision, p->tc.e_hi,
                        p->tc.e_lo, s);
}

// Forward at the loop's current phase + statistics (mode 1) or output (mode 2).
void enqueue_forward_current(ofa_plan* p, cudaStream_t s) {
  if (p->sep) {
    sep_tc_refresh_e32(p, s);
    enqueue_sep_forward(p, p->e32, s);
    launch_focal(p->part, 1, p->kp, p->K, p->t, p->w, p->theta, p->inten, p->c, p->hist, p->st,
                 1, p->weighting, ldexpf(1.f, p->amp_exp), p->amp_energy, s);
  } else if (!use_tc(p)) {
    launch_fwd_simt(p->e32, p->fx, p->fy, p->nx, p->ny, p->K, p->kp, p->part, nullptr, p->simt,
                    s);
    launch_focal(p->part, simt_fwd_tiles(p->ny), p->kp, p->K, p->t, p->w, p->theta, p->inten,
                 p->c, p->hist, p->st, 1, p->weighting, ldexpf(1.f, p->amp_exp), p->amp_energy,
                 s);
  } else {
    launch_fwd_tc(p, p->tc, nullptr, s, false);
    launch_focal(p->part, fwd_n_part(p->nyp, p->tc), p->kp, p->K, p->t, p->w, p->theta,
                 p->inten, p->c, p->hist, p->st, 1, p->weighting, ldexpf(1.f, p->amp_exp),
                 p->amp_energy, s);
  }
}

ofa_status build_graph(ofa_plan* p, int iters, cudaGraphExec_t* exec) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return ofa_cuda_check(p, e, "cudaStreamBeginCapture");
  for (int i = 0; i < iters; ++i) enqueue_iteration(p, p->cap_stream);
  e = cudaStreamEndCapture(p->cap_stream, &g);
  if (e != cudaSuccess) return ofa_cuda_check(p, e, "cudaStreamEndCapture");
  // an executable that a destroyed plan of the same key left takes this graph's kernel
  // arguments (the update also checks that nodes and kernels match); else instantiate
  if (cudaGraphExec_t cached = take_cached_exec(p->device, exec_key(p, iters))) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(cached, g, &info) == cudaSuccess) {
      cudaGraphDestroy(g);
      *exec = cached;
      return OFA_OK;
    }
    cudaGetLastError();   // the refused update leaves no error behind
    cudaGraphExecDestroy(cached);
  }
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return ofa_cuda_check(p, e, "cudaGraphInstantiate");
}

ofa_status sync_and_check(ofa_plan* p) {
  cudaError_t e = cudaMemcpyAsync(p->st_host, p->st, sizeof(OfaDevState), cudaMemcpyDeviceToHost,
                                  p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  ofa_status s = ofa_cuda_check(p, e, "synchronising the plan's stream");
  if (s != OFA_OK) return s;
  if (p->st_host->err & OFA_ERRBIT_TIMEOUT)
    return ofa_fail(p, OFA_ERR_TIMEOUT, "a bounded device wait gave up (tensor-core pipeline)");
  if (p->st_host->err & OFA_ERRBIT_LAUNCH)
    return ofa_fail(p, OFA_ERR_CUDA,
                    "the fused loop kernel ran without its 2-CTA clusters or co-resident grid");
  if (p->st_host->err & OFA_ERRBIT_NUMERIC)
    return ofa_fail(p, OFA_ERR_NUMERIC, "sum of focus intensities is zero or not finite");
  return OFA_OK;
}

ofa_status ensure_aux(ofa_plan* p) {
  if (!use_tc(p) || p->aux_ready) return OFA_OK;
  TcOperands& a = p->tc_aux;
  a = p->tc;  // shares the static operands and their maps
  a.e_hi = a.e_lo = nullptr;
  TcOperands tmp;
  tmp.elem_bytes = p->tc.elem_bytes;
  tmp.npass = p->tc.npass;
  ofa_status s = alloc_tc(p, tmp, false);
  if (s != OFA_OK) {
    free_tc(tmp);
    return ofa_fail(p, s, "allocating forward/adjoint field planes");
  }
  a.e_hi = tmp.e_hi;
  a.e_lo = tmp.e_lo;
  std::string err;
  TcOperands probe = a;
  if (!tc_encode_maps(p, probe, err)) {
    dfree(a.e_hi);
    dfree(a.e_lo);
    return ofa_fail(p, OFA_ERR_CUDA, err);
  }
  a.tm_e_hi = probe.tm_e_hi;
  a.tm_e_lo = probe.tm_e_lo;
  p->aux_ready = true;
  return OFA_OK;
}

}  // namespace

// ------------------------------------------------------------------ shared helpers
ofa_status ofa_fail(ofa_plan* p, ofa_status s, const std::string& msg) {
  if (p) p->last_error = msg;
  else g_thread_error = msg;
  return s;
}

ofa_status ofa_cuda_check(ofa_plan* p, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return OFA_OK;
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  return ofa_fail(p, e == cudaErrorMemoryAllocation ? OFA_ERR_OOM : OFA_ERR_CUDA, msg);
}

void ofa_set_thread_error(const std::string& msg) { g_thread_error = msg; }

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* ofa_status_string(ofa_status s) {
  int i = (int)s;
  if (i < 0 || i >= (int)(sizeof(kStatusNames) / sizeof(kStatusNames[0]))) return "OFA_UNKNOWN";
  return kStatusNames[i];
}

const char* ofa_last_error(const ofa_plan* p) {
  return p ? p->last_error.c_str() : g_thread_error.c_str();
}

ofa_status ofa_options_default(ofa_options* o) {
  if (!o) return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "options pointer is NULL");
  std::memset(o, 0, sizeof(*o));
  o->precision = OFA_PREC_F16X3;
  o->seed = 0;
  o->cuda_stream = nullptr;
  o->amplitude = nullptr;
  o->waist_frac = 0.4;
  o->phi0 = nullptr;
  o->mem_space = OFA_MEM_HOST;
  o->weighting = 1;
  o->autotune = 1;
  o->focus_z = nullptr;
  o->separable = -1;
  o->fused_loop = 0;
  o->separable_loop = -1;
  o->separable_tc = -1;
  return OFA_OK;
}

ofa_status ofa_fft_equivalent_size(int m0, double pitch, double wavelength, double focal_length,
                                   double focal_sampling, int* m_out) {
  if (m0 < 1 || !finite_pos(pitch) || !finite_pos(wavelength) || !finite_pos(focal_length) ||
      !finite_pos(focal_sampling) || !m_out)
    return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "ofa_fft_equivalent_size: bad argument");
  const double na = m0 * pitch / (2.0 * focal_length);      // NA of the pupil aperture
  const double m = m0 * wavelength / (2.0 * na * focal_sampling);
  if (!(m < 2147483647.0))
    return ofa_fail(nullptr, OFA_ERR_OUT_OF_RANGE, "ofa_fft_equivalent_size: overflow");
  *m_out = (int)std::ceil(m - 1e-9);
  return OFA_OK;
}

ofa_status ofa_max_foci_per_axis(double pitch, double wavelength, double focal_length, double gap,
                                 int* count_out) {
  if (!finite_pos(pitch) || !finite_pos(wavelength) || !finite_pos(focal_length) ||
      !finite_pos(gap) || !count_out)
    return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "ofa_max_foci_per_axis: bad argument");
  const double field = wavelength * focal_length / pitch;    // alias-free field width
  *count_out = (int)std::floor(field / gap + 1e-12);
  return OFA_OK;
}

ofa_status ofa_check_foci(int n_foci, const double* xy, double px, double py, double wavelength,
                          double focal_length, int* bad_index) {
  if (bad_index) *bad_index = -1;
  if (n_foci < 1 || !xy || !finite_pos(px) || !finite_pos(py) || !finite_pos(wavelength) ||
      !finite_pos(focal_length))
    return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "ofa_check_foci: bad argument");
  const double hx = wavelength * focal_length / (2.0 * px);
  const double hy = wavelength * focal_length / (2.0 * py);
  for (int k = 0; k < n_foci; ++k) {
    const double x = xy[2 * k], y = xy[2 * k + 1];
    if (!std::isfinite(x) || !std::isfinite(y)) {
      if (bad_index) *bad_index = k;
      return ofa_fail(nullptr, OFA_ERR_INVALID_ARG,
                      "focus " + std::to_string(k) + " has a non-finite coordinate");
    }
    if (std::fabs(x) >= hx || std::fabs(y) >= hy) {
      if (bad_index) *bad_index = k;
      return ofa_fail(nullptr, OFA_ERR_OUT_OF_RANGE,
                      "focus " + std::to_string(k) + " lies outside the alias-free field");
    }
  }
  return OFA_OK;
}

ofa_status ofa_plan_config(const ofa_plan* p, int* c) {
  if (!p || !c) return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < 12; ++i) c[i] = 0;
  if (p->sep_loop) {
    c[8] = 1; c[11] = p->sep_loop_grid;
    return OFA_OK;
  }
  if (!use_tc(p) && !p->sep_tc) return OFA_OK;
  const TcOperands& t = p->tc;
  c[0] = t.fwd_bn; c[1] = t.fwd_split; c[2] = t.fwd_cg; c[3] = t.bwd_bn; c[4] = t.bwd_cg;
  c[5] = p->K <= 4096 && !p->sep_tc ? 1 : 0; c[6] = t.fwd_rb; c[7] = t.bwd_rb;
  if (p->loop.ready) {
    c[8] = 1; c[9] = p->loop.cg; c[10] = p->loop.split; c[11] = p->loop.grid;
  }
  return OFA_OK;
}

ofa_status ofa_plan_form(const ofa_plan* p, int* separable, int* ux, int* uy) {
  if (!p) return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "plan is NULL");
  if (separable) *separable = p->sep ? 1 : 0;
  if (ux) *ux = p->sep ? p->ux : 0;
  if (uy) *uy = p->sep ? p->uy : 0;
  return OFA_OK;
}

ofa_status ofa_plan_info(const ofa_plan* p, int* nx, int* ny, int* n_foci, int* precision) {
  if (!p) return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "plan is NULL");
  if (nx) *nx = p->nx;
  if (ny) *ny = p->ny;
  if (n_foci) *n_foci = p->K;
  if (precision) *precision = p->precision;
  return OFA_OK;
}

ofa_status ofa_destroy(ofa_plan* p) {
  if (!p) return OFA_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  // the plan's work must be finished before its arena is handed to another plan
  cudaStreamSynchronize(p->stream);
  destroy_graphs(p);
  if (p->arena) {
    give_back_arena(p->device, p->arena, p->arena_bytes);
    for (void** slot : p->arena_slots) *slot = nullptr;
    p->arena = nullptr;
  }
  void* bufs[] = {p->focus_xy, p->focus_z, p->t,     p->amp,   p->phi,   p->w,    p->fx,
                  p->fy,       p->fyT,   p->part,  p->theta, p->inten, p->c,
                  p->hist,     p->st,    p->scratch_phi, p->counters, p->e32, p->e32_aux,
                  p->meas,     p->fxu,   p->fyu,   p->gt,    p->tconj, p->ones, p->ixy,
                  p->row_ptr,  p->row_foci, p->sep_gridk};
  for (void* b : bufs) dfree(b);
  if (p->st_host) give_back_st_host(p->device, p->st_host);
  free_tc(p->tc);
  if (p->aux_ready) {
    dfree(p->tc_aux.e_hi);
    dfree(p->tc_aux.e_lo);
  }
  give_back_stream(p->device, p->cap_stream);
  if (p->own_stream) give_back_stream(p->device, p->stream);
  if (prev >= 0) cudaSetDevice(prev);
  delete p;
  return OFA_OK;
}

ofa_status ofa_plan_create(ofa_plan** out, int nx, int ny, double pitch_x, double pitch_y,
                           double wavelength, double focal_length, int n_foci,
                           const double* focus_xy, const float* target_intensity,
                           const ofa_options* opt_in) {
  if (!out) return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "out pointer is NULL");
  *out = nullptr;
  ofa_options opt;
  if (opt_in) opt = *opt_in;
  else ofa_options_default(&opt);
  if (nx < 1 || ny < 1 || n_foci < 1 || !focus_xy || !target_intensity)
    return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "sizes must be >= 1 and pointers non-NULL");
  if (nx > 32768 || ny > 32768 || n_foci > (1 << 22))
    return ofa_fail(nullptr, OFA_ERR_UNSUPPORTED, "pupil or focus count too large");
  if (!finite_pos(pitch_x) || !finite_pos(pitch_y) || !finite_pos(wavelength) ||
      !finite_pos(focal_length))
    return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "pitch, wavelength and focal length must be > 0");
  if (opt.precision < OFA_PREC_FP32 || opt.precision > OFA_PREC_F16X3)
    return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "unknown precision");
  if (opt.mem_space != OFA_MEM_HOST && opt.mem_space != OFA_MEM_DEVICE)
    return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "unknown memory space");
  if (!opt.amplitude && !finite_pos(opt.waist_frac))
    return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "waist_frac must be > 0");

  const size_t npix = (size_t)nx * ny;
  // Host copies of the small inputs for validation.
  std::vector<double> xy(2 * (size_t)n_foci);
  std::vector<float> tgt(n_foci);
  std::vector<double> zz(opt.focus_z ? (size_t)n_foci : 0);
  if (opt.mem_space == OFA_MEM_DEVICE) {
    cudaError_t e = cudaMemcpy(xy.data(), focus_xy, xy.size() * sizeof(double),
                               cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(tgt.data(), target_intensity, tgt.size() * sizeof(float),
                     cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && opt.focus_z)
      e = cudaMemcpy(zz.data(), opt.focus_z, zz.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ofa_cuda_check(nullptr, e, "reading device inputs");
  } else {
    std::memcpy(xy.data(), focus_xy, xy.size() * sizeof(double));
    std::memcpy(tgt.data(), target_intensity, tgt.size() * sizeof(float));
    if (opt.focus_z) std::memcpy(zz.data(), opt.focus_z, zz.size() * sizeof(double));
  }
  ofa_status vs = ofa_check_foci(n_foci, xy.data(), pitch_x, pitch_y, wavelength, focal_length,
                                 nullptr);
  if (vs != OFA_OK) return vs;
  // row shard: rows [row0, row0 + ny) of a pupil of ny_total rows
  const bool shard = opt.shard_ny_total != 0;
  const int row0 = shard ? opt.shard_row0 : 0;
  const int ny_total = shard ? opt.shard_ny_total : ny;
  if (shard && (row0 < 0 || opt.shard_ny_total < ny || row0 > opt.shard_ny_total - ny))
    return ofa_fail(nullptr, OFA_ERR_INVALID_ARG,
                    "a row shard needs 0 <= shard_row0 and shard_row0 + ny <= shard_ny_total");
  if (!shard && opt.shard_row0 != 0)
    return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "shard_row0 needs shard_ny_total");
  if (shard && opt.separable == 1)
    return ofa_fail(nullptr, OFA_ERR_UNSUPPORTED, "the separable form runs whole pupils only");
  if (opt.focus_z) {
    // the defocus phase shifts the local spatial frequency at the pupil edge by
    // z u_max / (lambda f^2): the effective position |x| + |z| u_max / f must stay
    // inside the alias-free field
    const double hx = wavelength * focal_length / (2.0 * pitch_x);
    const double hy = wavelength * focal_length / (2.0 * pitch_y);
    const double ux = 0.5 * (nx - 1) * pitch_x, uy = 0.5 * (ny_total - 1) * pitch_y;
    for (int k = 0; k < n_foci; ++k) {
      const double z = zz[k];
      if (!std::isfinite(z))
        return ofa_fail(nullptr, OFA_ERR_INVALID_ARG,
                        "focus " + std::to_string(k) + " has a non-finite axial offset");
      if (std::fabs(z) >= focal_length ||
          std::fabs(xy[2 * k]) + std::fabs(z) * ux / focal_length >= hx ||
          std::fabs(xy[2 * k + 1]) + std::fabs(z) * uy / focal_length >= hy)
        return ofa_fail(nullptr, OFA_ERR_OUT_OF_RANGE,
                        "focus " + std::to_string(k) +
                            ": the defocus phase of its axial offset is not sampled by the pupil");
    }
  }
  double tsum = 0.0;
  for (int k = 0; k < n_foci; ++k) {
    if (!std::isfinite(tgt[k]) || tgt[k] < 0.f)
      return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "target intensities must be finite and >= 0");
    tsum += tgt[k];
  }
  if (!(tsum > 0.0)) return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "target intensities sum to 0");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ofa_cuda_check(nullptr, e, "cudaGetDevice");
  int cc = 0, sm_count = 0;
  e = device_attrs(dev, &cc, &sm_count);
  if (e != cudaSuccess) return ofa_cuda_check(nullptr, e, "cudaDeviceGetAttribute");
  if (cc != 103)
    return ofa_fail(nullptr, OFA_ERR_UNSUPPORTED,
                    "this library is built for sm_103a (GB300) only; device is sm_" +
                        std::to_string(cc));

  ofa_plan* p = new ofa_plan();
  p->device = dev;
  p->nx = nx;
  p->ny = ny;
  p->row0 = row0;
  p->ny_total = ny_total;
  p->K = n_foci;
  p->precision = opt.precision;
  p->weighting = opt.weighting ? 1 : 0;
  p->px = pitch_x;
  p->py = pitch_y;
  p->lambda = wavelength;
  p->focal = focal_length;
  p->sm_count = sm_count;
  p->nxp = round_up(nx, 128);
  p->nyp = round_up(ny, 128);
  p->kp = round_up(n_foci, 128);

  // Separable grid form: with foci on the grid of their ux distinct x and uy distinct
  // y coordinates, Eq. 2 factors through those values (Theta on the grid is
  // Fyu E Fxu^T), costing nx ny (ux + uy) complex products instead of 2 nx ny K.
  std::vector<double> xs, ys;
  if (opt.separable != 0 && !opt.focus_z && !shard) {
    // The grid form runs on the CUDA cores: by default it is taken where its work,
    // nx ny (U_x + U_y) + K (nx + ny), is under 1/20 of the tensor-core forms'
    // 2 nx ny K_p (1/2 of the FP32 form's), where it was always the faster in
    // measurements (1000^2 pupil, 45 x 47 grid: 22 k vs 11 k it/s).  Smaller savings
    // can win too (9 x 9 grid, 14x less work: 60 k vs 41 k it/s): separable = 1.
    // The distinct values are counted only up to the bound this puts on U_x + U_y,
    // so a plan of scattered foci stops early.
    const double npix_d = (double)nx * ny;
    const double c_gen = 2.0 * npix_d * (double)round_up(n_foci, 128);
    const double gain = prec_is_tc(opt.precision) ? 20.0 : 2.0;
    const double bound = (c_gen / gain - (double)n_foci * (nx + ny)) / npix_d;
    const size_t limit = opt.separable == 1 ? (size_t)n_foci
                         : bound < 1.0 ? 0 : (size_t)std::min(bound, (double)n_foci);
    bool fits = ofa_host::distinct_coords(xy.data(), n_foci, 0, limit, xs);
    if (fits)
      fits = ofa_host::distinct_coords(xy.data(), n_foci, 1,
                                       opt.separable == 1 ? limit : limit - xs.size(), ys);
    if (fits && opt.separable != 1) {
      const double c_sep = npix_d * ((double)xs.size() + (double)ys.size()) +
                           (double)n_foci * (nx + ny);
      fits = c_sep * gain < c_gen;
    }
    p->sep = fits;
    p->ux = fits ? (int)xs.size() : 0;
    p->uy = fits ? (int)ys.size() : 0;
  }
  if (opt.separable == 1 && !p->sep) {
    delete p;
    return ofa_fail(nullptr, OFA_ERR_UNSUPPORTED, "the separable form needs 2D foci");
  }
  if (opt.separable_tc < -1 || opt.separable_tc > 1) {
    delete p;
    return ofa_fail(nullptr, OFA_ERR_UNSUPPORTED, "separable_tc must be -1, 0 or 1");
  }
  // The separable iteration on the tensor cores: a tensor-core precision, at most
  // SEP_TC_MAX_UX distinct x (one MMA tile of columns) and one focus per grid point.
  if (p->sep && opt.separable_tc != 0) {
    bool ok = prec_is_tc(opt.precision) && p->ux <= SEP_TC_MAX_UX && p->uy <= SEP_TC_MAX_UY &&
              sep_focal_u_fits(p->ux, p->uy, n_foci);
    if (ok) ok = ofa_host::one_focus_per_point(xy.data(), n_foci);
    if (!ok && opt.separable_tc == 1) {
      delete p;
      return ofa_fail(nullptr, OFA_ERR_UNSUPPORTED,
                      "the separable form on the tensor cores needs a tensor-core precision, "
                      "at most 128 distinct x and y, 4096 foci and one focus per grid point");
    }
    if (ok && opt.separable_tc == 1 && opt.separable_loop == 1) {
      delete p;
      return ofa_fail(nullptr, OFA_ERR_UNSUPPORTED,
                      "separable_tc = 1 and separable_loop = 1 exclude each other");
    }
    p->sep_tc = ok && (opt.separable_tc == 1 || p->ux + p->uy > 48);
    if (p->sep_tc) {
      // the forward's configuration (the contraction parts size p->gt)
      p->tc.elem_bytes = prec_elem_bytes(opt.precision);
      p->tc.npass = prec_npass(opt.precision);
      p->tc.kp = round_up(p->ux, 64);
      p->tc.fwd_bn = 128;
      p->tc.fwd_cg = 1;
      p->tc.fwd_split = sep_tc_split(p, p->tc, sm_count);
    }
  }

  auto fail = [&](ofa_status s) {
    g_thread_error = p->last_error;
    g_fault_alloc_countdown = 0;
    g_arena = nullptr;
    ofa_destroy(p);
    return s;
  };
  {
    const char* f = getenv("OFA_FAULT_ALLOC");
    g_fault_alloc_countdown = f ? std::max(0, atoi(f)) : 0;
  }
#define OFA_TRY(call, what)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return fail(ofa_cuda_check(p, e_, what)); \
  } while (0)

  if (opt.cuda_stream) {
    p->stream = static_cast<cudaStream_t>(opt.cuda_stream);
  } else {
    OFA_TRY(take_stream(dev, &p->stream), "creating stream");
    p->own_stream = true;
  }
  OFA_TRY(take_stream(dev, &p->cap_stream), "creating capture stream");

  const bool tc = use_tc(p);
  const int n_part_max = tc ? (p->nyp / 128) * 8
                            : std::max(simt_fwd_tiles(ny), p->sep ? sep_fwd_blocks(ny, sm_count) : 1);
  // Reserve every device buffer, then carve them out of one allocation.
  std::vector<ArenaReq> reqs;
  g_arena = &reqs;
  auto reserve_all = [&]() -> cudaError_t {
    cudaError_t e = cudaSuccess;
    auto R = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    R(dalloc(&p->focus_xy, 2 * (size_t)n_foci));
    if (opt.focus_z) R(dalloc(&p->focus_z, (size_t)n_foci));
    R(dalloc(&p->t, n_foci));
    R(dalloc(&p->amp, npix));
    R(dalloc(&p->phi, npix));
    R(dalloc(&p->w, n_foci));
    R(dalloc(&p->fx, (size_t)n_foci * nx));
    R(dalloc(&p->fy, (size_t)n_foci * ny));
    R(dalloc(&p->part, (size_t)n_part_max * p->kp));
    R(dalloc(&p->theta, n_foci));
    R(dalloc(&p->inten, n_foci));
    R(dalloc(&p->c, p->kp));
    R(dalloc(&p->hist, OFA_HIST_CAP));
    R(dalloc(&p->counters, p->kp / 64 + 1));
    R(dalloc(&p->loop_bar, 4));
    R(dalloc(&p->meas, n_foci));
    R(dalloc(&p->amp_part, 3 * (size_t)AMP_STAT_BLOCKS));
    R(dalloc(&p->amp_count, 1));
    if (p->sep) {
      R(dalloc(&p->fxu, (size_t)p->ux * nx));
      R(dalloc(&p->fyu, (size_t)p->uy * ny));
      p->sep_parts = sep_parts(nx, ny, p->ux, sm_count);
      const int gt_parts = std::max(p->sep_parts, p->sep_tc ? p->tc.fwd_split : 1);
      R(dalloc(&p->gt, (size_t)gt_parts * p->ux * ny));
      R(dalloc(&p->tconj, (size_t)p->uy * nx));
      R(dalloc(&p->ones, (size_t)p->uy));
      R(dalloc(&p->ixy, (size_t)n_foci));
      R(dalloc(&p->row_ptr, (size_t)p->uy + 1));
      R(dalloc(&p->row_foci, (size_t)n_foci));
      R(dalloc(&p->sep_gridk, (size_t)p->ux * p->uy));
      if (p->sep_tc) R(dalloc(&p->sep_wprev, (size_t)n_foci));
      R(dalloc(&p->sep_coord, 2 * ((size_t)p->ux + p->uy)));
    }
    R(dalloc(&p->st, 1));
    if (!tc) {
      R(dalloc(&p->e32, npix));
      R(dalloc(&p->e32_aux, npix));
      const SimtSizes z = simt_sizes(nx, ny, n_foci, p->sep ? p->uy : n_foci);
      R(dalloc(&p->simt.p32, z.p32));
      R(dalloc(&p->simt.fxT, z.fxT));
      R(dalloc(&p->simt.fyT, z.fyT));
      R(dalloc(&p->simt.fws, z.fws));
      R(dalloc(&p->simt.cnt, z.cnt));
      // the separable form on the tensor cores keeps the FP32 buffers for its other
      // entry points
      if (p->sep_tc && e == cudaSuccess && alloc_tc(p, p->tc, true) != OFA_OK)
        e = cudaErrorMemoryAllocation;
    } else {
      R(dalloc(&p->fyT, (size_t)p->nyp * p->kp));
      if (e == cudaSuccess && alloc_tc(p, p->tc, true) != OFA_OK) e = cudaErrorMemoryAllocation;
    }
    return e;
  };
  {
    cudaError_t re = reserve_all();
    g_arena = nullptr;
    OFA_TRY(re, "alloc");
  }
  OFA_TRY(arena_commit(p, reqs), "alloc");
  p->st_host = take_cached_st_host(dev);
  if (!p->st_host)
    OFA_TRY(cudaMallocHost(reinterpret_cast<void**>(&p->st_host), sizeof(OfaDevState)),
            "pinned alloc");
  if (p->sep) {
    std::vector<int2> ixy(n_foci);
    std::vector<int> count(p->uy + 1, 0), order(n_foci);
    for (int k = 0; k < n_foci; ++k) {
      ixy[k].x = (int)(std::lower_bound(xs.begin(), xs.end(), xy[2 * k]) - xs.begin());
      ixy[k].y = (int)(std::lower_bound(ys.begin(), ys.end(), xy[2 * k + 1]) - ys.begin());
      count[ixy[k].y + 1]++;
      order[k] = k;
    }
    for (int r = 0; r < p->uy; ++r) count[r + 1] += count[r];
    // the focus at each grid point (a grid point holding two foci keeps the
    // general-order T of launch_sep_t)
    std::vector<int> gridk((size_t)p->ux * p->uy, -1);
    bool grid_unique = true;
    for (int k = 0; k < n_foci; ++k) {
      int& g = gridk[(size_t)ixy[k].y * p->ux + ixy[k].x];
      if (g >= 0) grid_unique = false;
      g = k;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return ixy[a].y != ixy[b].y ? ixy[a].y < ixy[b].y : ixy[a].x < ixy[b].x;
    });
    std::vector<float2> ones(p->uy, make_float2(1.f, 0.f));
    std::vector<double> ux2(2 * (size_t)p->ux, 0.0), uy2(2 * (size_t)p->uy, 0.0);
    for (int i = 0; i < p->ux; ++i) ux2[2 * i] = xs[i];
    for (int i = 0; i < p->uy; ++i) uy2[2 * i + 1] = ys[i];
    double* dcoord = p->sep_coord;
    // stream-ordered copies; the synchronisation below keeps the host vectors alive
    // until they are consumed
    cudaError_t ce = cudaSuccess;
    auto h2d = [&](void* dst, const void* src, size_t bytes) {
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, p->stream);
    };
    h2d(dcoord, ux2.data(), ux2.size() * sizeof(double));
    h2d(dcoord + ux2.size(), uy2.data(), uy2.size() * sizeof(double));
    h2d(p->ixy, ixy.data(), ixy.size() * sizeof(int2));
    h2d(p->row_ptr, count.data(), count.size() * sizeof(int));
    h2d(p->row_foci, order.data(), order.size() * sizeof(int));
    h2d(p->ones, ones.data(), ones.size() * sizeof(float2));
    h2d(p->sep_gridk, gridk.data(), gridk.size() * sizeof(int));
    if (ce == cudaSuccess) {
      const double lf = wavelength * focal_length;
      launch_dft_rows(dcoord, nullptr, 0, p->ux, nx, pitch_x, 0.5 * (nx - 1), lf, lf * focal_length,
                      p->fxu,
                      p->stream);
      launch_dft_rows(dcoord + ux2.size(), nullptr, 1, p->uy, ny, pitch_y, 0.5 * (ny - 1), lf,
                      lf * focal_length,
                      p->fyu, p->stream);
      ce = cudaStreamSynchronize(p->stream);
    }
    OFA_TRY(ce, "separable grid set-up");
    // the three-launch separable iteration when its shared-memory staging fits
    const size_t limit = sep_smem_limit();
    p->sep_fast = grid_unique && sep_fast_shape(nx, p->uy) &&
                  sep_fwd_smem(ny, p->ux, p->uy, sm_count) <= limit &&
                  sep_inv_smem(p->ux, p->uy) <= limit && sep_prepare() == cudaSuccess;
    cudaGetLastError();
    // the persistent loop: the shape fits, and one block per SM can be resident
    if (opt.separable_loop != 0 && !p->sep_tc) {
      int grid = 0, resident = 0;
      const bool ok = p->sep_fast &&
                      sep_loop_shape(nx, ny, p->ux, p->uy, n_foci, sm_count, nullptr, &grid) &&
                      sep_loop_prepare(ny, sm_count, &resident) == cudaSuccess && resident >= 1;
      cudaGetLastError();
      if (!ok && opt.separable_loop == 1) {
        p->last_error = "the separable loop needs the fast separable kernels, K <= 2560 and "
                        "one pupil-row block per SM";
        return fail(OFA_ERR_UNSUPPORTED);
      }
      p->sep_loop = ok;
      p->sep_loop_grid = ok ? grid : 0;
    }
  }

  // Small inputs: stream-ordered copies from host vectors that live until the
  // synchronisation at the end of set-up.
  std::vector<float> tn(n_foci), ones(n_foci, 1.f);
  for (int k = 0; k < n_foci; ++k) tn[k] = (float)(tgt[k] / tsum);
  OFA_TRY(cudaMemcpyAsync(p->focus_xy, xy.data(), xy.size() * sizeof(double),
                          cudaMemcpyHostToDevice, p->stream),
          "copy foci");
  if (opt.focus_z)
    OFA_TRY(cudaMemcpyAsync(p->focus_z, zz.data(), zz.size() * sizeof(double),
                            cudaMemcpyHostToDevice, p->stream),
            "copy axial offsets");
  OFA_TRY(cudaMemcpyAsync(p->t, tn.data(), tn.size() * sizeof(float), cudaMemcpyHostToDevice,
                          p->stream),
          "copy targets");
  OFA_TRY(cudaMemcpyAsync(p->w, ones.data(), ones.size() * sizeof(float),
                          cudaMemcpyHostToDevice, p->stream),
          "init weights");

  // Amplitude: copy or default, then scale by a power of two to max in (1/2, 1].
  if (opt.amplitude) {
    OFA_TRY(cudaMemcpyAsync(p->amp, opt.amplitude, npix * sizeof(float), kind_from(opt.mem_space),
                            p->stream),
            "copy amplitude");
  } else {
    launch_default_amplitude(p->amp, nx, ny, row0, ny_total, pitch_x, pitch_y, opt.waist_frac,
                             p->stream);
  }
  // its peak, energy and validity are reduced on the device and read back with the
  // state mirror at the end of set-up; the scale by 2^-amp_exp follows on the stream
  launch_amp_stats(p->amp, npix, p->amp_part, p->amp_count, p->st, p->stream);
  launch_scale_pow2(p->amp, npix, p->st, p->stream);

  if (opt.phi0) {
    OFA_TRY(cudaMemcpyAsync(p->phi, opt.phi0, npix * sizeof(float), kind_from(opt.mem_space),
                            p->stream),
            "copy phi0");
  } else {
    launch_default_phase(p->phi, nx, ny, row0, opt.seed, p->stream);
  }

  // Kernel (a): DFT rows with FP64 phase reduction.
  const double lam_f = wavelength * focal_length;
  const double lam_f2 = lam_f * focal_length;
  launch_dft_rows(p->focus_xy, p->focus_z, 0, n_foci, nx, pitch_x, 0.5 * (nx - 1), lam_f, lam_f2,
                  p->fx,
                  p->stream);
  launch_dft_rows(p->focus_xy, p->focus_z, 1, n_foci, ny, pitch_y, 0.5 * (ny_total - 1) - row0,
                  lam_f, lam_f2, p->fy,
                  p->stream);
  if (tc) {
    launch_transpose_fy(p->fy, n_foci, ny, p->kp, p->nyp, p->fyT, p->stream);
    launch_pack_fx(p->fx, n_foci, nx, p->kp, p->nxp, 0, p->precision, p->tc.bx_hi, p->tc.bx_lo,
                   p->stream);
    launch_pack_fx(p->fx, n_foci, nx, p->kp, p->nxp, 1, p->precision, p->tc.q_hi, p->tc.q_lo,
                   p->stream);
    launch_field_planes(p->phi, p->amp, nx, ny, p->nxp, p->precision, p->tc.e_hi, p->tc.e_lo,
                        p->stream);
    OFA_TRY(prepare_precision(dev, p->precision), "setting kernel shared-memory attributes");
    choose_tiles(p, p->tc, sm_count);
    std::string err;
    const int* kc = opt.kernel_config;
    const bool forced = kc[0] | kc[1] | kc[2] | kc[3] | kc[4];
    if (forced) {
      if (!tc_config_valid(p, p->tc, kc[0], kc[1], kc[2], kc[3], kc[4])) {
        p->last_error = "kernel_config {" + std::to_string(kc[0]) + ", " + std::to_string(kc[1]) +
                        ", " + std::to_string(kc[2]) + ", " + std::to_string(kc[3]) + ", " +
                        std::to_string(kc[4]) + "} cannot run these sizes";
        return fail(OFA_ERR_UNSUPPORTED);
      }
      p->tc.fwd_bn = kc[0]; p->tc.fwd_split = kc[1]; p->tc.fwd_cg = kc[2];
      p->tc.bwd_bn = kc[3]; p->tc.bwd_cg = kc[4];
    } else if (opt.autotune) {
      if (!tc_autotune(p, p->tc, err)) {
        p->last_error = err;
        return fail(OFA_ERR_CUDA);
      }
    }
    if (!tc_encode_maps(p, p->tc, err)) {
      p->last_error = err;
      return fail(OFA_ERR_CUDA);
    }
    p->loop_mode = opt.fused_loop;
    if (opt.fused_loop != 0) {
      std::string lerr;
      const bool ok = loop_eligible(p) &&
                      loop_prepare(p, opt.loop_config[0], opt.loop_config[1], lerr);
      if (!ok && opt.fused_loop == 1) {
        p->last_error = lerr.empty() ? "the fused loop needs K <= 4096" : lerr;
        return fail(OFA_ERR_UNSUPPORTED);
      }
      cudaGetLastError();
    }
  }
  if (!tc) {
    // FP32 inverse operands, contraction contiguous: conj(Fx)^T, Fy^T (separable: Fyu^T)
    if (p->sep) {
      launch_transpose_fy(p->fyu, p->uy, ny, simt_ldk(p->uy), ny, p->simt.fyT, p->stream);
    } else {
      launch_transpose_fy(p->fx, n_foci, nx, simt_ldk(n_foci), nx, p->simt.fxT, p->stream, true);
      launch_transpose_fy(p->fy, n_foci, ny, simt_ldk(n_foci), ny, p->simt.fyT, p->stream);
    }
    launch_field_f32(p->phi, p->amp, nx, ny, p->e32, p->stream);
    if (p->sep_tc) {
      // tensor-core operands of the separable iteration: Fx_u in the forward's and the
      // inverse's block forms, and the pupil field planes
      TcOperands& t = p->tc;
      launch_pack_fx(p->fxu, p->ux, nx, t.kp, p->nxp, 0, p->precision, t.bx_hi, t.bx_lo,
                     p->stream);
      launch_pack_fx(p->fxu, p->ux, nx, t.kp, p->nxp, 1, p->precision, t.q_hi, t.q_lo,
                     p->stream);
      launch_field_planes(p->phi, p->amp, nx, ny, p->nxp, p->precision, t.e_hi, t.e_lo,
                          p->stream);
      OFA_TRY(prepare_precision(dev, p->precision), "setting kernel shared-memory attributes");
      OFA_TRY(sep_focal_u_prepare(), "setting kernel shared-memory attributes");
      choose_tiles(p, t, sm_count);   // the inverse's tile width
      t.fwd_bn = 128;
      t.fwd_cg = 1;
      t.bwd_cg = 1;
      t.fwd_split = sep_tc_split(p, t, sm_count);
      std::string err;
      if (!tc_encode_maps(p, t, err)) {
        p->last_error = err;
        return fail(OFA_ERR_CUDA);
      }
    }
  }
  launch_set_j(p->st, 0, 1, p->stream);
  launch_control(p->st, 0.0, 1, p->stream);
  OFA_TRY(cudaGetLastError(), "launching set-up kernels");
  // the iteration graphs are captured on the host while the set-up runs on the device
  if (!p->loop.ready && !p->sep_loop) {
    ofa_status gs = build_graph(p, p->chunk_iters, &p->chunk_exec);
    if (gs == OFA_OK) gs = build_graph(p, 1, &p->one_exec);
    if (gs != OFA_OK) return fail(gs);
  }
  {
    const ofa_status ss = sync_and_check(p);
    if (ss != OFA_OK) return fail(ss);
  }
  const OfaDevState& sh = *p->st_host;
  if (sh.amp_bad) {
    p->last_error = "amplitude must be finite and >= 0";
    return fail(OFA_ERR_INVALID_ARG);
  }
  if (!(sh.amp_max > 0.0)) {
    p->last_error = "amplitude is zero everywhere";
    return fail(OFA_ERR_INVALID_ARG);
  }
  p->amp_exp = sh.amp_exp;
  p->amp_energy = sh.amp_energy;
  g_fault_alloc_countdown = 0;
#undef OFA_TRY
  *out = p;
  return OFA_OK;
}

ofa_status ofa_iterate(ofa_plan* p, int n_iter, double threshold, int* iters_done, double* xi) {
  if (!p) return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "plan is NULL");
  if (n_iter < 0 || !std::isfinite(threshold))
    return ofa_fail(p, OFA_ERR_INVALID_ARG, "n_iter must be >= 0 and threshold finite");
  cudaSetDevice(p->device);
  const bool use_thr = threshold > 0.0 && threshold < 1.0;
  if (p->sep_loop) {
    // one persistent launch runs the n_iter iterations (and stops at the threshold)
    launch_control(p->st, use_thr ? threshold : 0.0, 1, p->stream);
    int j0 = -1;
    const bool need_sync = iters_done || xi;
    if (need_sync) {
      ofa_status s = sync_and_check(p);
      if (s != OFA_OK) return s;
      j0 = p->st_host->j;
    }
    cudaError_t e = launch_sep_loop(p, n_iter, use_thr ? threshold : 0.0, p->stream);
    if (e != cudaSuccess) return ofa_cuda_check(p, e, "launching the separable loop");
    if (!need_sync && !use_thr) return OFA_OK;
    ofa_status s = sync_and_check(p);
    if (s != OFA_OK) return s;
    if (iters_done) *iters_done = p->st_host->j - j0;
    if (xi) {
      enqueue_forward_current(p, p->stream);
      s = sync_and_check(p);
      if (s != OFA_OK) return s;
      *xi = p->st_host->xi;
    }
    return OFA_OK;
  }
  if (p->loop.ready) {
    // one persistent launch runs the n_iter iterations (and stops at the threshold)
    launch_control(p->st, use_thr ? threshold : 0.0, 1, p->stream);
    int j0 = -1;
    const bool need_sync = iters_done || xi;
    if (need_sync) {
      ofa_status s = sync_and_check(p);
      if (s != OFA_OK) return s;
      j0 = p->st_host->j;
    }
    cudaError_t e = launch_loop(p, n_iter, use_thr ? threshold : 0.0, p->stream);
    if (e != cudaSuccess) return ofa_cuda_check(p, e, "launching the fused loop");
    if (!need_sync && !use_thr) return OFA_OK;
    ofa_status s = sync_and_check(p);
    if (s != OFA_OK) return s;
    if (iters_done) *iters_done = p->st_host->j - j0;
    if (xi) {
      enqueue_forward_current(p, p->stream);
      s = sync_and_check(p);
      if (s != OFA_OK) return s;
      *xi = p->st_host->xi;
    }
    return OFA_OK;
  }
  if (!p->chunk_exec) {
    ofa_status s = build_graph(p, p->chunk_iters, &p->chunk_exec);
    if (s != OFA_OK) return s;
    s = build_graph(p, 1, &p->one_exec);
    if (s != OFA_OK) return s;
  }
  launch_control(p->st, use_thr ? threshold : 0.0, 1, p->stream);
  // iterations done by this call = j after - j before; read j before on the device stream
  int j0 = -1;
  const bool need_sync = use_thr || iters_done || xi;
  if (need_sync) {
    ofa_status s = sync_and_check(p);
    if (s != OFA_OK) return s;
    j0 = p->st_host->j;
  }
  int left = n_iter;
  while (left > 0) {
    cudaError_t e;
    if (left >= p->chunk_iters) {
      e = cudaGraphLaunch(p->chunk_exec, p->stream);
      left -= p->chunk_iters;
    } else {
      e = cudaGraphLaunch(p->one_exec, p->stream);
      left -= 1;
    }
    if (e != cudaSuccess) return ofa_cuda_check(p, e, "cudaGraphLaunch");
    if (use_thr && (left % p->chunk_iters == 0 || left < p->chunk_iters)) {
      ofa_status s = sync_and_check(p);
      if (s != OFA_OK) return s;
      if (p->st_host->done) break;
    }
  }
  if (!need_sync) {
    return ofa_cuda_check(p, cudaGetLastError(), "enqueueing iterations");
  }
  ofa_status s = sync_and_check(p);
  if (s != OFA_OK) return s;
  if (iters_done) *iters_done = p->st_host->j - j0;
  if (xi) {
    enqueue_forward_current(p, p->stream);
    s = sync_and_check(p);
    if (s != OFA_OK) return s;
    *xi = p->st_host->xi;
  }
  return OFA_OK;
}

ofa_status ofa_iterate_measured(ofa_plan* p, const float* measured, int mem_space,
                                double* xi_measured) {
  if (!p || !measured) return ofa_fail(p, OFA_ERR_INVALID_ARG, "NULL argument");
  if (mem_space != OFA_MEM_HOST && mem_space != OFA_MEM_DEVICE)
    return ofa_fail(p, OFA_ERR_INVALID_ARG, "unknown memory space");
  cudaSetDevice(p->device);
  if (mem_space == OFA_MEM_HOST) {
    for (int k = 0; k < p->K; ++k)
      if (!std::isfinite(measured[k]) || measured[k] < 0.f)
        return ofa_fail(p, OFA_ERR_INVALID_ARG, "measured intensities must be finite and >= 0");
  }
  cudaStream_t s = p->stream;
  cudaError_t e = cudaMemcpyAsync(p->meas, measured, (size_t)p->K * sizeof(float),
                                  kind_from(mem_space), s);
  if (e != cudaSuccess) return ofa_cuda_check(p, e, "copying measured intensities");
  launch_control(p->st, 0.0, 1, s);
  // forward (partials only), focal step on the captured intensities, inverse
  const int n_part = p->sep ? 1 : use_tc(p) ? fwd_n_part(p->nyp, p->tc) : simt_fwd_tiles(p->ny);
  sep_tc_refresh_e32(p, s);
  if (p->sep) enqueue_sep_forward(p, p->e32, s);
  else if (use_tc(p)) launch_fwd_tc(p, p->tc, nullptr, s, false);
  else
    launch_fwd_simt(p->e32, p->fx, p->fy, p->nx, p->ny, p->K, p->kp, p->part, nullptr, p->simt,
                    s);
  launch_focal_measured(p->part, n_part, p->kp, p->K, p->t, p->w, p->theta, p->c, p->hist, p->st,
                        p->weighting, p->meas, s);
  if (p->sep) {
    enqueue_sep_inverse(p, nullptr, s);
    sep_tc_refresh_planes(p, s);
  } else if (use_tc(p)) {
    launch_build_p(p->fyT, p->c, nullptr, p->nyp, p->kp, p->precision, p->tc.p_hi, p->tc.p_lo, s);
    launch_bwd_tc(p, p->tc, nullptr, s);
  } else {
    launch_bwd_simt(p->c, p->simt.fxT, p->simt.fyT, p->nx, p->ny, p->K, p->amp, p->phi, p->e32,
                    nullptr, p->simt, s);
  }
  ofa_status st = sync_and_check(p);
  if (st != OFA_OK) return st;
  if (xi_measured) *xi_measured = p->st_host->xi;
  return OFA_OK;
}

ofa_status ofa_get_phase(const ofa_plan* cp, float* phi_out, int out_mem_space) {
  ofa_plan* p = const_cast<ofa_plan*>(cp);
  if (!p || !phi_out) return ofa_fail(p, OFA_ERR_INVALID_ARG, "NULL argument");
  if (out_mem_space != OFA_MEM_HOST && out_mem_space != OFA_MEM_DEVICE)
    return ofa_fail(p, OFA_ERR_INVALID_ARG, "unknown memory space");
  cudaSetDevice(p->device);
  const size_t bytes = (size_t)p->nx * p->ny * sizeof(float);
  cudaError_t e = cudaMemcpyAsync(phi_out, p->phi, bytes,
                                  out_mem_space == OFA_MEM_HOST ? cudaMemcpyDeviceToHost
                                                                : cudaMemcpyDeviceToDevice,
                                  p->stream);
  if (e != cudaSuccess) return ofa_cuda_check(p, e, "copying phi");
  if (out_mem_space == OFA_MEM_HOST) return sync_and_check(p);
  return OFA_OK;
}

ofa_status ofa_get_stats(ofa_plan* p, ofa_stats* stats) {
  if (!p || !stats) return ofa_fail(p, OFA_ERR_INVALID_ARG, "NULL argument");
  cudaSetDevice(p->device);
  enqueue_forward_current(p, p->stream);
  ofa_status s = sync_and_check(p);
  if (s != OFA_OK) return s;
  stats->iterations = p->st_host->j;
  stats->xi = p->st_host->xi;
  stats->uniformity = p->st_host->uniformity;
  stats->sum_intensity = p->st_host->sum_i;
  stats->energy_fraction = p->st_host->energy_fraction / ((double)p->nx * p->ny);
  return OFA_OK;
}

ofa_status ofa_get_xi_history(const ofa_plan* cp, double* xi_out, int capacity, int* count) {
  ofa_plan* p = const_cast<ofa_plan*>(cp);
  if (!p || !count || capacity < 0 || (capacity > 0 && !xi_out))
    return ofa_fail(p, OFA_ERR_INVALID_ARG, "bad argument");
  cudaSetDevice(p->device);
  ofa_status s = sync_and_check(p);
  if (s != OFA_OK) return s;
  const int total = p->st_host->hist_count;
  const int kept = total < OFA_HIST_CAP ? total : OFA_HIST_CAP;
  *count = kept;
  const int n = capacity < kept ? capacity : kept;
  if (n == 0) return OFA_OK;
  std::vector<double> ring(OFA_HIST_CAP);
  cudaError_t e = cudaMemcpy(ring.data(), p->hist, sizeof(double) * OFA_HIST_CAP,
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ofa_cuda_check(p, e, "reading xi history");
  const int start = total < OFA_HIST_CAP ? 0 : total % OFA_HIST_CAP;
  for (int i = 0; i < n; ++i) xi_out[i] = ring[(start + i) % OFA_HIST_CAP];
  return OFA_OK;
}

ofa_status ofa_get_state(const ofa_plan* cp, float* phi, float* w, int* j, int mem_space) {
  ofa_plan* p = const_cast<ofa_plan*>(cp);
  if (!p) return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "plan is NULL");
  if (mem_space != OFA_MEM_HOST && mem_space != OFA_MEM_DEVICE)
    return ofa_fail(p, OFA_ERR_INVALID_ARG, "unknown memory space");
  cudaSetDevice(p->device);
  const cudaMemcpyKind kd =
      mem_space == OFA_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  cudaError_t e = cudaSuccess;
  if (phi) e = cudaMemcpyAsync(phi, p->phi, (size_t)p->nx * p->ny * 4, kd, p->stream);
  if (e == cudaSuccess && w) e = cudaMemcpyAsync(w, p->w, (size_t)p->K * 4, kd, p->stream);
  if (e != cudaSuccess) return ofa_cuda_check(p, e, "copying state");
  ofa_status s = sync_and_check(p);
  if (s != OFA_OK) return s;
  if (j) *j = p->st_host->j;
  return OFA_OK;
}

ofa_status ofa_set_state(ofa_plan* p, const float* phi, const float* w, int j, int mem_space) {
  if (!p) return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "plan is NULL");
  if (j < 0 || (mem_space != OFA_MEM_HOST && mem_space != OFA_MEM_DEVICE))
    return ofa_fail(p, OFA_ERR_INVALID_ARG, "bad argument");
  cudaSetDevice(p->device);
  const cudaMemcpyKind kd = kind_from(mem_space);
  cudaError_t e = cudaSuccess;
  if (phi) e = cudaMemcpyAsync(p->phi, phi, (size_t)p->nx * p->ny * 4, kd, p->stream);
  if (e == cudaSuccess && w) e = cudaMemcpyAsync(p->w, w, (size_t)p->K * 4, kd, p->stream);
  if (e != cudaSuccess) return ofa_cuda_check(p, e, "copying state");
  if (use_tc(p))
    launch_field_planes(p->phi, p->amp, p->nx, p->ny, p->nxp, p->precision, p->tc.e_hi,
                        p->tc.e_lo, p->stream);
  else
    launch_field_f32(p->phi, p->amp, p->nx, p->ny, p->e32, p->stream);
  sep_tc_refresh_planes(p, p->stream);
  launch_set_j(p->st, j, 1, p->stream);
  return sync_and_check(p);
}

ofa_status ofa_forward(ofa_plan* p, const float* phi, float* theta, float* intensity) {
  if (!p || !phi) return ofa_fail(p, OFA_ERR_INVALID_ARG, "NULL argument");
  cudaSetDevice(p->device);
  float2* th = theta ? reinterpret_cast<float2*>(theta) : p->theta;
  float* in = intensity ? intensity : p->inten;
  const float out_scale = ldexpf(1.f, p->amp_exp);
  if (p->sep) {
    launch_field_f32(phi, p->amp, p->nx, p->ny, p->e32_aux, p->stream);
    enqueue_sep_forward(p, p->e32_aux, p->stream);
    launch_focal(p->part, 1, p->kp, p->K, p->t, p->w, th, in, p->c, p->hist, p->st, 2,
                 p->weighting, out_scale, p->amp_energy, p->stream);
  } else if (!use_tc(p)) {
    launch_field_f32(phi, p->amp, p->nx, p->ny, p->e32_aux, p->stream);
    launch_fwd_simt(p->e32_aux, p->fx, p->fy, p->nx, p->ny, p->K, p->kp, p->part, nullptr, p->simt,
                    p->stream);
    launch_focal(p->part, simt_fwd_tiles(p->ny), p->kp, p->K, p->t, p->w, th, in, p->c, p->hist,
                 p->st, 2, p->weighting, out_scale, p->amp_energy, p->stream);
  } else {
    ofa_status s = ensure_aux(p);
    if (s != OFA_OK) return s;
    launch_field_planes(phi, p->amp, p->nx, p->ny, p->nxp, p->precision, p->tc_aux.e_hi,
                        p->tc_aux.e_lo, p->stream);
    launch_fwd_tc(p, p->tc_aux, nullptr, p->stream, false);
    launch_focal(p->part, fwd_n_part(p->nyp, p->tc), p->kp, p->K, p->t, p->w, th, in, p->c,
                 p->hist, p->st, 2, p->weighting, out_scale, p->amp_energy, p->stream);
  }
  return ofa_cuda_check(p, cudaGetLastError(), "launching forward");
}

ofa_status ofa_shard_forward(ofa_plan* p, float* theta_partial) {
  if (!p || !theta_partial) return ofa_fail(p, OFA_ERR_INVALID_ARG, "NULL argument");
  cudaSetDevice(p->device);
  // the forward at the loop's current phase (the plan's own field), output only
  float2* th = reinterpret_cast<float2*>(theta_partial);
  const float out_scale = ldexpf(1.f, p->amp_exp);
  if (p->sep) {
    enqueue_sep_forward(p, p->e32, p->stream);
    launch_focal(p->part, 1, p->kp, p->K, p->t, p->w, th, p->inten, p->c, p->hist, p->st, 2,
                 p->weighting, out_scale, p->amp_energy, p->stream);
  } else if (!use_tc(p)) {
    launch_fwd_simt(p->e32, p->fx, p->fy, p->nx, p->ny, p->K, p->kp, p->part, nullptr, p->simt,
                    p->stream);
    launch_focal(p->part, simt_fwd_tiles(p->ny), p->kp, p->K, p->t, p->w, th, p->inten, p->c,
                 p->hist, p->st, 2, p->weighting, out_scale, p->amp_energy, p->stream);
  } else {
    launch_fwd_tc(p, p->tc, nullptr, p->stream, false);
    launch_focal(p->part, fwd_n_part(p->nyp, p->tc), p->kp, p->K, p->t, p->w, th, p->inten, p->c,
                 p->hist, p->st, 2, p->weighting, out_scale, p->amp_energy, p->stream);
  }
  return ofa_cuda_check(p, cudaGetLastError(), "launching the shard forward");
}

ofa_status ofa_shard_update(ofa_plan* p, const float* theta_total) {
  if (!p || !theta_total) return ofa_fail(p, OFA_ERR_INVALID_ARG, "NULL argument");
  cudaSetDevice(p->device);
  // statistics, weight update and focused field from the summed Theta (one partial
  // row of K values), then the inverse product and projection for this shard's rows
  cudaStream_t s = p->stream;
  launch_control(p->st, 0.0, 1, s);
  launch_focal(reinterpret_cast<const float2*>(theta_total), 1, p->kp, p->K, p->t, p->w,
               p->theta, p->inten, p->c, p->hist, p->st, 0, p->weighting, 1.f, p->amp_energy, s);
  if (p->sep) {
    enqueue_sep_inverse(p, nullptr, s);
    sep_tc_refresh_planes(p, s);
  } else if (use_tc(p)) {
    launch_build_p(p->fyT, p->c, nullptr, p->nyp, p->kp, p->precision, p->tc.p_hi, p->tc.p_lo, s);
    launch_bwd_tc(p, p->tc, nullptr, s);
  } else {
    launch_bwd_simt(p->c, p->simt.fxT, p->simt.fyT, p->nx, p->ny, p->K, p->amp, p->phi, p->e32,
                    nullptr, p->simt, s);
  }
  return ofa_cuda_check(p, cudaGetLastError(), "launching the shard update");
}

ofa_status ofa_adjoint(ofa_plan* p, const float* phi, const float* theta,
                       const float* grad_intensity, float* grad_phi) {
  if (!p || !phi || !theta || !grad_intensity || !grad_phi)
    return ofa_fail(p, OFA_ERR_INVALID_ARG, "NULL argument");
  cudaSetDevice(p->device);
  launch_grad_c(reinterpret_cast<const float2*>(theta), grad_intensity, p->K, p->kp, 1.f, p->c,
                p->st, p->stream);
  const float amp_factor = ldexpf(1.f, p->amp_exp);
  if (p->sep) {
    launch_sep_t(p->c, p->fxu, p->ixy, p->row_ptr, p->row_foci, p->uy, p->nx, p->tconj,
                 p->stream);
    sep_transpose_t(p, p->stream);
    launch_grad_simt(p->ones, p->simt.fxT, p->simt.fyT, p->nx, p->ny, p->uy, phi, p->amp,
                     amp_factor, p->st, grad_phi, p->simt, p->stream);
  } else if (!use_tc(p)) {
    launch_grad_simt(p->c, p->simt.fxT, p->simt.fyT, p->nx, p->ny, p->K, phi, p->amp,
                     amp_factor, p->st, grad_phi, p->simt, p->stream);
  } else {
    launch_build_p(p->fyT, p->c, nullptr, p->nyp, p->kp, p->precision, p->tc.p_hi, p->tc.p_lo,
                   p->stream);
    launch_grad_tc(p, p->tc, phi, amp_factor, grad_phi, p->stream);
  }
  return ofa_cuda_check(p, cudaGetLastError(), "launching adjoint");
}

ofa_status ofa_loss_adjoint(ofa_plan* p, const float* phi, const float* theta, float* grad_phi,
                            float* loss_hist, int loss_capacity, const int* step) {
  if (!p || !phi || !theta || !grad_phi) return ofa_fail(p, OFA_ERR_INVALID_ARG, "NULL argument");
  if (loss_hist && loss_capacity < 1)
    return ofa_fail(p, OFA_ERR_INVALID_ARG, "loss_capacity must be >= 1 with loss_hist");
  cudaSetDevice(p->device);
  launch_loss_grad_c(reinterpret_cast<const float2*>(theta), p->t, p->K, p->kp, p->c, p->st,
                     loss_hist, loss_hist ? loss_capacity : 0, step, p->stream);
  const float amp_factor = ldexpf(1.f, p->amp_exp);
  if (p->sep) {
    launch_sep_t(p->c, p->fxu, p->ixy, p->row_ptr, p->row_foci, p->uy, p->nx, p->tconj,
                 p->stream);
    sep_transpose_t(p, p->stream);
    launch_grad_simt(p->ones, p->simt.fxT, p->simt.fyT, p->nx, p->ny, p->uy, phi, p->amp,
                     amp_factor, p->st, grad_phi, p->simt, p->stream);
  } else if (!use_tc(p)) {
    launch_grad_simt(p->c, p->simt.fxT, p->simt.fyT, p->nx, p->ny, p->K, phi, p->amp,
                     amp_factor, p->st, grad_phi, p->simt, p->stream);
  } else {
    launch_build_p(p->fyT, p->c, nullptr, p->nyp, p->kp, p->precision, p->tc.p_hi, p->tc.p_lo,
                   p->stream);
    launch_grad_tc(p, p->tc, phi, amp_factor, grad_phi, p->stream);
  }
  return ofa_cuda_check(p, cudaGetLastError(), "launching the loss adjoint");
}

ofa_status ofa_adam_step(ofa_plan* p, float* phi, const float* grad_phi, float* m, float* v,
                         int* step, float lr, float beta1, float beta2, float eps) {
  if (!p || !phi || !grad_phi || !m || !v || !step)
    return ofa_fail(p, OFA_ERR_INVALID_ARG, "NULL argument");
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f))
    return ofa_fail(p, OFA_ERR_INVALID_ARG, "Adam needs lr > 0, 0 <= betas < 1, eps > 0");
  cudaSetDevice(p->device);
  launch_adam(phi, grad_phi, m, v, step, p->st, (size_t)p->nx * p->ny, lr, beta1, beta2, eps,
              p->stream);
  return ofa_cuda_check(p, cudaGetLastError(), "launching the Adam update");
}

ofa_status ofa_profile_kernels(ofa_plan* p, int reps, double* ms_out) {
  if (!p || reps < 1 || !ms_out) return ofa_fail(p, OFA_ERR_INVALID_ARG, "bad argument");
  cudaSetDevice(p->device);
  const bool tc = use_tc(p);
  const size_t npix = (size_t)p->nx * p->ny;
  // Save the loop state (the focal kernel updates w, j and the history; the
  // inverse rewrites phi and the field planes).
  float* phi_s = nullptr;
  float* w_s = nullptr;
  OfaDevState* st_s = nullptr;
  void* e_s[2] = {nullptr, nullptr};
  const size_t e_bytes = (size_t)p->nyp * 2 * p->nxp * p->tc.elem_bytes;
  cudaError_t e = cudaMalloc(&phi_s, npix * 4);
  if (e == cudaSuccess) e = cudaMalloc(&w_s, (size_t)p->K * 4);
  if (e == cudaSuccess) e = cudaMalloc(&st_s, sizeof(OfaDevState));
  const bool planes = tc || p->sep_tc;   // operand planes to save and restore
  if (e == cudaSuccess && planes) e = cudaMalloc(&e_s[0], e_bytes);
  if (e == cudaSuccess && planes && p->tc.npass == 3) e = cudaMalloc(&e_s[1], e_bytes);
  auto cleanup = [&]() {
    dfree(phi_s);
    dfree(w_s);
    dfree(st_s);
    dfree(e_s[0]);
    dfree(e_s[1]);
  };
  if (e != cudaSuccess) {
    cleanup();
    return ofa_cuda_check(p, e, "allocating profile scratch");
  }
  cudaStream_t s = p->stream;
  cudaMemcpyAsync(phi_s, p->phi, npix * 4, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(w_s, p->w, (size_t)p->K * 4, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(st_s, p->st, sizeof(OfaDevState), cudaMemcpyDeviceToDevice, s);
  if (planes) cudaMemcpyAsync(e_s[0], p->tc.e_hi, e_bytes, cudaMemcpyDeviceToDevice, s);
  if (e_s[1]) cudaMemcpyAsync(e_s[1], p->tc.e_lo, e_bytes, cudaMemcpyDeviceToDevice, s);
  launch_control(p->st, 0.0, 1, s);

  const int n_part = p->sep ? 1 : tc ? fwd_n_part(p->nyp, p->tc) : simt_fwd_tiles(p->ny);
  auto run = [&](int which) {
    switch (which) {
      case 0:
        if (p->sep_tc) {
          launch_fwd_sep_tc(p, p->tc, nullptr, s);
          launch_sep_tc_theta(p->gt, p->tc.fwd_split, p->fyu, p->sep_gridk, p->ny, p->ux, p->uy,
                              p->K, p->part, p->w, p->sep_wprev, nullptr, s);
        } else if (p->sep) {
          enqueue_sep_forward(p, p->e32, s);
        } else if (tc) {
          launch_fwd_tc(p, p->tc, nullptr, s, p->K <= 4096);  // + fused focal step
        } else {
          launch_fwd_simt(p->e32, p->fx, p->fy, p->nx, p->ny, p->K, p->kp, p->part, nullptr,
                          p->simt, s);
        }
        break;
      case 1:
        if ((tc && p->K <= 4096) || p->sep_tc) break;  // fused into another kernel
        launch_control(p->st, 0.0, 1, s);
        launch_focal(p->part, n_part, p->kp, p->K, p->t, p->w, p->theta, p->inten, p->c, p->hist,
                     p->st, 0, p->weighting, 1.f, p->amp_energy, s);
        break;
      case 2:
        if (p->sep_tc) {
          // the focal step and U in one launch (reported here; nothing in ms_out[1])
          launch_sep_focal_u(p->part, p->t, p->sep_wprev, p->w, p->c, p->hist, p->st,
                             p->weighting, p->ixy, p->K, p->fyu, nullptr, p->ny, p->ux, p->uy,
                             p->tc.kp, p->precision, p->tc.p_hi, p->tc.p_lo, s);
        } else if (p->sep) {
          // the three-launch separable form builds T inside the inverse (reported there)
          if (!p->sep_fast)
            launch_sep_t(p->c, p->fxu, p->ixy, p->row_ptr, p->row_foci, p->uy, p->nx, p->tconj,
                         s);
        } else if (tc) launch_build_p(p->fyT, p->c, nullptr, p->nyp, p->kp, p->precision,
                                    p->tc.p_hi, p->tc.p_lo, s);
        else launch_scale_conj(p->c, p->simt.fyT, p->ny, p->K, p->simt.p32, nullptr, s);
        break;
      default:
        if (p->sep_tc) launch_bwd_tc(p, p->tc, nullptr, s);
        else if (p->sep) enqueue_sep_inverse(p, nullptr, s);
        else if (tc) launch_bwd_tc(p, p->tc, nullptr, s);
        else launch_bwd_simt_product(p->simt.fxT, p->nx, p->ny, p->K, p->amp, p->phi, p->e32,
                                     nullptr, p->simt, s);
        break;
    }
  };
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  for (int which = 0; which < 4; ++which) {
    if (which == 1 && ((tc && p->K <= 4096) || p->sep_tc)) {
      ms_out[which] = 0.0;
      continue;
    }
    run(which);  // warm-up
    cudaEventRecord(ev0, s);
    for (int r = 0; r < reps; ++r) run(which);
    cudaEventRecord(ev1, s);
    cudaEventSynchronize(ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    ms_out[which] = (double)ms / reps;
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaMemcpyAsync(p->phi, phi_s, npix * 4, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(p->w, w_s, (size_t)p->K * 4, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(p->st, st_s, sizeof(OfaDevState), cudaMemcpyDeviceToDevice, s);
  if (planes) cudaMemcpyAsync(p->tc.e_hi, e_s[0], e_bytes, cudaMemcpyDeviceToDevice, s);
  if (e_s[1]) cudaMemcpyAsync(p->tc.e_lo, e_s[1], e_bytes, cudaMemcpyDeviceToDevice, s);
  if (!tc) launch_field_f32(p->phi, p->amp, p->nx, p->ny, p->e32, s);  // field of the restored phi
  ofa_status st = sync_and_check(p);
  cleanup();
  if (st != OFA_OK) return st;
  return ofa_cuda_check(p, cudaGetLastError(), "profiling kernels");
}

ofa_status ofa_profile_loop(ofa_plan* p, int n_iter, int reps, double* ms_per_iteration,
                            double* phase_us) {
  if (!p || n_iter < 1 || reps < 1 || !ms_per_iteration)
    return ofa_fail(p, OFA_ERR_INVALID_ARG, "bad argument");
  if (!p->loop.ready) return ofa_fail(p, OFA_ERR_UNSUPPORTED, "the plan does not run the fused loop");
  cudaSetDevice(p->device);
  const size_t npix = (size_t)p->nx * p->ny;
  const size_t e_bytes = (size_t)p->nyp * 2 * p->nxp * p->tc.elem_bytes;
  float* phi_s = nullptr;
  float* w_s = nullptr;
  OfaDevState* st_s = nullptr;
  void* e_s[2] = {nullptr, nullptr};
  unsigned long long* clk = nullptr;
  cudaError_t e = cudaMalloc(&phi_s, npix * 4);
  if (e == cudaSuccess) e = cudaMalloc(&w_s, (size_t)p->K * 4);
  if (e == cudaSuccess) e = cudaMalloc(&st_s, sizeof(OfaDevState));
  if (e == cudaSuccess) e = cudaMalloc(&e_s[0], e_bytes);
  if (e == cudaSuccess && p->tc.npass == 3) e = cudaMalloc(&e_s[1], e_bytes);
  if (e == cudaSuccess && phase_us) e = cudaMalloc(&clk, 6 * sizeof(unsigned long long));
  auto cleanup = [&]() {
    dfree(clk);
    dfree(phi_s);
    dfree(w_s);
    dfree(st_s);
    dfree(e_s[0]);
    dfree(e_s[1]);
  };
  if (e != cudaSuccess) {
    cleanup();
    return ofa_cuda_check(p, e, "allocating profile scratch");
  }
  cudaStream_t s = p->stream;
  cudaMemcpyAsync(phi_s, p->phi, npix * 4, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(w_s, p->w, (size_t)p->K * 4, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(st_s, p->st, sizeof(OfaDevState), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(e_s[0], p->tc.e_hi, e_bytes, cudaMemcpyDeviceToDevice, s);
  if (e_s[1]) cudaMemcpyAsync(e_s[1], p->tc.e_lo, e_bytes, cudaMemcpyDeviceToDevice, s);
  launch_control(p->st, 0.0, 1, s);
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  e = launch_loop(p, n_iter, 0.0, s);  // warm-up
  cudaEventRecord(ev0, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_loop(p, n_iter, 0.0, s);
  cudaEventRecord(ev1, s);
  cudaEventSynchronize(ev1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  *ms_per_iteration = (double)ms / ((double)reps * n_iter);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (phase_us && e == cudaSuccess) {
    unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
    cudaMemsetAsync(clk, 0, sizeof(h), s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_loop(p, n_iter, 0.0, s, clk);
    cudaMemcpyAsync(h, clk, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (int i = 0; i < 6; ++i) phase_us[i] = (double)h[i] / 1000.0 / ((double)reps * n_iter);
  }
  cudaMemcpyAsync(p->phi, phi_s, npix * 4, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(p->w, w_s, (size_t)p->K * 4, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(p->st, st_s, sizeof(OfaDevState), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(p->tc.e_hi, e_s[0], e_bytes, cudaMemcpyDeviceToDevice, s);
  if (e_s[1]) cudaMemcpyAsync(p->tc.e_lo, e_s[1], e_bytes, cudaMemcpyDeviceToDevice, s);
  ofa_status st = sync_and_check(p);
  cleanup();
  if (st != OFA_OK) return st;
  if (e != cudaSuccess) return ofa_cuda_check(p, e, "launching the fused loop");
  return ofa_cuda_check(p, cudaGetLastError(), "profiling the fused loop");
}

// ------------------------------------------------------------------ batch
struct ofa_batch {
  std::vector<ofa_plan*> plans;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  int exec_iters = 0;
  int device = 0;
  TcBatch* tc = nullptr;  // grouped tensor-core launches (NULL: plan after plan)
  std::string last_error;
};

ofa_status ofa_batch_create(ofa_batch** out, ofa_plan* const* plans, int count, void* stream) {
  if (!out || !plans || count < 1)
    return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "bad batch argument");
  *out = nullptr;
  ofa_batch* b = new ofa_batch();
  for (int i = 0; i < count; ++i) {
    if (!plans[i] || plans[i]->device != plans[0]->device) {
      delete b;
      return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "batch plans must be non-NULL, one device");
    }
    b->plans.push_back(plans[i]);
  }
  b->device = plans[0]->device;
  cudaSetDevice(b->device);
  b->stream = static_cast<cudaStream_t>(stream);
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return ofa_fail(nullptr, OFA_ERR_CUDA, "creating batch capture stream");
  }
  // Grouped launches when every plan is on the tensor-core path with one precision
  // and its focal step fits the forward kernel's last CTA; otherwise plan after plan.
  bool grouped = true;
  for (ofa_plan* p : b->plans)
    grouped = grouped && use_tc(p) && p->precision == plans[0]->precision &&
              p->K <= 4096;
  if (grouped) {
    if (cudaDeviceSynchronize() != cudaSuccess) {
      cudaStreamDestroy(b->cap_stream);
      delete b;
      return ofa_fail(nullptr, OFA_ERR_CUDA, "synchronising before the batch set-up");
    }
    std::string err;
    if (!tc_batch_create(plans, count, b->cap_stream, &b->tc, err)) {
      cudaStreamDestroy(b->cap_stream);
      delete b;
      return ofa_fail(nullptr, OFA_ERR_CUDA, "batch set-up: " + err);
    }
    cudaStreamSynchronize(b->cap_stream);
  }
  *out = b;
  return OFA_OK;
}

ofa_status ofa_trim(void) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ofa_cuda_check(nullptr, e, "cudaGetDevice");
  void* arena = nullptr;
  OfaDevState* h = nullptr;
  cudaStream_t streams[OFA_CACHED_STREAMS];
  int n_streams = 0;
  CachedExec execs[OFA_CACHED_EXECS];
  int n_execs = 0;
  if (dev >= 0 && dev < OFA_MAX_DEVICES) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    DeviceCache& c = g_cache[dev];
    arena = c.arena;
    h = c.st_host;
    c.arena = nullptr;
    c.arena_bytes = 0;
    c.st_host = nullptr;
    n_streams = c.n_streams;
    for (int i = 0; i < n_streams; ++i) streams[i] = c.streams[i];
    c.n_streams = 0;
    n_execs = c.n_execs;
    for (int i = 0; i < n_execs; ++i) execs[i] = c.execs[i];
    c.n_execs = 0;
  }
  if (arena) e = cudaFree(arena);
  if (h) {
    const cudaError_t e2 = cudaFreeHost(h);
    if (e == cudaSuccess) e = e2;
  }
  for (int i = 0; i < n_streams; ++i) {
    const cudaError_t e2 = cudaStreamDestroy(streams[i]);
    if (e == cudaSuccess) e = e2;
  }
  for (int i = 0; i < n_execs; ++i) {
    const cudaError_t e2 = cudaGraphExecDestroy(execs[i].exec);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return ofa_cuda_check(nullptr, e, "releasing cached memory");
  return OFA_OK;
}

ofa_status ofa_selftest_bounded_wait(void) {
  OfaDevState* st = nullptr;
  cudaError_t e = cudaMalloc(&st, sizeof(OfaDevState));
  if (e == cudaSuccess) e = cudaMemset(st, 0, sizeof(OfaDevState));
  if (e == cudaSuccess) {
    launch_selftest_wait(st, nullptr);
    e = cudaGetLastError();
  }
  OfaDevState h{};
  if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(OfaDevState), cudaMemcpyDeviceToHost);
  if (st) cudaFree(st);
  if (e != cudaSuccess) return ofa_cuda_check(nullptr, e, "bounded-wait self-test");
  if (h.err & OFA_ERRBIT_TIMEOUT)
    return ofa_fail(nullptr, OFA_ERR_TIMEOUT, "a bounded device wait gave up (self-test)");
  return ofa_fail(nullptr, OFA_OK, "the self-test wait completed");
}

ofa_status ofa_batch_info(const ofa_batch* b, int* grouped, int* fwd_bn, int* inv_bn) {
  if (!b) return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "batch is NULL");
  int f = 0, i = 0;
  if (b->tc) tc_batch_config(b->tc, &f, &i);
  if (grouped) *grouped = b->tc != nullptr;
  if (fwd_bn) *fwd_bn = f;
  if (inv_bn) *inv_bn = i;
  return OFA_OK;
}

ofa_status ofa_batch_iterate(ofa_batch* b, int n_iter) {
  if (!b || n_iter < 0) return ofa_fail(nullptr, OFA_ERR_INVALID_ARG, "bad batch argument");
  cudaSetDevice(b->device);
  if (n_iter == 0) return OFA_OK;
  if (!b->exec || b->exec_iters != n_iter) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return ofa_fail(nullptr, OFA_ERR_CUDA, "batch capture");
    for (ofa_plan* p : b->plans) launch_control(p->st, 0.0, 1, b->cap_stream);
    for (int it = 0; it < n_iter; ++it) {
      if (b->tc) tc_batch_enqueue_iteration(b->tc, b->cap_stream);
      else
        for (ofa_plan* p : b->plans)
          if (!p->sep_loop && !p->loop.ready) enqueue_iteration(p, b->cap_stream);
    }
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (e != cudaSuccess) return ofa_fail(nullptr, OFA_ERR_CUDA, "batch capture end");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return ofa_fail(nullptr, OFA_ERR_CUDA, "batch graph instantiate");
    b->exec_iters = n_iter;
  }
  // The plans' own streams must see the batch's work in order.
  cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
  if (e != cudaSuccess) return ofa_fail(nullptr, OFA_ERR_CUDA, "batch graph launch");
  // plans whose own iterations run as one persistent launch run it here too, so that a
  // batch of plans run one after another gives each plan's own results bit for bit
  if (!b->tc)
    for (ofa_plan* p : b->plans) {
      if (p->sep_loop) e = launch_sep_loop(p, n_iter, 0.0, b->stream);
      else if (p->loop.ready) e = launch_loop(p, n_iter, 0.0, b->stream);
      if (e != cudaSuccess) return ofa_fail(nullptr, OFA_ERR_CUDA, "batch persistent launch");
    }
  return OFA_OK;
}

ofa_status ofa_batch_destroy(ofa_batch* b) {
  if (!b) return OFA_OK;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  tc_batch_destroy(b->tc);
  delete b;
  return OFA_OK;
}

}  // extern "C"
