/*
 * ofa.h -- C ABI of the GB300 GSW-MTP optical-focus-array library.
 *
 * The library computes phase-only holograms (CGHs) for arbitrary optical
 * focus arrays with the method of Liu et al., "Fast generation of arbitrary
 * optical focus array" (arXiv 2206.12661):
 *   - far-field propagation between the SLM pupil and the focal plane written
 *     as a matrix triple product with arbitrarily sampled DFT matrices
 *     (Eq. 1, Eq. 2), evaluated only at the foci (zero elements removed);
 *   - the weighted Gerchberg-Saxton loop with the paper's generalized
 *     weighting update (Algorithm 1).
 *
 * Conventions shared by every call
 *   - Pupil arrays are row-major [ny][nx] float32 (rows along y).  Pupil
 *     sample positions are centred: u_m = (m - (nx-1)/2) * pitch_x, likewise v_n.
 *   - Focus positions are float64 metres in the focal plane, [K][2] = (x, y).
 *     Spatial frequency of pupil position u is u / (wavelength * focal_length).
 *   - Complex vectors are interleaved float32 pairs (re, im).
 *   - Every call returns an ofa_status; no C++ exception crosses the ABI.
 *     Device errors raised by asynchronous work surface at the next call
 *     that synchronises; a plan stays destroyable after any error.
 *   - A plan is bound to one CUDA stream and one device (the device current
 *     at creation).  Calls on one plan are not thread-safe; distinct plans
 *     are independent.
 *   - "device" pointers are CUDA device (or managed) addresses on the plan's
 *     device; "host" pointers are ordinary host memory.  Inputs are deep
 *     copied: the library never keeps a caller's pointer after a call returns.
 */
#ifndef OFA_H_
#define OFA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ofa_plan ofa_plan;
typedef struct ofa_batch ofa_batch;

typedef enum ofa_status {
  OFA_OK = 0,
  OFA_ERR_INVALID_ARG = 1,   /* null pointer, non-positive size, non-finite value */
  OFA_ERR_OUT_OF_RANGE = 2,  /* focus outside the alias-free field |x| < lambda f / (2 p) */
  OFA_ERR_CUDA = 3,          /* a CUDA runtime/driver call failed (see ofa_last_error) */
  OFA_ERR_OOM = 4,           /* device or host allocation failed */
  OFA_ERR_NUMERIC = 5,       /* sum of focus intensities is zero or not finite */
  OFA_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  OFA_ERR_UNSUPPORTED = 7    /* option not available on this device or for these sizes */
} ofa_status;

/* Arithmetic of the two matrix products of the loop.  Every form accumulates
 * in FP32; the DFT phase arguments are always reduced modulo one turn before the
 * FP32 sincos (exactly, in 64-bit fixed point, for a plan's DFT rows). */
typedef enum ofa_precision {
  OFA_PREC_FP32 = 0,    /* FP32 FMA on the CUDA cores                              */
  OFA_PREC_TF32 = 1,    /* tensor cores, TF32 operands, one product                */
  OFA_PREC_BF16 = 2,    /* tensor cores, BF16 operands, one product                */
  OFA_PREC_BF16X3 = 3,  /* tensor cores, BF16 hi+lo split, three products          */
  OFA_PREC_F16X3 = 4    /* tensor cores, FP16 hi+lo split with power-of-two
                           operand scaling, three products (FP32-level accuracy) */
} ofa_precision;

typedef enum ofa_mem_space { OFA_MEM_HOST = 0, OFA_MEM_DEVICE = 1 } ofa_mem_space;

typedef struct ofa_options {
  int precision;             /* ofa_precision; default OFA_PREC_F16X3 */
  uint64_t seed;             /* seed of the default initial phase; default 0 */
  void* cuda_stream;         /* cudaStream_t the plan runs on; NULL = a non-blocking stream the
                                plan creates and owns */
  const float* amplitude;    /* [ny][nx] pupil amplitude A >= 0, or NULL for the default
                                Gaussian exp(-(u^2/wx^2 + v^2/wy^2)), w = waist_frac * n * p.
                                Checked on the device: a negative, infinite or NaN value, or
                                A = 0 everywhere, fails creation with OFA_ERR_INVALID_ARG.
                                The plan stores A 2^-e, the power of two e putting max A 2^-e
                                in (1/2, 1], so amplitudes that differ by a power of two give
                                the same phases bit for bit. */
  double waist_frac;         /* default 0.4 */
  const float* phi0;         /* [ny][nx] initial guess phi_0 (radians), or NULL for
                                2*pi*(splitmix64 stream of seed >> 11)/2^53 - pi per pixel */
  int mem_space;             /* ofa_mem_space of focus_xy, target, amplitude and phi0 */
  int weighting;             /* 1 = generalized weighting of Algorithm 1 (default),
                                0 = plain GS (w stays 1) */
  int autotune;              /* tensor-core forms: 1 = time the candidate tile widths,
                                split-K factors and CTA groups (single SMs or 2-SM pairs)
                                of both products at creation and keep the fastest
                                (default; results are cached per device, size and
                                precision for the process), 0 = a static cost model */
  const double* focus_z;     /* [K] axial offsets z_k (m) of the foci from the focal plane
                                (a 3D array), or NULL for z = 0.  Focus k's rows then carry
                                the defocus phase of the pupil function, a Fresnel (paraxial)
                                lens term: Fx[k][m] = exp(-i 2 pi (x_k u_m / (lambda f) +
                                z_k u_m^2 / (2 lambda f^2))), Fy likewise with v_n; each
                                |z_k| < f, and |x_k| + |z_k| u_max / f must stay inside the
                                alias-free field (u_max = (nx - 1) pitch_x / 2; same in y),
                                else OFA_ERR_OUT_OF_RANGE.  In mem_space; default NULL */
  int separable;             /* separable grid form: with foci on the grid of their U_x
                                distinct x and U_y distinct y values (the paper's regular
                                arrays), Theta on that grid is Fy_u E Fx_u^T (Eq. 2 through
                                the distinct coordinates) and the inverse factors the same
                                way, nx ny (U_x + U_y) complex products per iteration instead
                                of 2 nx ny K; these run in FP32 on the CUDA cores whatever
                                the precision.  -1 = when the work shrinks by more than
                                20x for the tensor-core forms, 2x for FP32 (default),
                                0 = never, 1 = always (OFA_ERR_UNSUPPORTED with focus_z) */
  int kernel_config[5];      /* tensor-core forms: a fixed kernel configuration instead of
                                the autotuner's choice, {forward tile width (128 or 256
                                accumulator columns), forward split-K factor (1, 2 or 4),
                                forward CTA group (1, or 2 for 2-SM pairs), inverse tile
                                width (128 or 256), inverse CTA group (1 or 2)}.  All zero
                                = chosen at creation (default).  A configuration these
                                sizes cannot run (split-K beyond the contraction's
                                k-blocks, 2-SM pairs over an odd number of 128-row tiles)
                                -> OFA_ERR_UNSUPPORTED.  Ignored by the FP32 and separable
                                forms. */
  int fused_loop;            /* tensor-core forms with K <= 4096: run each ofa_iterate call as
                                one persistent cooperative launch that keeps every CTA
                                resident and synchronises the grid between the forward
                                product, the focal step and the inverse product (no serial
                                focal tail, no separate operand-build launch).  0 = never:
                                one launch per product, replayed from CUDA graphs (default;
                                measured faster on GB300), 1 = always (OFA_ERR_UNSUPPORTED
                                if it cannot run), -1 = whenever the device can co-schedule
                                it */
  int loop_config[2];        /* fused loop: {CTA group (1, or 2 for 2-SM pairs), forward split
                                of the contraction (1..4)}; zeros = chosen at creation */
  int shard_row0;
  int shard_ny_total;        /* row shard (see ofa_shard_forward): this plan holds pupil rows
                                [shard_row0, shard_row0 + ny) of a pupil of shard_ny_total rows;
                                pupil row n sits at v = (shard_row0 + n - (shard_ny_total - 1)/2)
                                pitch_y, and the default amplitude and phase are that pupil's
                                rows.  Both 0 = the whole pupil (default).  Not with the
                                separable form. */
  int separable_loop;        /* separable form with K <= 512 foci: run each ofa_iterate call as
                                one persistent cooperative launch (every block keeps its
                                constant operands resident, computes the focal step itself
                                and meets the others at grid barriers between the forward
                                product, the partial-Theta sums and the inverse product).
                                -1 = whenever the grid, its shared memory and the device
                                allow it (default), 0 = never (two or three launches per
                                iteration from CUDA graphs), 1 = always (OFA_ERR_UNSUPPORTED
                                if it cannot run).  ofa_plan_config reports it as the fused
                                loop. */
  int separable_tc;          /* separable form with a tensor-core precision, U_x, U_y <= 128,
                                K <= 4096 and at most one focus per grid point: run the
                                iteration's products on the tensor cores in the plan's
                                precision -- G = E Fx_u^T per contraction part, Theta from G,
                                the focal step with U = conj(Fy_u)^T C, then the inverse
                                E' = U conj(Fx_u) --
                                instead of FP32 on the CUDA cores (the persistent loop is
                                then not used).  -1 = when U_x + U_y > 48 (default), 0 = never,
                                1 = always (OFA_ERR_UNSUPPORTED if it cannot run).  Statistics,
                                ofa_forward and the gradient entry points keep the FP32
                                products.  ofa_plan_config reports its tile configuration. */
} ofa_options;

typedef struct ofa_stats {
  int iterations;            /* completed iterations j (forward + update + inverse) */
  double xi;                 /* intensity accuracy of the latest forward (Algorithm 1) */
  double uniformity;         /* 1 - (max r - min r)/(max r + min r), r_k = Ihat_k / t_k */
  double sum_intensity;      /* sum_k |Theta_k|^2 of the latest forward (plan scale) */
  double energy_fraction;    /* sum_k |Theta_k|^2 / (nx * ny * sum A^2): share of the pupil
                                energy landing on the foci (exact Parseval share when the
                                foci sit on distinct points of the pupil's DFT grid) */
} ofa_stats;

/* Fill *opt with the defaults listed above.  Host only; never fails for non-NULL opt. */
ofa_status ofa_options_default(ofa_options* opt);

/*
 * ofa_plan_create -- problem statement of Algorithm 1 (Input) with the system
 * parameters of Table 1.
 *   nx, ny                 pupil (SLM) samples, >= 1
 *   pitch_x, pitch_y       pupil sample pitch (m), > 0
 *   wavelength, focal_length  (m), > 0
 *   n_foci                 K >= 1
 *   focus_xy               [K][2] float64 focus positions (m); each must lie in the
 *                          alias-free field |x| < lambda f / (2 pitch_x), same in y
 *                          (sampling conditions of Eq. 2 still hold), else
 *                          OFA_ERR_OUT_OF_RANGE
 *   target_intensity       [K] float32 target intensities I~ >= 0 (any scale; the
 *                          loop uses I~ / sum I~), sum > 0
 *   opt                    NULL = defaults
 * Builds the DFT rows Fx[k][m] = exp(-i 2 pi x_k u_m / (lambda f)) and Fy likewise
 * (phase arguments reduced modulo one turn exactly, in 64-bit fixed point, before the
 * FP32 sincos), sets E_0 = A exp(i phi_0), w_0 = 1, j = 0.
 * The plan owns every device buffer it allocates.  *out is NULL on failure.
 */
ofa_status ofa_plan_create(ofa_plan** out, int nx, int ny, double pitch_x, double pitch_y,
                           double wavelength, double focal_length, int n_foci,
                           const double* focus_xy, const float* target_intensity,
                           const ofa_options* opt);

/*
 * ofa_iterate -- run n_iter iterations of Algorithm 1: forward MTP at the foci,
 * I = |Theta|^2, intensity accuracy xi, generalized weight update
 * w_j = w_{j-1} sqrt(I~/I), focused field w_j sqrt(I~) exp(i arg Theta),
 * inverse MTP (adjoint of Eq. 2), phi = arg(E), E = A exp(i phi).
 *   threshold   stop before the update once xi > threshold (the loop's break);
 *               threshold <= 0 or >= 1 disables the test and runs exactly n_iter.
 *   iters_done  (nullable, host) iterations completed by this call
 *   xi          (nullable, host) xi of one extra forward at the final phase.
 * With both outputs NULL and the threshold disabled the call only enqueues work
 * on the plan's stream and returns without synchronising.
 */
ofa_status ofa_iterate(ofa_plan* plan, int n_iter, double threshold, int* iters_done, double* xi);

/*
 * ofa_iterate_measured -- one iteration in the camera-in-the-loop mode of the
 * paper's experiments (Results and discussion section): once the intensity accuracy has passed a threshold
 * (0.95 there), the calculated focus intensities are replaced by captured ones in
 * the weight update, w_j = w_{j-1} sqrt(I~ / I_meas) at unit sums; the focused field
 * keeps the phase of the calculated Theta (a camera records intensities only).
 *   measured     [K] float32 captured focus intensities >= 0, any common scale, in
 *                mem_space (host values are checked: non-finite or negative ->
 *                OFA_ERR_INVALID_ARG)
 *   xi_measured  (nullable, host) intensity accuracy of the captured intensities
 * Runs forward, update and inverse once (not graph-captured: each call follows a
 * capture) and synchronises.  The caller decides when to switch to this mode and
 * captures the OFA of the current phase (ofa_get_phase) between calls.
 */
ofa_status ofa_iterate_measured(ofa_plan* plan, const float* measured, int mem_space,
                                double* xi_measured);

/* Copy the current CGH phi [ny][nx] (radians in (-pi, pi]) to phi_out, which lives in
 * out_mem_space.  Synchronises the plan's stream for host output. */
ofa_status ofa_get_phase(const ofa_plan* plan, float* phi_out, int out_mem_space);

/* Release every resource of the plan.  NULL-safe.  The plan's device buffers live
 * in one allocation; the library keeps the last one released on each device (the
 * larger, if it already holds one), the pinned state mirror, up to eight idle streams
 * and up to eight iteration-graph executables for the next plan of similar size to
 * reuse, so a create/destroy loop allocates once and refreshes graph executables
 * instead of instantiating them.  ofa_trim frees what is kept. */
ofa_status ofa_destroy(ofa_plan* plan);

/* Free the device memory, pinned host memory, streams and graph executables that
 * destroyed plans left for reuse on the current device (at most one plan arena, one
 * state mirror, eight streams and eight executables).  Plans still alive are not
 * affected.  OFA_OK, or OFA_ERR_CUDA if a free fails. */
ofa_status ofa_trim(void);

/* Statistics of one forward at the current phase (runs that forward; host output). */
ofa_status ofa_get_stats(ofa_plan* plan, ofa_stats* stats);

/* xi of the forward at the start of each iteration since creation (or the last
 * set_state), oldest first: copies min(capacity, count) values, *count = number kept.
 * The plan keeps the most recent 65536. */
ofa_status ofa_get_xi_history(const ofa_plan* plan, double* xi_out, int capacity, int* count);

/* Loop state (phi [ny][nx], w [K], j) -- checkpoint / resume.  Pointers live in
 * mem_space; any of phi / w may be NULL to leave that part untouched (set) or
 * unread (get).  Resuming from a saved state reproduces the uninterrupted run
 * bit for bit on the same device and precision. */
ofa_status ofa_get_state(const ofa_plan* plan, float* phi, float* w, int* j, int mem_space);
ofa_status ofa_set_state(ofa_plan* plan, const float* phi, const float* w, int j, int mem_space);

/*
 * ofa_forward -- Eq. 2 at the foci for a given phase, without touching the loop
 * state: theta = P_MTP(A exp(i phi)), intensity = |theta|^2.
 *   phi        device [ny][nx]
 *   theta      device [K] complex (nullable)
 *   intensity  device [K] (nullable)
 * Enqueued on the plan's stream; no synchronisation.
 */
ofa_status ofa_forward(ofa_plan* plan, const float* phi, float* theta, float* intensity);

/*
 * ofa_adjoint -- gradient of a loss L(I) of the focus intensities with respect to
 * the phase, given g = dL/dI (device [K]) and the theta returned by ofa_forward
 * for the same phi:  dL/dphi = 2 Im(conj(E) B),  B = P_MTP^H(g * theta),
 * E = A exp(i phi).  grad_phi is device [ny][nx].  Uses the same adjoint product
 * as the loop's inverse propagation.  Enqueued on the plan's stream.
 */
ofa_status ofa_adjoint(ofa_plan* plan, const float* phi, const float* theta,
                       const float* grad_intensity, float* grad_phi);

/*
 * Row shards -- one hologram split by pupil rows over several plans (devices or ranks).
 * Eq. 2 separates over the pupil rows: Theta_k = sum over the shards of
 * sum_{n in shard} Fy[k,n] sum_m E[n,m] Fx[k,m].  So each shard (a plan created with
 * ofa_options.shard_row0 / shard_ny_total) computes its partial Theta, the partials are
 * summed over the shards (an all-reduce of K complex values), and each shard runs the
 * generalized weighting update on the sum -- identically, so every shard keeps the same
 * weights -- and the inverse product for its own rows:
 *   ofa_shard_forward  theta_partial (device [K] complex, the plan's amplitude units) =
 *                      Eq. 2 at the foci over this shard's rows at its current phase
 *   ofa_shard_update   theta_total (device [K] complex, the sum of all shards' partials):
 *                      intensities, xi (recorded in the plan's history), w <- w
 *                      sqrt(I~/I), focused field, inverse product and phi = arg for this
 *                      shard's rows; j advances by one
 * Both enqueue on the plan's stream.  The caller sums the partials in a fixed order to
 * keep runs reproducible.  Threshold stops are the caller's (compare xi across calls).
 */
ofa_status ofa_shard_forward(ofa_plan* plan, float* theta_partial);
ofa_status ofa_shard_update(ofa_plan* plan, const float* theta_total);

/*
 * ofa_loss_adjoint -- the intensity loss of the differentiable form and its gradient,
 * all in the library: from the theta that ofa_forward returned for phi,
 *   L = sum_k (I_k / S - t_k)^2,  I = |theta|^2,  S = sum I,  t = I~ / sum I~,
 *   g_k = dL/dI_k = (2 / S) [(I_k / S - t_k) - sum_j (I_j / S - t_j) I_j / S],
 * and grad_phi = dL/dphi = 2 Im(conj(E) B), B = P_MTP^H(g * theta) (the adjoint product
 * of ofa_adjoint).  S and the sums are reduced in FP64.
 *   phi, theta   device [ny][nx], [K] complex (as for ofa_adjoint)
 *   grad_phi     device [ny][nx] output
 *   loss_hist    device float array of loss_capacity (>= 1) values (nullable):
 *                loss_hist[*step] = L (or [0] if step is NULL); an index outside
 *                [0, loss_capacity) is not written
 *   step         device int (nullable), e.g. the counter of ofa_adam_step
 * Enqueued on the plan's stream.  Buffers the caller initialises on another stream must
 * be ready before the call (the library orders nothing across streams).  (The loss is
 * this library's reading of the paper's intensity-precision goal; the paper itself
 * optimises by GSW, not by gradients.)
 */
ofa_status ofa_loss_adjoint(ofa_plan* plan, const float* phi, const float* theta,
                            float* grad_phi, float* loss_hist, int loss_capacity,
                            const int* step);

/*
 * ofa_adam_step -- one Adam update of the phase (Kingma and Ba; the bias-corrected form
 * with torch's order of operations): t = *step + 1, m <- b1 m + (1 - b1) g,
 * v <- b2 v + (1 - b2) g^2, phi <- phi - lr / (1 - b1^t) m / (sqrt(v) / sqrt(1 - b2^t) + eps),
 * then *step = t.  phi, grad_phi, m, v are device [ny][nx] float32 (m and v zero at the
 * start), step a device int (0 at the start).  lr > 0, 0 <= b1, b2 < 1, eps > 0, else
 * OFA_ERR_INVALID_ARG.  Enqueued on the plan's stream; the step counter lives on the
 * device so that a captured CUDA graph of forward, loss adjoint and update replays.
 */
ofa_status ofa_adam_step(ofa_plan* plan, float* phi, const float* grad_phi, float* m, float* v,
                         int* step, float lr, float beta1, float beta2, float eps);

/*
 * ofa_profile_kernels -- measurement aid: average device time (ms) of each kernel
 * of one loop iteration, each launched `reps` (>= 1) times back to back on the
 * plan's stream between CUDA events, after one untimed launch:
 *   ms_out[0] forward product (+ per-focus dot; in the tensor-core forms also the
 *   focal statistics and weight update, which run in its last CTA), ms_out[1] focal
 *   statistics and weight update as a separate kernel (0 for the tensor-core forms),
 *   ms_out[2] inverse left-operand build (P = conj(Fy)^T diag(c): the split operand
 *   planes of the tensor-core forms, the FP32 conj(Fy)^T c of OFA_PREC_FP32; the
 *   separable form's first inverse product), ms_out[3] inverse product (+ phase
 *   projection).  The separable form on the tensor cores reports its forward product
 *   with the Theta sums in ms_out[0] and its focal step with U in ms_out[2] (0 in
 *   ms_out[1]).
 * The loop state (phi, w, j, xi history) is saved before and restored after, so
 * the call does not change the result of later iterations.  Synchronises.
 */
ofa_status ofa_profile_kernels(ofa_plan* plan, int reps, double* ms_out);

/*
 * ofa_profile_loop -- measurement aid for the fused loop (ofa_options.fused_loop):
 * average device time (ms) of one iteration, from `reps` (>= 1) launches of n_iter
 * (>= 1) iterations each, back to back on the plan's stream between CUDA events after
 * one untimed launch.  phase_us (nullable, host [6]) receives the average microseconds
 * per iteration that the first CTA spends in each phase, from %globaltimer stamps of a
 * separate set of launches: forward products and their epilogues, wait at the barrier
 * after the forward, focal step, operand build, wait at the barrier after the operand
 * build, inverse products and their epilogues.  The loop state is saved before and
 * restored after.  OFA_ERR_UNSUPPORTED if the plan does not run the fused loop.
 * Synchronises.
 */
ofa_status ofa_profile_loop(ofa_plan* plan, int n_iter, int reps, double* ms_per_iteration,
                            double* phase_us);

/* Kernel configuration of a plan (host output, 12 ints), in the order of
 * ofa_options.kernel_config followed by derived values: forward tile width
 * (accumulator columns), forward split-K factor, forward CTA group (1, or 2 for 2-SM MMA
 * pairs of 256 accumulator rows), inverse tile width, inverse CTA group, 1 if the focal
 * step runs in the forward kernel's last CTA, forward and inverse operand row width per
 * pipeline stage (bytes of K); then the fused loop: 1 if ofa_iterate runs it, its CTA
 * group, its forward split and its CTAs per launch.  The FP32 and separable forms report
 * zeros, except the separable form on the tensor cores (ofa_options.separable_tc), which
 * reports its tiles, and the separable persistent loop, reported as the fused loop. */
ofa_status ofa_plan_config(const ofa_plan* plan, int* config_out);

/* Form of a plan: *separable = 1 with the U_x and U_y distinct focus coordinates it
 * factors through (see ofa_options.separable), else 0 and zeros.  Outputs nullable. */
ofa_status ofa_plan_form(const ofa_plan* plan, int* separable, int* ux, int* uy);

/* Problem sizes of a plan (any output may be NULL). */
ofa_status ofa_plan_info(const ofa_plan* plan, int* nx, int* ny, int* n_foci, int* precision);

/*
 * Batched holograms: many independent problems of uneven pupil size and focus
 * count advanced together (the paper optimises one hologram at a time; batching is
 * a calling convention over the same loop).  When every plan uses one tensor-core
 * precision and has at most 4096 foci, each iteration of all plans is three
 * grouped launches (forward product with the per-plan focal step fused, inverse
 * operand build, inverse product), each covering the tiles of every plan, largest
 * problems first, with the tile widths timed on this batch at creation; otherwise
 * the plans' own iterations run one after another.  n iterations are one CUDA
 * graph launch on cuda_stream.
 *   plans        host array of count (>= 1) plan handles on one device; the plans
 *                keep their own buffers and state and must outlive the batch
 *   cuda_stream  cudaStream_t the batch's iterations are enqueued on
 * ofa_batch_create synchronises the device (the grouped set-up times candidate
 * kernels); ofa_batch_iterate only enqueues.  A plan must not be iterated on its
 * own while a batch iteration of it is in flight.
 */
ofa_status ofa_batch_create(ofa_batch** out, ofa_plan* const* plans, int count, void* cuda_stream);
ofa_status ofa_batch_iterate(ofa_batch* batch, int n_iter);
ofa_status ofa_batch_destroy(ofa_batch* batch);
/* 1 in *grouped when the batch runs grouped launches (then the forward and inverse
 * tile widths), else 0 and zeros.  Any output may be NULL. */
ofa_status ofa_batch_info(const ofa_batch* batch, int* grouped, int* fwd_bn, int* inv_bn);

/*
 * ofa_forward_noalloc -- the focal field at the foci for callers that cannot
 * allocate device memory: a real-time loop refreshing an SLM hologram that must
 * not pay for (or fail in) cudaMalloc once it runs, or an application whose
 * device memory is all reserved by a framework allocator.  It needs no plan:
 * theta_k = sum over the pupil of A exp(i phi) exp(-i 2 pi (x_k u + y_k v)/(lambda f)),
 * the same quantity as ofa_forward, computed in FP32 with the DFT phase arguments
 * reduced in FP64.  (The paper has no counterpart; this is a calling convention.)
 *   nx, ny, pitches, wavelength, focal_length, n_foci   as for ofa_plan_create;
 *                          ny <= 2048, n_foci <= 8192, nx <= 32768, else
 *                          OFA_ERR_INVALID_ARG (the limits of the built-in scratch)
 *   focus_xy               device [K][2] float64 (m); foci are not range-checked
 *   phi, amplitude         device [ny][nx] float32
 *   theta                  device [K] complex output (nullable)
 *   intensity              device [K] output |theta|^2 (nullable; not both NULL)
 *   cuda_stream            cudaStream_t the work is enqueued on (NULL = legacy stream)
 * Allocates nothing: its scratch is a 2 MiB static device array that every GPU
 * loading the library holds until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  After a device reset the next call sees the new
 * context and looks the address up again (again outside any capture).  All calls
 * share the array, so calls that overlap on the GPU race and must be serialised by
 * the caller.  A CUDA error left pending by earlier work is returned as
 * OFA_ERR_CUDA (and cleared) before anything is launched.  Enqueues only; no
 * synchronisation.
 */
ofa_status ofa_forward_noalloc(int nx, int ny, double pitch_x, double pitch_y,
                               double wavelength, double focal_length, int n_foci,
                               const double* focus_xy, const float* phi,
                               const float* amplitude, float* theta, float* intensity,
                               void* cuda_stream);

/*
 * ofa_selftest_bounded_wait -- diagnostic of failure detection (the paper has no
 * counterpart).  Every wait of the tensor-core kernels (on TMA data, a free stage,
 * the accumulator) gives up after about one second, records the fact in the plan's
 * device state and makes the next synchronising call return OFA_ERR_TIMEOUT instead
 * of hanging.  This call runs one such wait on a barrier that nothing signals and
 * returns what a plan would: OFA_ERR_TIMEOUT when the wait gave up as designed (the
 * expected result; ofa_last_error(NULL) says so), OFA_OK if it did not give up,
 * OFA_ERR_CUDA on a CUDA failure.  Takes about one second; synchronises the current
 * device.  Plan creation honours OFA_FAULT_ALLOC=N in the environment: the N-th
 * device allocation of that call fails as out of memory (OFA_ERR_OOM, everything
 * already allocated is freed), for testing the error paths.
 */
ofa_status ofa_selftest_bounded_wait(void);

/* Host-only helpers (no GPU needed). */

/* Zero-padded FFT size of the conventional IFTA along one axis, Eq. 3:
 * M = M0 lambda / (2 NA dd) with NA = M0 pitch / (2 f), i.e. ceil(lambda f / (pitch dd))
 * for focal-plane sampling interval dd (m).  (Table 1 gives 4551.) */
ofa_status ofa_fft_equivalent_size(int m0, double pitch, double wavelength,
                                   double focal_length, double focal_sampling, int* m_out);

/* Foci per axis that fit the alias-free field lambda f / pitch at spacing gap (m):
 * floor(lambda f / (pitch gap)).  (Table 1 with a 20-camera-pixel gap gives 227.) */
ofa_status ofa_max_foci_per_axis(double pitch, double wavelength, double focal_length,
                                 double gap, int* count_out);

/* Validate focus positions against the alias-free field, exactly as
 * ofa_plan_create does: OFA_OK, OFA_ERR_OUT_OF_RANGE (first offender in
 * *bad_index, nullable) or OFA_ERR_INVALID_ARG.  Host pointers. */
ofa_status ofa_check_foci(int n_foci, const double* focus_xy, double pitch_x, double pitch_y,
                          double wavelength, double focal_length, int* bad_index);

const char* ofa_status_string(ofa_status status);
/* Message of the last failure on this plan (or of the last failed create/host call
 * on this thread when plan is NULL).  Valid until the next call on the same plan. */
const char* ofa_last_error(const ofa_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* OFA_H_ */
