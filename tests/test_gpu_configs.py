"""Every tensor-core kernel configuration, and one step at full size, against the oracle.

The autotuner picks, per device and shape, a forward configuration (tile width 128 or
256 accumulator columns, split-K 1, 2 or 4, single CTAs or 2-SM pairs) and an inverse
configuration (tile width, CTA group) for the per-product kernels.  Plans here force
each configuration through ofa_options.kernel_config (with the fused loop off, so the
iteration runs those kernels), so every candidate the autotuner can choose is checked:
forward amplitudes from the oracle's iterate, and one iteration of Algorithm 1 from
that iterate (new weights and new phase).  The fused loop kernel (one persistent
launch per ofa_iterate call) is checked the same way in each of its configurations
(CTA group 1 or 2, forward split 1, 2 or 4).

Tolerances (readings of the 1e-5 focus-amplitude bar, per precision form):
  amplitudes   relative L2 over the foci AND max over the foci of | |Theta_gpu| -
               |Theta_ref| | / max |Theta_ref|, both within the form's amplitude
               tolerance;
  weights      2x: w_k = w_{k-1} sqrt(t_k / Ihat_k) carries the relative amplitude
               error of focus k once, plus half the relative error of sum I;
  phase        3x, weighted by |E'|: c_k carries the weight error and the phase error
               of Theta_k (each about the amplitude tolerance), and the inverse
               product adds its own rounding, bounded by the same tolerance; the DFT
               rows of well-separated foci are nearly orthogonal, so the inverse keeps
               relative L2 errors.
"""
import functools
import math

import numpy as np
import pytest

import oracle as O
from paper_2206_12661_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AMP_TOL = {"fp32": 1e-5, "f16x3": 1e-5, "bf16x3": 1e-5, "tf32": 2e-3, "bf16": 1e-2}
W_FACTOR, PHASE_FACTOR = 2.0, 3.0

FWD = [(bn, split, cg) for bn in (128, 256) for split in (1, 2, 4) for cg in (1, 2)]
INV = [(bn, cg) for bn in (128, 256) for cg in (1, 2)]
# configuration i: forward FWD[i] with inverse INV[i % 4] (covers every candidate of both)
CONFIGS = [FWD[i] + INV[i % len(INV)] for i in range(len(FWD))]


def cfg_id(c):
    return "f{}s{}g{}_i{}g{}".format(*c)


def ragged(nx=333, ny=250, K=300, seed=21):
    rng = np.random.default_rng(seed)
    half = 532e-9 * 0.2 / (2 * 8e-6)
    xy = rng.uniform(-0.9 * half, 0.9 * half, (K, 2))
    t = rng.uniform(0.5, 1.0, K).astype(np.float32)
    return I.Workload(f"ragged{nx}x{ny}_{K}", nx, ny, 8e-6, 8e-6, 532e-9, 0.2, xy, t,
                      I.gaussian_amplitude(nx, ny), I.uniform_phase(rng, nx, ny), 3)


def ragged_grid(nx=333, ny=250, cols=13, rows=41, seed=23):
    """A regular cols x rows grid on a ragged pupil (row and column padding of every
    operand plane), targets U[0.5, 1]."""
    rng = np.random.default_rng(seed)
    half = 532e-9 * 0.2 / (2 * 8e-6)
    xx, yy = np.meshgrid(np.linspace(-0.8 * half, 0.8 * half, cols),
                         np.linspace(-0.8 * half, 0.8 * half, rows))
    xy = np.stack([xx.ravel(), yy.ravel()], 1)
    t = rng.uniform(0.5, 1.0, xy.shape[0]).astype(np.float32)
    return I.Workload(f"grid{cols}x{rows}_{nx}x{ny}", nx, ny, 8e-6, 8e-6, 532e-9, 0.2, xy, t,
                      I.gaussian_amplitude(nx, ny), I.uniform_phase(rng, nx, ny), 3)


WORKLOADS = {"ragged333x250_300": ragged, "grid13x41_333x250": ragged_grid,
             "pupil1024_poisson1000":
             lambda: I.named("pupil1024_poisson1000"),
             "pupil1920x1152_grid2500": lambda: I.named("pupil1920x1152_grid2500"),
             "table1_grid9x9": lambda: I.named("table1_grid9x9"),
             "table1_grid45x47": lambda: I.named("table1_grid45x47"),
             "table1_grid20x20": lambda: I.table1_workload(20, 20, seed=9)}


@functools.lru_cache(maxsize=None)
def reference(name, j=2):
    """The oracle's iterate j (phi_j, w_j) and one step from it: Theta, w_{j+1}, E'."""
    w = WORKLOADS[name]()
    fx, fy = O.plan_matrices(w.nx, w.ny, w.pitch_x, w.pitch_y, w.wavelength, w.focal_length,
                             w.focus_xy)
    run = O.gsw(w.amplitude, w.phi0, fx, fy, w.target, j)
    phi_j = run["phi"].astype(np.float32)
    w_j = run["w"].astype(np.float32)
    A = w.amplitude.astype(np.float64)
    theta = O.forward(O.pupil_field(A, phi_j.astype(np.float64)), fx, fy)
    w_new = O.generalized_weights(w_j.astype(np.float64), w.target, np.abs(theta) ** 2)
    back = O.adjoint(O.focused_field(w_new, w.target, theta), fx, fy)
    return w, j, phi_j, w_j, theta, w_new, back


def check_plan(ofa, name, prec, j=2, **kw):
    w, j, phi_j, w_j, theta, w_new, back = reference(name, j)
    plan = ofa.Plan.from_workload(w, precision=prec,
                                  stream=torch.cuda.current_stream().cuda_stream, **kw)
    cfg = ofa.ofa_plan_config(plan.handle)
    # forward from the same iterate
    phi_d = torch.from_numpy(phi_j).cuda()
    th = torch.zeros(w.n_foci, 2, device="cuda")
    ofa.ofa_forward(plan.handle, phi_d, th, None)
    torch.cuda.synchronize()
    g = th.cpu().numpy().astype(np.float64)
    g = g[:, 0] + 1j * g[:, 1]
    a, b = np.abs(g), np.abs(theta)
    amp_l2 = np.linalg.norm(a - b) / np.linalg.norm(b)
    amp_max = np.max(np.abs(a - b)) / b.max()
    # one iteration from the same iterate
    plan.set_state(phi_j, w_j, j)
    plan.iterate(1)
    phi_g, w_g, j_g = plan.get_state()
    plan.close()
    wrel = np.linalg.norm(w_g - w_new) / np.linalg.norm(w_new)
    mag = np.abs(back)
    d = np.abs(np.exp(1j * phi_g) - np.exp(1j * np.angle(back)))
    perr = math.sqrt(np.sum((mag * d) ** 2) / np.sum(mag ** 2))
    print(f"{name} {prec} {cfg}: amp L2 {amp_l2:.2e} max {amp_max:.2e}; w {wrel:.2e}; "
          f"phase {perr:.2e}")
    tol = AMP_TOL[prec]
    assert j_g == j + 1
    assert amp_l2 < tol and amp_max < tol, (amp_l2, amp_max)
    assert wrel < W_FACTOR * tol, wrel
    assert perr < PHASE_FACTOR * tol, perr
    return cfg


@pytest.fixture(scope="module")
def dev(ofa):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3", "tf32", "bf16"])
@pytest.mark.parametrize("config", CONFIGS, ids=cfg_id)
def test_every_kernel_config_ragged(ofa, dev, prec, config):
    """333 x 250 pupil, 300 foci: every tile ragged in all three dimensions."""
    cfg = check_plan(ofa, "ragged333x250_300", prec, kernel_config=config, fused_loop=0)
    assert (cfg["fwd_bn"], cfg["fwd_split"], cfg["fwd_cta_group"], cfg["inv_bn"],
            cfg["inv_cta_group"]) == tuple(config)


@pytest.mark.parametrize("config", CONFIGS, ids=cfg_id)
def test_every_kernel_config_pupil1024_poisson1000(ofa, dev, config):
    """The benchmark workload (1024^2 pupil, 1000 foci) in the default F16X3 form."""
    cfg = check_plan(ofa, "pupil1024_poisson1000", "f16x3", kernel_config=config,
                     fused_loop=0)
    assert cfg["fwd_split"] == config[1]


LOOP_CONFIGS = [(cg, split) for cg in (1, 2) for split in (1, 2, 4)]


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3", "tf32", "bf16"])
@pytest.mark.parametrize("loop", LOOP_CONFIGS, ids=lambda c: "cg{}s{}".format(*c))
def test_fused_loop_configs_ragged(ofa, dev, prec, loop):
    """The fused loop kernel in every configuration on the ragged pupil."""
    cfg = check_plan(ofa, "ragged333x250_300", prec, fused_loop=1, loop_config=loop)
    assert (cfg["fused_loop"], cfg["loop_cta_group"], cfg["loop_split"]) == (1,) + tuple(loop)


@pytest.mark.parametrize("loop", LOOP_CONFIGS, ids=lambda c: "cg{}s{}".format(*c))
def test_fused_loop_configs_pupil1024_poisson1000(ofa, dev, loop):
    cfg = check_plan(ofa, "pupil1024_poisson1000", "f16x3", fused_loop=1, loop_config=loop)
    assert cfg["fused_loop"] == 1 and cfg["loop_ctas"] >= 2


@pytest.mark.parametrize("prec", ["fp32", "f16x3", "bf16x3"])
@pytest.mark.parametrize("name", ["pupil1024_poisson1000", "pupil1920x1152_grid2500"])
def test_one_step_full_size(ofa, dev, prec, name):
    """One step from the same iterate at full size, in the default configuration."""
    cfg = check_plan(ofa, name, prec)
    assert cfg["fused_loop"] == 0


@pytest.mark.parametrize("j", [2, 5])
@pytest.mark.parametrize("name", ["table1_grid9x9", "table1_grid45x47"])
def test_separable_one_step(ofa, dev, name, j):
    """The separable grid form (FP32): forward amplitudes and one iteration from the
    oracle's iterate j, at the start and in the steep climb of xi (iteration 5), in the
    plan's default execution (the persistent loop)."""
    cfg = check_plan(ofa, name, "fp32", j=j, separable=1)
    assert cfg["fused_loop"] == 1


@pytest.mark.parametrize("loop", [0, 1])
@pytest.mark.parametrize("name", ["table1_grid9x9", "table1_grid20x20", "table1_grid45x47"])
def test_separable_loop_one_step(ofa, dev, name, loop):
    """The separable form's persistent loop and its multi-launch form, one step from the
    oracle's iterate 5, on grids with 1 to 15 foci per block in the loop's Theta sums and
    1 to 5 per thread in its focal step (81, 400 and 2115 foci)."""
    cfg = check_plan(ofa, name, "fp32", j=5, separable=1, separable_loop=loop)
    assert cfg["fused_loop"] == loop


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3", "tf32", "bf16"])
@pytest.mark.parametrize("name", ["grid13x41_333x250", "table1_grid9x9", "table1_grid20x20",
                                  "table1_grid45x47"])
def test_separable_tc_one_step(ofa, dev, name, prec):
    """The separable form's iteration on the tensor cores (forced), one step from the
    oracle's iterate 5: G = E Fx_u^T per contraction part, Theta and the new weights from
    it, U = conj(Fy_u)^T C and the inverse product with the phase projection, within the
    form's tolerances; on a ragged pupil and on grids of 9 to 47 distinct coordinates, in
    every tensor-core precision (TF32: four-byte operand planes)."""
    cfg = check_plan(ofa, name, prec, j=5, separable=1, separable_tc=1)
    assert cfg["fwd_bn"] == 128 and cfg["fused_loop"] == 0, cfg


@pytest.mark.parametrize("prec", ["f16x3", "tf32"])
def test_fused_loop_one_step_1920x1152(ofa, dev, prec):
    """The fused loop where the CTAs run several units per phase: 1920 x 1152 has an odd
    number of 128-row tiles (single CTAs), 180 forward and 270 inverse units over the
    SMs, so the accumulators alternate between two TMEM buffers and Fy is read from
    global memory in the forward epilogue."""
    cfg = check_plan(ofa, "pupil1920x1152_grid2500", prec, fused_loop=1)
    assert cfg["fused_loop"] == 1 and cfg["loop_cta_group"] == 1


@pytest.mark.parametrize("prec", ["f16x3", "tf32"])
def test_fused_loop_matches_per_product_kernels(ofa, dev, prec):
    """The same 20 iterations with and without the fused loop: the xi histories agree
    (the two differ only in the order of FP32 sums) and both runs are bitwise
    repeatable."""
    w = I.named("pupil256_grid100_uniform")
    runs = {}
    for mode in (0, 1, 1):
        plan = ofa.Plan.from_workload(w, precision=prec, fused_loop=mode)
        assert ofa.ofa_plan_config(plan.handle)["fused_loop"] == mode
        plan.iterate(20)
        runs.setdefault(mode, []).append((plan.xi_history(), plan.phase()))
        plan.close()
    h0, h1 = runs[0][0][0], runs[1][0][0]
    assert np.max(np.abs(h0 - h1)) < (1e-4 if prec == "f16x3" else 2e-3)
    assert np.array_equal(runs[1][0][1], runs[1][1][1])


def test_fused_loop_threshold_and_resume(ofa, dev):
    """Threshold stop inside one launch, a stopped loop staying stopped, and resume."""
    w = I.named("pupil256_grid100_uniform")
    fx, fy = O.plan_matrices(w.nx, w.ny, w.pitch_x, w.pitch_y, w.wavelength, w.focal_length,
                             w.focus_xy)
    ref = O.gsw(w.amplitude, w.phi0, fx, fy, w.target, 50, threshold=0.99)
    plan = ofa.Plan.from_workload(w, precision="f16x3", fused_loop=1)
    it, _ = plan.iterate(50, threshold=0.99, want_stats=True)
    assert abs(it - ref["iters"]) <= 1, (it, ref["iters"])
    hist = plan.xi_history()
    assert hist[-1] > 0.99 and np.all(hist[:-1] <= 0.99)
    plan.close()
    # resume: 7 + 5 iterations equal 12 bit for bit
    a = ofa.Plan.from_workload(w, precision="f16x3", fused_loop=1)
    a.iterate(12)
    full = a.phase()
    a.close()
    b = ofa.Plan.from_workload(w, precision="f16x3", fused_loop=1)
    b.iterate(7)
    phi7, w7, j7 = b.get_state()
    b.close()
    c = ofa.Plan.from_workload(w, precision="f16x3", fused_loop=1)
    c.set_state(phi7, w7, j7)
    c.iterate(5)
    assert np.array_equal(c.phase(), full)
    c.close()


def test_unsupported_config_is_rejected(ofa, dev):
    w = WORKLOADS["ragged333x250_300"]()
    w2 = ragged(300, 260, 40, seed=3)          # 3 row tiles: no 2-SM pairs
    for wl, cfg in ((w, (192, 1, 1, 128, 1)), (w, (128, 8, 1, 128, 1)),
                    (w2, (128, 1, 2, 128, 1)), (w2, (128, 1, 1, 128, 2))):
        with pytest.raises(ofa.OfaError) as e:
            ofa.Plan.from_workload(wl, precision="f16x3", kernel_config=cfg)
        assert e.value.status == ofa.OFA_ERR_UNSUPPORTED
