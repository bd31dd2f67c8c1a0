"""Pupil-row shards of one hologram, emulated on one GPU, against the oracle and the
unsharded plan (the multi-GPU form of the loop: partial Theta per shard, one sum of K
complex values, replicated weight update, inverse per shard).

Tolerances as in the one-step tests: amplitudes within the form's amplitude tolerance,
weights within 2x and the |E'|-weighted phase within 3x of it."""
import functools
import math

import numpy as np
import pytest

import oracle as O
from paper_2206_12661_gb300 import inputs as I
from paper_2206_12661_gb300 import shard as SH

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AMP_TOL = {"fp32": 1e-5, "f16x3": 1e-5}


@pytest.fixture(scope="module")
def dev(ofa):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def ragged(nx=300, ny=260, K=120, seed=41):
    rng = np.random.default_rng(seed)
    half = 532e-9 * 0.2 / (2 * 8e-6)
    xy = rng.uniform(-0.9 * half, 0.9 * half, (K, 2))
    t = rng.uniform(0.5, 1.0, K).astype(np.float32)
    return I.Workload(f"ragged{nx}x{ny}_{K}", nx, ny, 8e-6, 8e-6, 532e-9, 0.2, xy, t,
                      I.gaussian_amplitude(nx, ny), I.uniform_phase(rng, nx, ny), 3)


WORKLOADS = {"ragged300x260_120": ragged,
             "pupil1024_poisson1000": lambda: I.named("pupil1024_poisson1000")}


@functools.lru_cache(maxsize=None)
def reference(name, j=2):
    w = WORKLOADS[name]()
    fx, fy = O.plan_matrices(w.nx, w.ny, w.pitch_x, w.pitch_y, w.wavelength, w.focal_length,
                             w.focus_xy)
    run = O.gsw(w.amplitude, w.phi0, fx, fy, w.target, j)
    phi_j, w_j = run["phi"].astype(np.float32), run["w"].astype(np.float32)
    theta, _, xi, w_new, _ = O.gsw_step(w.amplitude, phi_j.astype(np.float64),
                                        w_j.astype(np.float64), fx, fy, w.target)
    back = O.adjoint(O.focused_field(w_new, w.target, theta), fx, fy)
    return w, j, phi_j, w_j, theta, xi, w_new, back


STREAM = {}


def stream():
    """One non-default stream for the shards and the sum of their partials."""
    if "s" not in STREAM:
        STREAM["s"] = torch.cuda.Stream()
    return STREAM["s"]


def make_shards(w, G, prec):
    s = stream()
    torch.cuda.synchronize()
    return [SH.PlanShard(w, r0, rows, precision=prec, stream=s.cuda_stream)
            for r0, rows in SH.row_ranges(w.ny, G)]


@pytest.mark.parametrize("prec", ["f16x3", "fp32"])
@pytest.mark.parametrize("G", [2, 4])
@pytest.mark.parametrize("name", ["ragged300x260_120", "pupil1024_poisson1000"])
def test_sharded_step_matches_oracle(ofa, dev, name, G, prec):
    """One step of G row shards from the oracle's iterate: the summed Theta, the
    replicated weights and every shard's phase rows against the unsharded oracle step."""
    w, j, phi_j, w_j, theta, xi, w_new, back = reference(name)
    shards = make_shards(w, G, prec)
    for s in shards:
        s.plan.set_state(phi_j[s.row0:s.row0 + s.rows], w_j, j)
    loop = SH.ShardedLoop(shards)
    with torch.cuda.stream(stream()):
        total = loop.step()
    torch.cuda.synchronize()
    t = total.cpu().numpy().astype(np.float64)
    got = t[:, 0] + 1j * t[:, 1]
    a, b = np.abs(got), np.abs(theta)
    amp = np.linalg.norm(a - b) / np.linalg.norm(b)
    phis, ws = [], []
    for s in shards:
        phi_s, w_s, j_s = s.plan.get_state()
        assert j_s == j + 1
        phis.append(phi_s)
        ws.append(w_s)
        assert abs(s.plan.xi_history()[-1] - xi) < 1e-5
        s.close()
    phi_g = np.concatenate(phis, axis=0)
    for w_s in ws[1:]:                       # every shard holds the same weights, bitwise
        assert np.array_equal(w_s, ws[0])
    wrel = np.linalg.norm(ws[0] - w_new) / np.linalg.norm(w_new)
    mag = np.abs(back)
    d = np.abs(np.exp(1j * phi_g) - np.exp(1j * np.angle(back)))
    perr = math.sqrt(np.sum((mag * d) ** 2) / np.sum(mag ** 2))
    tol = AMP_TOL[prec]
    print(f"{name} G={G} {prec}: amp {amp:.2e}, w {wrel:.2e}, phase {perr:.2e}")
    assert amp < tol and wrel < 2 * tol and perr < 3 * tol, (amp, wrel, perr)


@pytest.mark.parametrize("G", [2, 4])
def test_sharded_run_matches_unsharded_plan(ofa, dev, G):
    """20 iterations over G shards and on one plan: the xi histories agree (the shards
    sum the partial Theta in a different order) and the final phases agree."""
    w = I.named("pupil256_grid100_uniform")
    w.target = np.random.default_rng(7).uniform(0.5, 1.0, w.n_foci).astype(np.float32)
    shards = make_shards(w, G, "fp32")
    with torch.cuda.stream(stream()):
        SH.ShardedLoop(shards).run(20)
    torch.cuda.synchronize()
    hist = shards[0].plan.xi_history()
    phi_s = np.concatenate([s.plan.get_state()[0] for s in shards], axis=0)
    for s in shards:
        s.close()
    plan = ofa.Plan.from_workload(w, precision="fp32")
    plan.iterate(20)
    ref_hist, ref_phi = plan.xi_history(), plan.phase()
    plan.close()
    assert len(hist) == 20
    assert np.max(np.abs(hist - ref_hist)) < 1e-4
    mag = w.amplitude.astype(np.float64)
    d = np.abs(np.exp(1j * phi_s) - np.exp(1j * ref_phi))
    assert math.sqrt(np.sum((mag * d) ** 2) / np.sum(mag ** 2)) < 1e-3


def test_shard_needs_its_stream(ofa, dev):
    with pytest.raises(ValueError):
        SH.PlanShard(ragged(), 0, 130, precision="fp32", stream=None)


def test_shard_options_are_checked(ofa, dev):
    w = ragged()
    with pytest.raises(ofa.OfaError) as e:
        ofa.Plan(w.nx, 100, w.pitch_x, w.pitch_y, w.wavelength, w.focal_length, w.focus_xy,
                 w.target, shard=(200, 260))
    assert e.value.status == ofa.OFA_ERR_INVALID_ARG
