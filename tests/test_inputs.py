"""The synthetic workloads match the recipes they are documented with (CPU only).

Every parity test and the bench draw their inputs from paper_2206_12661_gb300.inputs;
these tests pin the recipe itself: seeds reproduce, the Poisson-disk foci keep their
minimum spacing inside the stated region, grid jitter stays within its bound, the
batch draws its sizes and focus counts from the stated ranges, and every focus lies
inside the alias-free field of view.
"""
import math

import numpy as np
import pytest

from paper_2206_12661_gb300 import inputs as I


def alias_free(w) -> bool:
    hx = w.wavelength * w.focal_length / (2 * w.pitch_x)
    hy = w.wavelength * w.focal_length / (2 * w.pitch_y)
    return bool(np.all(np.abs(w.focus_xy[:, 0]) < hx) and np.all(np.abs(w.focus_xy[:, 1]) < hy))


@pytest.mark.parametrize("name", sorted(I.NAMED))
def test_named_workloads_are_seeded_and_well_formed(name):
    a, b = I.named(name), I.named(name)
    for f in ("focus_xy", "target", "amplitude", "phi0"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert a.focus_xy.dtype == np.float64 and a.focus_xy.shape == (a.n_foci, 2)
    assert a.target.dtype == np.float32 and a.target.shape == (a.n_foci,)
    assert a.amplitude.shape == (a.ny, a.nx) and a.phi0.shape == (a.ny, a.nx)
    assert a.phi0.min() >= -math.pi and a.phi0.max() < math.pi
    assert np.all(a.target > 0) and np.all(a.target <= 1)
    assert np.all(a.amplitude >= 0) and a.amplitude.max() <= 1
    assert alias_free(a)


def test_poisson1000_spacing_and_region():
    w = I.named("pupil1024_poisson1000")
    assert w.nx == w.ny == 1024 and w.n_foci == 1000 and w.n_iter == 100
    spacing = 3 * I.spot_size(1024)
    assert spacing == pytest.approx(38.96e-6, rel=1e-3)
    d = w.focus_xy[:, None, :] - w.focus_xy[None, :, :]
    dist = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(dist, np.inf)
    assert dist.min() >= spacing * (1 - 1e-12)
    assert np.all(np.abs(w.focus_xy) <= 1.0e-3)           # the 2.0 mm x 2.0 mm region
    assert w.target.min() >= 0.5 and w.target.max() <= 1.0


def test_poisson_disk_rejects_a_region_too_small():
    # the literal 400 um region cannot hold 1000 foci at a 3-spot spacing
    with pytest.raises(ValueError):
        I.poisson_workload(1024, 1000, roi=400e-6, seed=2)


def test_jittered_grid_stays_within_its_jitter():
    w = I.named("pupil256_grid100_uniform")
    pitch = 3 * I.spot_size(256)
    g = w.focus_xy / pitch
    # each focus is a lattice point (centred, half-integer offsets for an even count)
    # moved by at most 0.3 pitch per axis
    frac = g - (np.round(g - 0.5) + 0.5)
    assert np.all(np.abs(frac) <= 0.3 + 1e-9)
    assert w.n_foci == 100 and np.all(w.target == 1)


def test_gaussian_amplitude_closed_form():
    n, p = 64, 8e-6
    a = I.gaussian_amplitude(n, n, p, p, 0.4)
    u = (np.arange(n) - (n - 1) / 2) * p
    wx = 0.4 * n * p
    ref = np.exp(-(u[None, :] ** 2 + u[:, None] ** 2) / wx ** 2)
    assert np.allclose(a, ref, rtol=1e-6, atol=0)


def test_batch_draws_from_the_stated_ranges():
    ws = I.batch_workloads(count=256, seed=5)
    assert len(ws) == 256
    ns = {w.nx for w in ws}
    assert ns <= {512, 768, 1024} and len(ns) == 3
    ks = np.array([w.n_foci for w in ws])
    assert ks.min() >= 16 and ks.max() <= 4096
    # log-uniform over [16, 4096]: mean (4096 - 16) / ln 256 = 735.8
    assert 500 < ks.mean() < 1000
    assert all(alias_free(w) for w in ws)


def test_volume_layers_and_table1_grid():
    v = I.named("pupil512_volume147")
    assert v.n_foci == 147
    assert sorted(set(np.round(v.focus_z, 12))) == [-0.05, 0.0, 0.05]
    t = I.named("table1_grid9x9")
    assert (t.nx, t.pitch_x, t.wavelength, t.focal_length) == (1000, 12.5e-6, 785e-9, 0.25)
    xs = np.unique(np.round(t.focus_xy[:, 0], 12))
    assert len(xs) == 9 and np.allclose(np.diff(xs), 20 * 3.45e-6)


def test_table1_random66_recipe():
    """The paper's second simulated OFA: 66 spots at random cells of a camera-pixel
    lattice, with exactly 45 distinct x and 47 distinct y (its 45 x 47 MTP grid)."""
    w = I.named("table1_random66")
    step = 12 * 3.45e-6
    assert w.n_foci == 66 and (w.nx, w.ny) == (1000, 1000)
    xs = np.unique(np.round(w.focus_xy[:, 0], 12))
    ys = np.unique(np.round(w.focus_xy[:, 1], 12))
    assert (len(xs), len(ys)) == (45, 47)
    # on the lattice (centred, 12-pixel step), no two spots in one cell
    assert np.allclose(np.round(w.focus_xy / step * 2) / 2, w.focus_xy / step, atol=1e-9)
    assert len({(round(x, 12), round(y, 12)) for x, y in w.focus_xy}) == 66
    d = np.sqrt(((w.focus_xy[:, None] - w.focus_xy[None]) ** 2).sum(-1)) + np.eye(66)
    assert d.min() >= step - 1e-12
    assert alias_free(w)
    assert np.all((w.target >= 0.5) & (w.target <= 1.0))
    assert np.array_equal(w.focus_xy, I.named("table1_random66").focus_xy)
