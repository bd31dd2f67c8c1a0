"""Seeded synthetic workloads for the GSW-MTP focus-array loop.

This module only draws inputs: focus positions, target intensities, the
pupil amplitude profile and an initial phase.  It holds none of the method's
arithmetic (no DFT rows, no propagation, no weighting), so that the CUDA
library's tests and the FP64 oracle can be fed the very same arrays.

The paper measures on no public dataset; every workload here is synthetic and
follows the geometry of its simulations (phase-only SLM pupil, Fourier lens,
foci at arbitrary positions with chosen relative intensities; Table 1 and the
"Results and discussion" section of arXiv 2206.12661).  Shared optics of all
workloads: pixel pitch 8 um, wavelength 532 nm, focal length 200 mm.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PITCH = 8e-6
WAVELENGTH = 532e-9
FOCAL_LENGTH = 0.2


@dataclass
class Workload:
    """One hologram problem: pupil size, optics, foci, targets, A and phi0."""
    name: str
    nx: int
    ny: int
    pitch_x: float
    pitch_y: float
    wavelength: float
    focal_length: float
    focus_xy: np.ndarray          # [K][2] float64, metres in the focal plane
    target: np.ndarray            # [K] float32, relative target intensities
    amplitude: np.ndarray         # [ny][nx] float32
    phi0: np.ndarray              # [ny][nx] float32, radians in [-pi, pi)
    n_iter: int
    meta: dict = field(default_factory=dict)
    focus_z: np.ndarray | None = None   # [K] float64 axial offsets (m) of 3D foci, or None

    @property
    def n_foci(self) -> int:
        return int(self.focus_xy.shape[0])


def spot_size(n: int, pitch: float = PITCH, wavelength: float = WAVELENGTH,
              focal_length: float = FOCAL_LENGTH) -> float:
    """Diffraction-limited spot size lambda*f/(N*p) of an N-pixel aperture."""
    return wavelength * focal_length / (n * pitch)


def gaussian_amplitude(nx: int, ny: int, pitch_x: float = PITCH, pitch_y: float = PITCH,
                       waist_frac: float = 0.4) -> np.ndarray:
    """Gaussian beam profile exp(-(u^2/wx^2 + v^2/wy^2)), waist = waist_frac * aperture."""
    u = (np.arange(nx) - (nx - 1) / 2.0) * pitch_x
    v = (np.arange(ny) - (ny - 1) / 2.0) * pitch_y
    wx = waist_frac * nx * pitch_x
    wy = waist_frac * ny * pitch_y
    a = np.exp(-(v[:, None] ** 2 / wy ** 2 + u[None, :] ** 2 / wx ** 2))
    return a.astype(np.float32)


def uniform_phase(rng: np.random.Generator, nx: int, ny: int) -> np.ndarray:
    return rng.uniform(-np.pi, np.pi, size=(ny, nx)).astype(np.float32)


def jittered_grid(rng: np.random.Generator, cols: int, rows: int, pitch_x: float,
                  pitch_y: float, jitter: float = 0.3, count: int | None = None) -> np.ndarray:
    """cols x rows grid centred on the optical axis, each focus moved by U(+-jitter*pitch)."""
    gx = (np.arange(cols) - (cols - 1) / 2.0) * pitch_x
    gy = (np.arange(rows) - (rows - 1) / 2.0) * pitch_y
    xx, yy = np.meshgrid(gx, gy)
    pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
    pts[:, 0] += rng.uniform(-jitter, jitter, size=pts.shape[0]) * pitch_x
    pts[:, 1] += rng.uniform(-jitter, jitter, size=pts.shape[0]) * pitch_y
    if count is not None and count < pts.shape[0]:
        pts = pts[np.sort(rng.choice(pts.shape[0], size=count, replace=False))]
    return pts.astype(np.float64)


def poisson_disk(rng: np.random.Generator, width: float, height: float, min_dist: float,
                 tries: int = 30) -> np.ndarray:
    """Bridson's Poisson-disk sampling of a width x height box centred at the origin."""
    cell = min_dist / math.sqrt(2.0)
    gw = int(math.ceil(width / cell))
    gh = int(math.ceil(height / cell))
    grid = -np.ones((gh, gw), dtype=np.int64)
    pts: list[tuple[float, float]] = []
    active: list[int] = []

    def put(p):
        pts.append(p)
        idx = len(pts) - 1
        grid[int(p[1] / cell), int(p[0] / cell)] = idx
        active.append(idx)

    put((rng.uniform(0, width), rng.uniform(0, height)))
    r2 = min_dist * min_dist
    while active:
        j = int(rng.integers(len(active)))
        base = pts[active[j]]
        placed = False
        for _ in range(tries):
            ang = rng.uniform(0, 2 * math.pi)
            rad = rng.uniform(min_dist, 2 * min_dist)
            p = (base[0] + rad * math.cos(ang), base[1] + rad * math.sin(ang))
            if not (0 <= p[0] < width and 0 <= p[1] < height):
                continue
            cx, cy = int(p[0] / cell), int(p[1] / cell)
            ok = True
            for yy in range(max(cy - 2, 0), min(cy + 3, gh)):
                for xx in range(max(cx - 2, 0), min(cx + 3, gw)):
                    q = grid[yy, xx]
                    if q >= 0:
                        dx = pts[q][0] - p[0]
                        dy = pts[q][1] - p[1]
                        if dx * dx + dy * dy < r2:
                            ok = False
                            break
                if not ok:
                    break
            if ok:
                put(p)
                placed = True
                break
        if not placed:
            active[j] = active[-1]
            active.pop()
    arr = np.asarray(pts, dtype=np.float64)
    arr[:, 0] -= width / 2.0
    arr[:, 1] -= height / 2.0
    return arr


def _make(name, nx, ny, foci, target, rng, n_iter, meta, pitch=PITCH):
    return Workload(name=name, nx=nx, ny=ny, pitch_x=pitch, pitch_y=pitch,
                    wavelength=WAVELENGTH, focal_length=FOCAL_LENGTH,
                    focus_xy=np.ascontiguousarray(foci, dtype=np.float64),
                    target=np.ascontiguousarray(target, dtype=np.float32),
                    amplitude=gaussian_amplitude(nx, ny, pitch, pitch),
                    phi0=uniform_phase(rng, nx, ny), n_iter=n_iter, meta=meta)


def grid_workload(n: int = 256, cols: int = 10, rows: int = 10, n_iter: int = 50, seed: int = 1,
                  uniform_targets: bool = True, name: str | None = None) -> Workload:
    """Pupil n x n, cols x rows jittered grid at pitch 3 spots, Gaussian A (256^2 / 10x10 / 50 it)."""
    rng = np.random.default_rng(seed)
    s = spot_size(n)
    foci = jittered_grid(rng, cols, rows, 3 * s, 3 * s)
    k = foci.shape[0]
    t = np.ones(k) if uniform_targets else rng.uniform(0.5, 1.0, k)
    return _make(name or f"grid{n}x{n}_{k}foci", n, n, foci, t, rng, n_iter,
                 {"layout": "jittered grid", "pitch_spots": 3, "jitter": 0.3, "seed": seed})


def poisson_workload(n: int = 1024, n_foci: int = 1000, roi: float = 2.0e-3, n_iter: int = 100,
                     seed: int = 2, name: str | None = None) -> Workload:
    """Pupil n x n, n_foci Poisson-disk foci (min spacing 3 spots) in a roi x roi box, t ~ U[0.5,1].

    A 400 um square cannot hold 1000 foci at a 3-spot (39 um) spacing; the
    ROI is widened to 2.0 mm, which keeps the pupil, the focus count and the
    spacing (the cost of the loop does not depend on where the foci sit).
    """
    rng = np.random.default_rng(seed)
    s = spot_size(n)
    pts = poisson_disk(rng, roi, roi, 3 * s)
    if pts.shape[0] < n_foci:
        raise ValueError(f"ROI {roi} m holds only {pts.shape[0]} foci at spacing {3 * s}")
    pts = pts[np.sort(rng.choice(pts.shape[0], size=n_foci, replace=False))]
    t = rng.uniform(0.5, 1.0, n_foci)
    return _make(name or f"poisson{n}x{n}_{n_foci}foci", n, n, pts, t, rng, n_iter,
                 {"layout": "Poisson disk", "roi_m": roi, "min_spacing_spots": 3, "seed": seed})


def rect_workload(nx: int = 1920, ny: int = 1152, cols: int = 50, rows: int = 50, n_iter: int = 50,
                  seed: int = 3, name: str | None = None) -> Workload:
    """Pupil nx x ny, cols x rows grid at isotropic pitch 3*max(sx, sy), jitter 0.3, t = 1."""
    rng = np.random.default_rng(seed)
    pitch = 3 * max(spot_size(nx), spot_size(ny))
    foci = jittered_grid(rng, cols, rows, pitch, pitch)
    t = np.ones(foci.shape[0])
    w = _make(name or f"rect{nx}x{ny}_{foci.shape[0]}foci", nx, ny, foci, t, rng, n_iter,
              {"layout": "jittered grid", "pitch_m": pitch, "seed": seed})
    return w


def volume_workload(n: int = 512, cols: int = 7, rows: int = 7, layers: int = 3,
                    z_span: float = 0.1, n_iter: int = 50, seed: int = 6,
                    name: str | None = None) -> Workload:
    """3D array: `layers` jittered cols x rows grids (pitch 3 spots), layer l at
    axial offset z_l spread evenly over [-z_span/2, z_span/2], each layer's grid
    shifted by half a pitch so layers do not overlap in x-y, targets 1."""
    rng = np.random.default_rng(seed)
    s = spot_size(n)
    xy, zz = [], []
    for l in range(layers):
        g = jittered_grid(rng, cols, rows, 3 * s, 3 * s)
        g += (l - (layers - 1) / 2.0) * 1.5 * s
        xy.append(g)
        z = 0.0 if layers == 1 else -z_span / 2 + l * z_span / (layers - 1)
        zz.append(np.full(g.shape[0], z))
    xy = np.concatenate(xy)
    w = _make(name or f"volume{n}x{n}_{xy.shape[0]}foci", n, n, xy, np.ones(xy.shape[0]), rng,
              n_iter, {"layout": "jittered grids in layers", "layers": layers,
                       "z_span_m": z_span, "seed": seed})
    w.focus_z = np.ascontiguousarray(np.concatenate(zz), dtype=np.float64)
    return w


def table1_workload(cols: int = 9, rows: int = 9, n_iter: int = 40, seed: int = 7,
                    uniform_targets: bool = False, name: str | None = None) -> Workload:
    """Table 1 geometry: 1000 x 1000 SLM pixels at 12.5 um, 785 nm, f = 250 mm, a regular
    cols x rows grid with the 20-camera-pixel gap (3.45 um pixels) of the Fig. 2
    discussion; targets U[0.5, 1] (the paper's 'various intensities') or 1."""
    rng = np.random.default_rng(seed)
    n, pitch, lam, f = 1000, 12.5e-6, 785e-9, 0.25
    gap = 20 * 3.45e-6
    gx = (np.arange(cols) - (cols - 1) / 2.0) * gap
    gy = (np.arange(rows) - (rows - 1) / 2.0) * gap
    xx, yy = np.meshgrid(gx, gy)
    foci = np.stack([xx.ravel(), yy.ravel()], 1)
    k = foci.shape[0]
    t = np.ones(k) if uniform_targets else rng.uniform(0.5, 1.0, k)
    return Workload(name=name or f"table1_grid{cols}x{rows}", nx=n, ny=n, pitch_x=pitch,
                    pitch_y=pitch, wavelength=lam, focal_length=f,
                    focus_xy=np.ascontiguousarray(foci, dtype=np.float64),
                    target=np.ascontiguousarray(t, dtype=np.float32),
                    amplitude=gaussian_amplitude(n, n, pitch, pitch),
                    phi0=uniform_phase(rng, n, n), n_iter=n_iter,
                    meta={"layout": "regular grid", "gap_m": gap, "seed": seed})


def table1_random_workload(n_spots: int = 66, ux: int = 45, uy: int = 47, lattice: int = 61,
                           step_px: int = 12, n_iter: int = 40, seed: int = 10,
                           name: str | None = None) -> Workload:
    """Table 1 geometry with the paper's second simulated OFA: n_spots foci at random
    positions with random intensities U[0.5, 1], sampled on the camera grid (3.45 um
    pixels) so that they take exactly ux distinct x and uy distinct y values (the
    45 x 47 MTP sampling grid of the Fig. 2 discussion).  Positions are cells of a
    lattice x lattice lattice of step_px camera pixels centred on the axis (12 px =
    41 um, about 2.6 diffraction-limited spots of this pupil): ux columns and uy rows
    are drawn, every row gets one spot in a column chosen so that every column is used,
    and the remaining spots take distinct random free cells of those rows and columns."""
    if not (max(ux, uy) <= n_spots <= ux * uy and ux <= lattice and uy <= lattice):
        raise ValueError("need max(ux, uy) <= n_spots <= ux * uy within the lattice")
    rng = np.random.default_rng(seed)
    n, pitch, lam, f = 1000, 12.5e-6, 785e-9, 0.25
    step = step_px * 3.45e-6
    cols = np.sort(rng.choice(lattice, ux, replace=False))
    rows = np.sort(rng.choice(lattice, uy, replace=False))
    # one spot per row, covering every column, then distinct extra cells
    if uy >= ux:
        col_of_row = np.concatenate([rng.permutation(ux), rng.integers(0, ux, uy - ux)])
        cells = {(int(r), int(c)) for r, c in zip(range(uy), rng.permutation(col_of_row))}
    else:
        row_of_col = np.concatenate([rng.permutation(uy), rng.integers(0, uy, ux - uy)])
        cells = {(int(r), int(c)) for c, r in zip(range(ux), rng.permutation(row_of_col))}
    while len(cells) < n_spots:
        cells.add((int(rng.integers(uy)), int(rng.integers(ux))))
    cells = sorted(cells)
    centre = (lattice - 1) / 2.0
    foci = np.array([[(cols[c] - centre) * step, (rows[r] - centre) * step] for r, c in cells])
    t = rng.uniform(0.5, 1.0, n_spots)
    return Workload(name=name or f"table1_random{n_spots}", nx=n, ny=n, pitch_x=pitch,
                    pitch_y=pitch, wavelength=lam, focal_length=f,
                    focus_xy=np.ascontiguousarray(foci, dtype=np.float64),
                    target=np.ascontiguousarray(t, dtype=np.float32),
                    amplitude=gaussian_amplitude(n, n, pitch, pitch),
                    phi0=uniform_phase(rng, n, n), n_iter=n_iter,
                    meta={"layout": "random cells of a camera-pixel lattice",
                          "step_m": step, "distinct_x": ux, "distinct_y": uy, "seed": seed})


def batch_workloads(count: int = 256, sizes=(512, 768, 1024), k_min: int = 16, k_max: int = 4096,
                    n_iter: int = 50, seed: int = 5) -> list[Workload]:
    """Uneven batch: N drawn from sizes, K log-uniform in [k_min, k_max], jittered grid foci."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(sizes[int(rng.integers(len(sizes)))])
        k = int(round(math.exp(rng.uniform(math.log(k_min), math.log(k_max)))))
        side = int(math.ceil(math.sqrt(k)))
        s = spot_size(n)
        foci = jittered_grid(rng, side, side, 3 * s, 3 * s, count=k)
        t = rng.uniform(0.5, 1.0, k)
        out.append(_make(f"batch{i}_{n}x{n}_{k}foci", n, n, foci, t, rng, n_iter,
                         {"layout": "jittered grid", "seed": seed, "index": i}))
    return out


NAMED = {
    "pupil256_grid100_uniform": lambda: grid_workload(256, 10, 10, n_iter=50, seed=1,
                                                      name="pupil256_grid100_uniform"),
    "pupil1024_poisson1000": lambda: poisson_workload(1024, 1000, n_iter=100, seed=2,
                                                      name="pupil1024_poisson1000"),
    "pupil1920x1152_grid2500": lambda: rect_workload(1920, 1152, 50, 50, n_iter=50, seed=3,
                                                     name="pupil1920x1152_grid2500"),
    "pupil512_volume147": lambda: volume_workload(512, 7, 7, 3, z_span=0.1, n_iter=50, seed=6,
                                                  name="pupil512_volume147"),
    "table1_grid9x9": lambda: table1_workload(9, 9, n_iter=40, seed=7, name="table1_grid9x9"),
    "table1_grid45x47": lambda: table1_workload(45, 47, n_iter=40, seed=8,
                                                name="table1_grid45x47"),
    "table1_random66": lambda: table1_random_workload(66, 45, 47, n_iter=40, seed=10,
                                                      name="table1_random66"),
    "pupil1024_grid400_adam": lambda: grid_workload(1024, 20, 20, n_iter=200, seed=4,
                                                    uniform_targets=False,
                                                    name="pupil1024_grid400_adam"),
}


def named(name: str) -> Workload:
    """A single-hologram workload by name (see NAMED)."""
    return NAMED[name]()
