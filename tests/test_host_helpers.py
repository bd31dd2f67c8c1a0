"""Host-side helpers of plan creation, compiled on their own (CPU only).

csrc/ofa_host.h holds the plain C++ that plan creation runs on the host to choose the
separable grid form: the bounded count of distinct focus coordinates (the grid of the
separable form of Eq. 2) and the test that no two foci share a grid point.  Here it is
compiled with the system C++ compiler into a small driver and checked against numpy on
regular grids, scattered foci, repeated and signed-zero coordinates, and at the bound.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2206_12661_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "ofa_host.h"
// argv: file of 2n doubles (x, y pairs), coordinate c, bound lim
int main(int argc, char** argv) {
  std::FILE* f = std::fopen(argv[1], "rb");
  std::vector<double> xy;
  double v;
  while (std::fread(&v, sizeof v, 1, f) == 1) xy.push_back(v);
  std::fclose(f);
  const int n = (int)(xy.size() / 2);
  std::vector<double> out;
  const bool ok = ofa_host::distinct_coords(xy.data(), n, std::atoi(argv[2]),
                                            (size_t)std::atoll(argv[3]), out);
  std::printf("%d %d", ok ? 1 : 0, ofa_host::one_focus_per_point(xy.data(), n) ? 1 : 0);
  if (ok)
    for (double d : out) std::printf(" %.17g", d);
  std::printf("\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("host")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    out = d / "driver"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(out)], check=True)
    return out


def run(exe, tmp_path, xy, c, lim):
    f = tmp_path / "xy.bin"
    np.asarray(xy, dtype=np.float64).reshape(-1).tofile(f)
    out = subprocess.run([str(exe), str(f), str(c), str(lim)], check=True, capture_output=True,
                         text=True).stdout.split()
    ok, unique = out[0] == "1", out[1] == "1"
    return ok, unique, np.array([float(v) for v in out[2:]])


def grid(cols, rows, gap=69e-6):
    gx = (np.arange(cols) - (cols - 1) / 2.0) * gap
    gy = (np.arange(rows) - (rows - 1) / 2.0) * gap
    xx, yy = np.meshgrid(gx, gy)
    return np.stack([xx.ravel(), yy.ravel()], 1), gx, gy


@pytest.mark.parametrize("cols,rows", [(9, 9), (45, 47), (1, 5), (13, 1)])
def test_grid_coordinates_are_the_distinct_values(exe, tmp_path, cols, rows):
    xy, gx, gy = grid(cols, rows)
    rng = np.random.default_rng(cols * 100 + rows)
    xy = xy[rng.permutation(len(xy))]            # any focus order
    okx, unique, ux = run(exe, tmp_path, xy, 0, cols)
    oky, _, uy = run(exe, tmp_path, xy, 1, rows)
    assert okx and oky and unique
    assert np.array_equal(ux, np.sort(gx)) and np.array_equal(uy, np.sort(gy))


def test_count_stops_past_the_bound(exe, tmp_path):
    xy, _, _ = grid(45, 47)
    assert run(exe, tmp_path, xy, 0, 45)[0]        # exactly at the bound
    assert not run(exe, tmp_path, xy, 0, 44)[0]    # one past it
    assert not run(exe, tmp_path, xy, 1, 0)[0]


def test_scattered_foci(exe, tmp_path):
    rng = np.random.default_rng(3)
    xy = rng.uniform(-1e-3, 1e-3, (500, 2))
    ok, unique, ux = run(exe, tmp_path, xy, 0, 500)
    assert ok and unique and np.array_equal(ux, np.unique(xy[:, 0]))
    assert not run(exe, tmp_path, xy, 0, 100)[0]


def test_signed_zero_and_repeats_count_once(exe, tmp_path):
    xy = np.array([[0.0, 1e-4], [-0.0, 2e-4], [3e-4, 1e-4], [3e-4, 1e-4]])
    ok, unique, ux = run(exe, tmp_path, xy, 0, 2)
    assert ok and len(ux) == 2 and ux[0] == 0.0 and ux[1] == 3e-4
    assert not unique                               # the last two foci share a point
    ok, unique, uy = run(exe, tmp_path, xy[:3], 1, 2)
    assert ok and unique and np.array_equal(uy, [1e-4, 2e-4])
