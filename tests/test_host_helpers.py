"""Host-side helpers of plan creation, compiled on their own (CPU only).

csrc/ofa_host.h holds the plain C++ that plan creation runs on the host; here it is
compiled with the system C++ compiler into a small driver and checked against numpy
on random amplitudes, on sizes that are and are not multiples of its eight lanes,
and on every invalid value the library must reject.
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
#include <vector>
#include "ofa_host.h"
int main(int argc, char** argv) {
  std::FILE* f = std::fopen(argv[1], "rb");
  std::vector<float> a;
  float x;
  while (std::fread(&x, sizeof x, 1, f) == 1) a.push_back(x);
  std::fclose(f);
  double amax = -1.0, energy = -1.0;
  const bool ok = ofa_host::amplitude_stats(a.data(), a.size(), &amax, &energy);
  std::printf("%d %.17g %.17g\n", ok ? 1 : 0, amax, energy);
  return 0;
}
"""


@pytest.fixture(scope="module")
def stats_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("host")
    src = d / "stats.cpp"
    src.write_text(DRIVER)
    exe = d / "stats"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return exe


def run(exe, tmp_path, a):
    f = tmp_path / "a.bin"
    np.asarray(a, dtype=np.float32).tofile(f)
    out = subprocess.run([str(exe), str(f)], check=True, capture_output=True, text=True).stdout
    ok, amax, energy = out.split()
    return ok == "1", float(amax), float(energy)


@pytest.mark.parametrize("n", [1, 7, 8, 9, 1000, 4099])
def test_amplitude_stats_matches_numpy(stats_exe, tmp_path, n):
    a = np.random.default_rng(n).uniform(0.0, 2.0, n).astype(np.float32)
    ok, amax, energy = run(stats_exe, tmp_path, a)
    a64 = a.astype(np.float64)
    assert ok
    assert amax == a64.max()
    assert energy == pytest.approx(float(np.sum(a64 * a64)), rel=1e-13)


def test_amplitude_stats_all_zero_is_valid_with_zero_peak(stats_exe, tmp_path):
    ok, amax, energy = run(stats_exe, tmp_path, np.zeros(20))
    assert ok and amax == 0.0 and energy == 0.0


@pytest.mark.parametrize("bad", [-1e-30, -1.0, np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("where", [0, 5, 8, 16, 18])
def test_amplitude_stats_rejects_invalid_values(stats_exe, tmp_path, bad, where):
    a = np.ones(19, dtype=np.float32)
    a[where] = bad
    ok, _, _ = run(stats_exe, tmp_path, a)
    assert not ok


def test_amplitude_stats_accepts_the_largest_float(stats_exe, tmp_path):
    a = np.full(10, np.finfo(np.float32).max, dtype=np.float32)
    ok, amax, energy = run(stats_exe, tmp_path, a)
    assert ok and amax == float(np.finfo(np.float32).max) and np.isfinite(energy)
