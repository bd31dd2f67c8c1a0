"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol that include/ofa.h declares, and its host helpers follow the paper."""
import json
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ofa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ofa_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(ofa):
    names = declared_symbols()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", ofa.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ofa_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    bound = {n for n, _, _ in ofa.SIGNATURES}
    assert set(names) == bound


def test_status_strings(ofa):
    assert ofa.ofa_status_string(0) == "OFA_OK"
    assert ofa.ofa_status_string(2) == "OFA_ERR_OUT_OF_RANGE"
    assert ofa.ofa_status_string(6) == "OFA_ERR_TIMEOUT"
    assert ofa.ofa_status_string(99) == "OFA_UNKNOWN"


def test_options_default(ofa):
    o = ofa.ofa_options_default()
    assert o.precision == ofa.OFA_PREC_F16X3
    assert o.waist_frac == 0.4
    assert o.weighting == 1
    assert o.autotune == 1
    assert o.separable == -1 and not o.focus_z
    assert o.separable_loop == -1 and o.separable_tc == -1
    assert not o.amplitude and not o.phi0 and not o.cuda_stream


def test_eq3_zero_padding_table1(ofa):
    g = json.load(open(os.path.join(GOLDEN, "table1_eq3.json")))
    m = ofa.ofa_fft_equivalent_size(g["slm_pixels"], g["slm_pitch_m"], g["wavelength_m"],
                                    g["focal_length_m"], g["camera_pitch_m"])
    assert m == g["zero_padded_size"]


def test_max_foci_table1(ofa):
    g = json.load(open(os.path.join(GOLDEN, "table1_eq3.json")))
    gap = g["min_gap_camera_pixels"] * g["camera_pitch_m"]
    n = ofa.ofa_max_foci_per_axis(g["slm_pitch_m"], g["wavelength_m"], g["focal_length_m"], gap)
    assert n == g["max_foci_per_axis"]


def test_alias_free_field_validation(ofa):
    g = json.load(open(os.path.join(GOLDEN, "table1_eq3.json")))
    lam, f, p = g["wavelength_m"], g["focal_length_m"], g["slm_pitch_m"]
    gap = g["min_gap_camera_pixels"] * g["camera_pitch_m"]
    half = lam * f / (2 * p)

    def grid(n):
        c = (np.arange(n) - (n - 1) / 2) * gap
        xx, yy = np.meshgrid(c, c)
        return np.stack([xx.ravel(), yy.ravel()], 1)

    st, bad = ofa.ofa_check_foci(grid(227), p, p, lam, f)
    assert st == ofa.OFA_OK and bad == -1
    st, bad = ofa.ofa_check_foci(grid(229), p, p, lam, f)
    assert st == ofa.OFA_ERR_OUT_OF_RANGE and bad == 0
    xy = np.array([[0.0, 0.0], [half * 0.999, 0.0], [0.0, -half]])
    st, bad = ofa.ofa_check_foci(xy, p, p, lam, f)
    assert st == ofa.OFA_ERR_OUT_OF_RANGE and bad == 2
    st, bad = ofa.ofa_check_foci(np.array([[np.nan, 0.0]]), p, p, lam, f)
    assert st == ofa.OFA_ERR_INVALID_ARG and bad == 0


def test_plan_create_rejects_bad_input_before_touching_cuda(ofa):
    xy = np.zeros((3, 2))
    t = np.ones(3, np.float32)
    with pytest.raises(ofa.OfaError) as e:
        ofa.ofa_plan_create(0, 16, 8e-6, 8e-6, 532e-9, 0.2, xy, t)
    assert e.value.status == ofa.OFA_ERR_INVALID_ARG
    with pytest.raises(ofa.OfaError) as e:
        ofa.ofa_plan_create(16, 16, 8e-6, 8e-6, 532e-9, 0.2, np.array([[1.0, 0.0]]),
                            np.ones(1, np.float32))
    assert e.value.status == ofa.OFA_ERR_OUT_OF_RANGE
    with pytest.raises(ofa.OfaError) as e:
        ofa.ofa_plan_create(16, 16, 8e-6, 8e-6, 532e-9, 0.2, xy, np.zeros(3, np.float32))
    assert e.value.status == ofa.OFA_ERR_INVALID_ARG
    with pytest.raises(ofa.OfaError) as e:
        ofa.ofa_plan_create(16, 16, 8e-6, -1.0, 532e-9, 0.2, xy, t)
    assert e.value.status == ofa.OFA_ERR_INVALID_ARG
    o = ofa.ofa_options_default()
    o.precision = 17
    with pytest.raises(ofa.OfaError) as e:
        ofa.ofa_plan_create(16, 16, 8e-6, 8e-6, 532e-9, 0.2, xy, t, o)
    assert e.value.status == ofa.OFA_ERR_INVALID_ARG
    assert "precision" in ofa.ofa_last_error()


def test_3d_axial_offsets_validated_before_touching_cuda(ofa):
    xy = np.array([[1e-3, 0.0], [0.0, -1e-3]])
    t = np.ones(2, np.float32)
    o = ofa.ofa_options_default()
    z = np.array([0.0, np.nan])
    o.focus_z = z.ctypes.data
    with pytest.raises(ofa.OfaError) as e:
        ofa.ofa_plan_create(64, 64, 8e-6, 8e-6, 532e-9, 0.2, xy, t, o)
    assert e.value.status == ofa.OFA_ERR_INVALID_ARG
    # |z| >= f, and a defocus whose phase the pupil cannot sample
    for bad in (np.array([0.0, 0.25]), np.array([0.19, 0.0])):
        o.focus_z = bad.ctypes.data
        n = 4096 if bad[0] else 64
        with pytest.raises(ofa.OfaError) as e:
            ofa.ofa_plan_create(n, n, 8e-6, 8e-6, 532e-9, 0.2, xy, t, o)
        assert e.value.status == ofa.OFA_ERR_OUT_OF_RANGE, ofa.ofa_last_error()


def test_null_safe_destroy(ofa):
    ofa.ofa_destroy(None)
    ofa.ofa_batch_destroy(None)
