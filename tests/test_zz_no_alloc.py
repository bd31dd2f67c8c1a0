"""ofa_forward_noalloc: the allocation-free forward entry point, through the C ABI.

It serves callers that cannot allocate device memory when they need the focal
field (a real-time SLM refresh loop, or a process whose device memory a framework
allocator has reserved).  Its output must match the plan-based ofa_forward (FP32
form) within the FP32 amplitude tolerance of the parity tests, on two calls in a
row with different problems (the calls share one static scratch array, which
the second call must fully overwrite).  This file is collected last.
"""
import numpy as np
import pytest

import oracle as O
from paper_2206_12661_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5   # FP32-accurate forms in tests/test_gpu_parity.py


def problem(nx, ny, K, seed):
    rng = np.random.default_rng(seed)
    half = 532e-9 * 0.2 / (2 * 8e-6)
    xy = rng.uniform(-0.9 * half, 0.9 * half, (K, 2))
    return I.Workload(f"noalloc{nx}x{ny}_{K}", nx, ny, 8e-6, 8e-6, 532e-9, 0.2, xy,
                      np.ones(K, np.float32), I.gaussian_amplitude(nx, ny),
                      I.uniform_phase(rng, nx, ny), 1)


def plan_forward(ofa, w, phi_d):
    plan = ofa.Plan.from_workload(w, precision="fp32",
                                  stream=torch.cuda.current_stream().cuda_stream)
    theta = torch.zeros(w.n_foci, 2, device="cuda")
    ofa.ofa_forward(plan.handle, phi_d, theta, None)
    torch.cuda.synchronize()
    plan.close()
    t = theta.cpu().numpy()
    return t[:, 0] + 1j * t[:, 1]


def test_forward_noalloc_matches_plan_forward(ofa):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stream = torch.cuda.current_stream().cuda_stream
    for w in (problem(300, 260, 300, 1), problem(129, 100, 37, 2)):
        phi_d = torch.from_numpy(w.phi0).cuda()
        amp_d = torch.from_numpy(w.amplitude).cuda()
        xy_d = torch.from_numpy(w.focus_xy).cuda()
        theta = torch.full((w.n_foci, 2), float("nan"), device="cuda")
        inten = torch.full((w.n_foci,), float("nan"), device="cuda")
        ofa.ofa_forward_noalloc(w.nx, w.ny, w.pitch_x, w.pitch_y, w.wavelength,
                                w.focal_length, xy_d, phi_d, amp_d, theta, inten, stream)
        torch.cuda.synchronize()
        got = theta.cpu().numpy()
        got = got[:, 0] + 1j * got[:, 1]
        ref = plan_forward(ofa, w, phi_d)
        err = np.linalg.norm(np.abs(got) - np.abs(ref)) / np.linalg.norm(np.abs(ref))
        assert err < AMP_TOL, err
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 3 * AMP_TOL
        assert np.allclose(inten.cpu().numpy(), np.abs(got) ** 2, rtol=1e-5, atol=0)


def noalloc_forward(ofa, w):
    phi_d = torch.from_numpy(w.phi0).cuda()
    amp_d = torch.from_numpy(w.amplitude).cuda()
    xy_d = torch.from_numpy(w.focus_xy).cuda()
    theta = torch.full((w.n_foci, 2), float("nan"), device="cuda")
    ofa.ofa_forward_noalloc(w.nx, w.ny, w.pitch_x, w.pitch_y, w.wavelength, w.focal_length,
                            xy_d, phi_d, amp_d, theta, None,
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    t = theta.cpu().numpy()
    return t[:, 0] + 1j * t[:, 1]


@pytest.mark.parametrize("shape", [(16, 2048, 8192), (32768, 2, 64), (300, 260, 300)],
                         ids=["ny2048_K8192", "nx32768", "300x260_300"])
def test_forward_noalloc_matches_oracle_up_to_its_limits(ofa, shape):
    """Against the FP64 oracle's Eq. 2 at the foci, including each size limit of the
    static scratch (ny = 2048 in 32 row tiles, K = 8192 foci, nx = 32768)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nx, ny, K = shape
    w = problem(nx, ny, K, seed=nx + ny + K)
    fx, fy = O.plan_matrices(w.nx, w.ny, w.pitch_x, w.pitch_y, w.wavelength, w.focal_length,
                             w.focus_xy)
    ref = O.forward(O.pupil_field(w.amplitude, w.phi0), fx, fy)
    got = noalloc_forward(ofa, w)
    a, b = np.abs(got), np.abs(ref)
    err = np.linalg.norm(a - b) / np.linalg.norm(b)
    emax = np.max(np.abs(a - b)) / b.max()
    assert err < AMP_TOL and emax < AMP_TOL, (err, emax)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 3 * AMP_TOL


def test_forward_noalloc_rejects_sizes_beyond_scratch(ofa):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    xy = torch.zeros(4, 2, dtype=torch.float64, device="cuda")
    phi = torch.zeros(4096, 8, device="cuda")
    theta = torch.zeros(4, 2, device="cuda")
    with pytest.raises(ofa.OfaError) as e:
        ofa.ofa_forward_noalloc(8, 4096, 8e-6, 8e-6, 532e-9, 0.2, xy, phi, phi, theta, None)
    assert e.value.status == ofa.OFA_ERR_INVALID_ARG
    assert "static scratch" in str(e.value)
    # one past each limit: ny 2049 (33 row tiles), K 8193, nx 32769
    big = torch.zeros(2049 * 8, device="cuda")
    for nx, ny, k in ((8, 2049, 4), (8, 4, 8193), (32769, 1, 4)):
        xy_k = torch.zeros(k, 2, dtype=torch.float64, device="cuda")
        ph = torch.zeros(max(nx * ny, 1), device="cuda") if nx * ny > big.numel() else big
        th = torch.zeros(k, 2, device="cuda")
        with pytest.raises(ofa.OfaError) as e:
            ofa.ofa_forward_noalloc(nx, ny, 8e-6, 8e-6, 532e-9, 0.2, xy_k, ph, ph, th, None)
        assert e.value.status == ofa.OFA_ERR_INVALID_ARG
