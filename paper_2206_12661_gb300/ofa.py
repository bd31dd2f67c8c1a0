"""ctypes binding of libofa (include/ofa.h): argument marshalling only.

Every function named ``ofa_*`` here calls the C function of the same name;
every step of the hologram loop runs in the CUDA library.  Device pointers may
be given as integers or as objects with ``data_ptr()`` (torch tensors); host
arrays as numpy arrays.  There is no CPU fallback: if libofa.so cannot be
loaded, importing this module raises.

``Plan`` is a small convenience wrapper that owns an ``ofa_plan*``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libofa.so")

OFA_OK = 0
OFA_ERR_INVALID_ARG = 1
OFA_ERR_OUT_OF_RANGE = 2
OFA_ERR_CUDA = 3
OFA_ERR_OOM = 4
OFA_ERR_NUMERIC = 5
OFA_ERR_TIMEOUT = 6
OFA_ERR_UNSUPPORTED = 7

OFA_PREC_FP32 = 0
OFA_PREC_TF32 = 1
OFA_PREC_BF16 = 2
OFA_PREC_BF16X3 = 3
OFA_PREC_F16X3 = 4
PRECISIONS = {"fp32": OFA_PREC_FP32, "tf32": OFA_PREC_TF32, "bf16": OFA_PREC_BF16,
              "bf16x3": OFA_PREC_BF16X3, "f16x3": OFA_PREC_F16X3}

OFA_MEM_HOST = 0
OFA_MEM_DEVICE = 1


class ofa_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("seed", C.c_uint64), ("cuda_stream", C.c_void_p),
                ("amplitude", C.c_void_p), ("waist_frac", C.c_double), ("phi0", C.c_void_p),
                ("mem_space", C.c_int), ("weighting", C.c_int), ("autotune", C.c_int),
                ("focus_z", C.c_void_p), ("separable", C.c_int),
                ("kernel_config", C.c_int * 5), ("fused_loop", C.c_int),
                ("loop_config", C.c_int * 2), ("shard_row0", C.c_int),
                ("shard_ny_total", C.c_int), ("separable_loop", C.c_int),
                ("separable_tc", C.c_int)]


class ofa_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("xi", C.c_double), ("uniformity", C.c_double),
                ("sum_intensity", C.c_double), ("energy_fraction", C.c_double)]


# (name, restype, argtypes) of every symbol declared in include/ofa.h
_P = C.c_void_p
_I = C.c_int
_D = C.c_double
SIGNATURES = [
    ("ofa_options_default", _I, [C.POINTER(ofa_options)]),
    ("ofa_plan_create", _I, [C.POINTER(_P), _I, _I, _D, _D, _D, _D, _I, _P, _P,
                             C.POINTER(ofa_options)]),
    ("ofa_iterate", _I, [_P, _I, _D, C.POINTER(_I), C.POINTER(_D)]),
    ("ofa_get_phase", _I, [_P, _P, _I]),
    ("ofa_destroy", _I, [_P]),
    ("ofa_get_stats", _I, [_P, C.POINTER(ofa_stats)]),
    ("ofa_get_xi_history", _I, [_P, _P, _I, C.POINTER(_I)]),
    ("ofa_get_state", _I, [_P, _P, _P, C.POINTER(_I), _I]),
    ("ofa_set_state", _I, [_P, _P, _P, _I, _I]),
    ("ofa_forward", _I, [_P, _P, _P, _P]),
    ("ofa_adjoint", _I, [_P, _P, _P, _P, _P]),
    ("ofa_profile_kernels", _I, [_P, _I, _P]),
    ("ofa_plan_config", _I, [_P, _P]),
    ("ofa_profile_loop", _I, [_P, _I, _I, C.POINTER(_D), _P]),
    ("ofa_shard_forward", _I, [_P, _P]),
    ("ofa_loss_adjoint", _I, [_P, _P, _P, _P, _P, _I, _P]),
    ("ofa_adam_step", _I, [_P, _P, _P, _P, _P, _P, C.c_float, C.c_float, C.c_float, C.c_float]),
    ("ofa_shard_update", _I, [_P, _P]),
    ("ofa_plan_info", _I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    ("ofa_batch_create", _I, [C.POINTER(_P), C.POINTER(_P), _I, _P]),
    ("ofa_batch_iterate", _I, [_P, _I]),
    ("ofa_batch_destroy", _I, [_P]),
    ("ofa_batch_info", _I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    ("ofa_selftest_bounded_wait", _I, []),
    ("ofa_trim", _I, []),
    ("ofa_iterate_measured", _I, [_P, _P, _I, C.POINTER(_D)]),
    ("ofa_plan_form", _I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    ("ofa_forward_noalloc", _I, [_I, _I, _D, _D, _D, _D, _I, _P, _P, _P, _P, _P, _P]),
    ("ofa_fft_equivalent_size", _I, [_I, _D, _D, _D, _D, C.POINTER(_I)]),
    ("ofa_max_foci_per_axis", _I, [_D, _D, _D, _D, C.POINTER(_I)]),
    ("ofa_check_foci", _I, [_I, _P, _D, _D, _D, _D, C.POINTER(_I)]),
    ("ofa_status_string", C.c_char_p, [_I]),
    ("ofa_last_error", C.c_char_p, [_P]),
]


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libofa.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


class OfaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{ofa_status_string(status)}: {msg}")
        self.status = status


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return int(x.ctypes.data)
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _check(status: int, plan=None):
    if status != OFA_OK:
        raise OfaError(status, ofa_last_error(plan))


# ---------------------------------------------------------------- 1:1 wrappers
def ofa_status_string(status: int) -> str:
    return _lib.ofa_status_string(int(status)).decode()


def ofa_last_error(plan=None) -> str:
    return (_lib.ofa_last_error(plan) or b"").decode()


def ofa_options_default() -> ofa_options:
    o = ofa_options()
    _check(_lib.ofa_options_default(C.byref(o)))
    return o


def ofa_plan_create(nx, ny, pitch_x, pitch_y, wavelength, focal_length, focus_xy, target,
                    opt: ofa_options | None = None):
    """Returns the plan handle (int).  focus_xy / target follow opt.mem_space."""
    out = C.c_void_p()
    k = int(focus_xy.shape[0])
    st = _lib.ofa_plan_create(C.byref(out), int(nx), int(ny), float(pitch_x), float(pitch_y),
                              float(wavelength), float(focal_length), k, _ptr(focus_xy),
                              _ptr(target), C.byref(opt) if opt is not None else None)
    _check(st, None)
    return out.value


def ofa_iterate(plan, n_iter: int, threshold: float = 0.0, want_stats: bool = False):
    if not want_stats:
        _check(_lib.ofa_iterate(plan, int(n_iter), float(threshold), None, None), plan)
        return None
    it = C.c_int()
    xi = C.c_double()
    _check(_lib.ofa_iterate(plan, int(n_iter), float(threshold), C.byref(it), C.byref(xi)), plan)
    return it.value, xi.value


def ofa_iterate_measured(plan, measured, mem_space: int = OFA_MEM_HOST) -> float:
    """One camera-in-the-loop iteration; returns the captured intensities' xi."""
    if mem_space == OFA_MEM_HOST:
        measured = np.ascontiguousarray(measured, dtype=np.float32)
    xi = C.c_double()
    _check(_lib.ofa_iterate_measured(plan, _ptr(measured), int(mem_space), C.byref(xi)), plan)
    return xi.value


def ofa_get_phase(plan, out, mem_space: int):
    _check(_lib.ofa_get_phase(plan, _ptr(out), int(mem_space)), plan)


def ofa_destroy(plan):
    _check(_lib.ofa_destroy(plan), None)


def ofa_get_stats(plan) -> ofa_stats:
    s = ofa_stats()
    _check(_lib.ofa_get_stats(plan, C.byref(s)), plan)
    return s


def ofa_get_xi_history(plan, capacity: int = 65536) -> np.ndarray:
    buf = np.zeros(max(capacity, 1), dtype=np.float64)
    n = C.c_int()
    _check(_lib.ofa_get_xi_history(plan, _ptr(buf), int(capacity), C.byref(n)), plan)
    return buf[:min(n.value, capacity)].copy()


def ofa_get_state(plan, phi_out=None, w_out=None, mem_space: int = OFA_MEM_HOST) -> int:
    j = C.c_int()
    _check(_lib.ofa_get_state(plan, _ptr(phi_out), _ptr(w_out), C.byref(j), int(mem_space)), plan)
    return j.value


def ofa_set_state(plan, phi=None, w=None, j: int = 0, mem_space: int = OFA_MEM_HOST):
    _check(_lib.ofa_set_state(plan, _ptr(phi), _ptr(w), int(j), int(mem_space)), plan)


def ofa_forward(plan, phi, theta=None, intensity=None):
    _check(_lib.ofa_forward(plan, _ptr(phi), _ptr(theta), _ptr(intensity)), plan)


def ofa_loss_adjoint(plan, phi, theta, grad_phi, loss_hist=None, step=None):
    cap = int(loss_hist.numel()) if loss_hist is not None else 0
    _check(_lib.ofa_loss_adjoint(plan, _ptr(phi), _ptr(theta), _ptr(grad_phi), _ptr(loss_hist),
                                 cap, _ptr(step)), plan)


def ofa_adam_step(plan, phi, grad_phi, m, v, step, lr=0.05, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(_lib.ofa_adam_step(plan, _ptr(phi), _ptr(grad_phi), _ptr(m), _ptr(v), _ptr(step),
                              float(lr), float(beta1), float(beta2), float(eps)), plan)


def ofa_shard_forward(plan, theta_partial):
    _check(_lib.ofa_shard_forward(plan, _ptr(theta_partial)), plan)


def ofa_shard_update(plan, theta_total):
    _check(_lib.ofa_shard_update(plan, _ptr(theta_total)), plan)


def ofa_adjoint(plan, phi, theta, grad_intensity, grad_phi):
    _check(_lib.ofa_adjoint(plan, _ptr(phi), _ptr(theta), _ptr(grad_intensity), _ptr(grad_phi)),
           plan)


def ofa_profile_kernels(plan, reps: int = 20) -> np.ndarray:
    """[forward, focal, inverse-operand build, inverse] average ms per launch."""
    out = np.zeros(4, dtype=np.float64)
    _check(_lib.ofa_profile_kernels(plan, int(reps), _ptr(out)), plan)
    return out


def ofa_plan_config(plan) -> dict:
    c = np.zeros(12, dtype=np.int32)
    _check(_lib.ofa_plan_config(plan, _ptr(c)), plan)
    keys = ["fwd_bn", "fwd_split", "fwd_cta_group", "inv_bn", "inv_cta_group", "focal_fused",
            "fwd_row_bytes", "inv_row_bytes", "fused_loop", "loop_cta_group", "loop_split",
            "loop_ctas"]
    return dict(zip(keys, (int(x) for x in c)))


LOOP_PHASES = ["forward", "barrier_after_forward", "focal", "operand_build",
               "barrier_after_build", "inverse"]


def ofa_profile_loop(plan, n_iter: int = 20, reps: int = 5, phases: bool = False):
    """Average ms per iteration of the fused loop kernel (OFA_ERR_UNSUPPORTED if unused);
    with phases=True also the microseconds per iteration of each phase (a dict)."""
    ms = C.c_double()
    ph = np.zeros(6, dtype=np.float64) if phases else None
    _check(_lib.ofa_profile_loop(plan, int(n_iter), int(reps), C.byref(ms), _ptr(ph)), plan)
    if not phases:
        return ms.value
    return ms.value, dict(zip(LOOP_PHASES, (float(x) for x in ph)))


def ofa_plan_form(plan) -> dict:
    a, b, c = C.c_int(0), C.c_int(0), C.c_int(0)
    _check(_lib.ofa_plan_form(plan, C.byref(a), C.byref(b), C.byref(c)), plan)
    return {"separable": bool(a.value), "ux": b.value, "uy": c.value}


def ofa_plan_info(plan):
    a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(_lib.ofa_plan_info(plan, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), plan)
    return a.value, b.value, c.value, d.value


def ofa_batch_create(plans, stream=None):
    arr = (C.c_void_p * len(plans))(*plans)
    out = C.c_void_p()
    _check(_lib.ofa_batch_create(C.byref(out), arr, len(plans), stream))
    return out.value


def ofa_batch_iterate(batch, n_iter: int):
    _check(_lib.ofa_batch_iterate(batch, int(n_iter)))


def ofa_batch_destroy(batch):
    _check(_lib.ofa_batch_destroy(batch))


def ofa_trim():
    """Free the memory that destroyed plans left for reuse on the current device."""
    _check(_lib.ofa_trim())


def ofa_selftest_bounded_wait() -> int:
    """Run one bounded device wait that nothing ends; returns the raw status
    (OFA_ERR_TIMEOUT is the expected, healthy outcome)."""
    return int(_lib.ofa_selftest_bounded_wait())


def ofa_batch_info(batch) -> dict:
    g, f, i = C.c_int(0), C.c_int(0), C.c_int(0)
    _check(_lib.ofa_batch_info(batch, C.byref(g), C.byref(f), C.byref(i)))
    return {"grouped": bool(g.value), "fwd_bn": f.value, "inv_bn": i.value}


def ofa_forward_noalloc(nx, ny, pitch_x, pitch_y, wavelength, focal_length, focus_xy, phi,
                        amplitude, theta=None, intensity=None, stream=None):
    """Plan-free focal field at the foci; every array is a device pointer/tensor."""
    k = int(focus_xy.shape[0])
    _check(_lib.ofa_forward_noalloc(int(nx), int(ny), float(pitch_x), float(pitch_y),
                                    float(wavelength), float(focal_length), k, _ptr(focus_xy),
                                    _ptr(phi), _ptr(amplitude), _ptr(theta), _ptr(intensity),
                                    stream))


def ofa_fft_equivalent_size(m0, pitch, wavelength, focal_length, focal_sampling) -> int:
    m = C.c_int()
    _check(_lib.ofa_fft_equivalent_size(int(m0), float(pitch), float(wavelength),
                                        float(focal_length), float(focal_sampling), C.byref(m)))
    return m.value


def ofa_max_foci_per_axis(pitch, wavelength, focal_length, gap) -> int:
    n = C.c_int()
    _check(_lib.ofa_max_foci_per_axis(float(pitch), float(wavelength), float(focal_length),
                                      float(gap), C.byref(n)))
    return n.value


def ofa_check_foci(focus_xy, pitch_x, pitch_y, wavelength, focal_length):
    """Returns (status, bad_index) without raising."""
    xy = np.ascontiguousarray(focus_xy, dtype=np.float64)
    bad = C.c_int()
    st = _lib.ofa_check_foci(int(xy.shape[0]), _ptr(xy), float(pitch_x), float(pitch_y),
                             float(wavelength), float(focal_length), C.byref(bad))
    return st, bad.value


# ---------------------------------------------------------------- convenience
class Plan:
    """Owns one ofa_plan*.  Host numpy inputs; stream = torch stream handle (int) or None."""

    def __init__(self, nx, ny, pitch_x, pitch_y, wavelength, focal_length, focus_xy, target,
                 precision="f16x3", amplitude=None, phi0=None, seed=0, weighting=True,
                 stream=None, waist_frac=0.4, mem_space=OFA_MEM_HOST, autotune=True,
                 focus_z=None, separable=-1, kernel_config=None, fused_loop=None,
                 loop_config=None, shard=None, separable_loop=None, separable_tc=None):
        opt = ofa_options_default()
        opt.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        opt.seed = int(seed)
        opt.cuda_stream = stream
        opt.weighting = 1 if weighting else 0
        opt.autotune = 1 if autotune else 0
        opt.separable = int(separable)
        if shard is not None:           # (row0, ny_total): rows [row0, row0 + ny)
            opt.shard_row0, opt.shard_ny_total = int(shard[0]), int(shard[1])
        if fused_loop is not None:
            opt.fused_loop = int(fused_loop)
        if separable_loop is not None:
            opt.separable_loop = int(separable_loop)
        if separable_tc is not None:
            opt.separable_tc = int(separable_tc)
        if loop_config is not None:
            opt.loop_config[0], opt.loop_config[1] = int(loop_config[0]), int(loop_config[1])
        if kernel_config is not None:
            for i, v in enumerate(kernel_config):
                opt.kernel_config[i] = int(v)
        opt.waist_frac = float(waist_frac)
        opt.mem_space = int(mem_space)
        if mem_space == OFA_MEM_HOST:
            focus_xy = np.ascontiguousarray(focus_xy, dtype=np.float64)
            target = np.ascontiguousarray(target, dtype=np.float32)
            if amplitude is not None:
                amplitude = np.ascontiguousarray(amplitude, dtype=np.float32)
            if phi0 is not None:
                phi0 = np.ascontiguousarray(phi0, dtype=np.float32)
            if focus_z is not None:
                focus_z = np.ascontiguousarray(focus_z, dtype=np.float64)
        self._keep = (focus_xy, target, amplitude, phi0, focus_z)
        opt.amplitude = _ptr(amplitude)
        opt.phi0 = _ptr(phi0)
        opt.focus_z = _ptr(focus_z)
        self.nx, self.ny, self.K = int(nx), int(ny), int(focus_xy.shape[0])
        self.handle = ofa_plan_create(nx, ny, pitch_x, pitch_y, wavelength, focal_length,
                                      focus_xy, target, opt)
        # the stream the caller gave (None or 0: a stream the library created)
        self.stream = int(stream) if stream else None
        self._keep = None

    @classmethod
    def from_workload(cls, w, **kw):
        if getattr(w, "focus_z", None) is not None:
            kw.setdefault("focus_z", w.focus_z)
        return cls(w.nx, w.ny, w.pitch_x, w.pitch_y, w.wavelength, w.focal_length, w.focus_xy,
                   w.target, amplitude=w.amplitude, phi0=w.phi0, **kw)

    def iterate(self, n_iter, threshold=0.0, want_stats=False):
        return ofa_iterate(self.handle, n_iter, threshold, want_stats)

    def phase(self) -> np.ndarray:
        out = np.empty((self.ny, self.nx), dtype=np.float32)
        ofa_get_phase(self.handle, out, OFA_MEM_HOST)
        return out

    def stats(self) -> ofa_stats:
        return ofa_get_stats(self.handle)

    def xi_history(self) -> np.ndarray:
        return ofa_get_xi_history(self.handle)

    def get_state(self):
        phi = np.empty((self.ny, self.nx), dtype=np.float32)
        w = np.empty(self.K, dtype=np.float32)
        j = ofa_get_state(self.handle, phi, w, OFA_MEM_HOST)
        return phi, w, j

    def set_state(self, phi=None, w=None, j=0):
        phi = None if phi is None else np.ascontiguousarray(phi, dtype=np.float32)
        w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
        ofa_set_state(self.handle, phi, w, j, OFA_MEM_HOST)

    def close(self):
        if getattr(self, "handle", None):
            ofa_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
