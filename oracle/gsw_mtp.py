"""FP64 CPU oracle of the GSW-MTP focus-array loop (arXiv 2206.12661).

TEST INFRASTRUCTURE.  Only the tests, the smoke check of the package entry
file and the CPU-baseline leg of the benchmark may import this module.  The
CUDA library never calls it, and it shares no code, table or constant
generator with the CUDA path.

Everything here is plain complex128 numpy in the paper's notation, one small
function per quantity, so that a reader can check each against the text:

* Eq. 1 / Eq. 2 -- far-field propagation written as a matrix triple product
  Theta = Omega_y E Omega_x, evaluated only at the foci (zero elements of the
  focal plane removed).  Per focus k this is
  Theta_k = sum_n Fy[k,n] sum_m E[n,m] Fx[k,m] with
  Fx[k,m] = exp(-i 2 pi x_k u_m / (lambda f)) and Fy[k,n] likewise in y.
* Results and discussion section -- the GSW weighting generalized to
  nonuniform targets: one cycle (gsw_step) is forward operator, intensities,
  intensity accuracy xi, weight update w sqrt(I~/I), focal amplitude
  constraint w sqrt(I~) exp(i arg Theta), inverse operator, pupil amplitude
  constraint (phase only); gsw() repeats it until xi passes a threshold.

Readings where the paper is silent or loose (the same list is kept in the
design notes of the repository):

* inverse propagation is the adjoint of Eq. 2 (the paper says the inverse is
  "formulated similarly"; Omega is not square, so no true inverse exists);
  any positive scale in front of it drops out of arg().
* spatial frequency k_x = u / (lambda f) for pupil coordinate u (Fourier lens);
  pupil coordinates are centred, u_m = (m - (N-1)/2) p.
* target and computed intensities are both normalised to unit sum before
  they enter xi and the weight update (a global factor on w changes nothing
  that arg() sees).
* xi uses the Euclidean norm over the foci; its denominator is the computed
  intensity, as printed in Algorithm 1.
* arg(0) = 0 (atan2 convention); I_k is clamped to 1e-30 in the update.
* one iteration = forward, statistics, weight update, inverse, projection;
  the final xi of a run comes from one extra forward after the last inverse.

Parity status: every function below is pinned by the CPU tests against
something other than itself (FFT equivalence, brute force, single-focus
closed form, Parseval, adjoint identity, invariances, a textbook uniform-GSW
restatement, finite differences, a published splitmix64 vector).
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


# ---------------------------------------------------------------- geometry
def pupil_coords(n: int, pitch: float) -> np.ndarray:
    """Centred pupil sample positions u_m = (m - (n-1)/2) * pitch (metres)."""
    return (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * float(pitch)


def dft_rows(focal: np.ndarray, pupil: np.ndarray, lam_f: float, focus_z=None,
             focal_length=None) -> np.ndarray:
    """Rows of the arbitrarily sampled DFT matrix of Eq. 2 at the foci.

    Omega[k, m] = exp(-i 2 pi focal_k * pupil_m / (lambda f)): the exponent of
    Eq. 1 with spatial frequency pupil_m / (lambda f), one row per focus.

    3D foci (the axial position of a spot set by a defocus phase of the pupil
    function, Conclusion and outlook section): with axial offsets z_k the pupil field seen by focus k
    carries the paraxial (Fresnel) defocus exp(-i pi z_k (u^2 + v^2) / (lambda f^2)),
    whose u and v factors fold into the two rows:
    Omega[k, m] *= exp(-i pi z_k pupil_m^2 / (lambda f^2)).
    """
    focal = np.asarray(focal, dtype=np.float64)
    pupil = np.asarray(pupil, dtype=np.float64)
    arg = TWO_PI * np.outer(focal, pupil) / float(lam_f)
    if focus_z is not None:
        lam_f2 = float(lam_f) * float(focal_length)
        arg = arg + np.pi * np.outer(np.asarray(focus_z, np.float64), pupil ** 2) / lam_f2
    return np.exp(-1j * arg)


def plan_matrices(nx, ny, pitch_x, pitch_y, wavelength, focal_length, focus_xy, focus_z=None):
    """Fx [K][nx] and Fy [K][ny] for a centred pupil and foci (x_k, y_k[, z_k])."""
    lam_f = float(wavelength) * float(focal_length)
    focus_xy = np.asarray(focus_xy, dtype=np.float64)
    fx = dft_rows(focus_xy[:, 0], pupil_coords(nx, pitch_x), lam_f, focus_z, focal_length)
    fy = dft_rows(focus_xy[:, 1], pupil_coords(ny, pitch_y), lam_f, focus_z, focal_length)
    return fx, fy


# ------------------------------------------------------------- propagation
def pupil_field(amplitude: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """E = A exp(i phi): the pupil function of Eq. 1."""
    return np.asarray(amplitude, np.float64) * np.exp(1j * np.asarray(phi, np.float64))


def forward(E: np.ndarray, fx: np.ndarray, fy: np.ndarray) -> np.ndarray:
    """Forward MTP at the foci (Eq. 2): Theta_k = sum_n Fy[k,n] (E Fx^T)[n,k].

    E is [ny][nx] (rows along y), fx [K][nx], fy [K][ny]; returns Theta [K].
    """
    G = np.asarray(E, np.complex128) @ fx.T          # G[n, k] = sum_m E[n,m] Fx[k,m]
    return np.sum(fy * G.T, axis=1)                  # Theta_k = sum_n Fy[k,n] G[n,k]


def adjoint(theta: np.ndarray, fx: np.ndarray, fy: np.ndarray) -> np.ndarray:
    """Inverse MTP read as the adjoint of Eq. 2, focal samples off the foci = 0.

    E'[n,m] = sum_k conj(Fy[k,n]) Theta_k conj(Fx[k,m]); returns [ny][nx].
    """
    left = np.conj(fy).T * np.asarray(theta, np.complex128)[None, :]   # [ny][K]
    return left @ np.conj(fx)


def phase_projection(E: np.ndarray) -> np.ndarray:
    """phi = arg(E) in (-pi, pi], with arg(0) = 0: the phase-only CGH (pupil amplitude
    constraint)."""
    return np.arctan2(E.imag, E.real)


# ------------------------------------------------------------- statistics
def normalise(v: np.ndarray) -> np.ndarray:
    v = np.asarray(v, np.float64)
    return v / v.sum()


def intensity_accuracy(target: np.ndarray, intensity: np.ndarray) -> float:
    """Intensity accuracy xi = 1 - ||I~ - I|| / ||I|| over the foci, both normalised to
    unit sum (the accuracy measure of the Results and discussion section)."""
    t = normalise(target)
    i = normalise(intensity)
    return float(1.0 - np.linalg.norm(t - i) / np.linalg.norm(i))


def uniformity(target: np.ndarray, intensity: np.ndarray) -> float:
    """U = 1 - (max r - min r)/(max r + min r), r_k = I_k / I~_k over foci with I~_k > 0.

    Not defined in the paper; for uniform targets it is the usual
    1 - (Imax - Imin)/(Imax + Imin).
    """
    t = normalise(target)
    i = normalise(intensity)
    r = i[t > 0] / t[t > 0]
    return float(1.0 - (r.max() - r.min()) / (r.max() + r.min()))


# ------------------- generalized weighting (Results and discussion section)
IHAT_FLOOR = 1e-30


def generalized_weights(w: np.ndarray, target: np.ndarray, intensity: np.ndarray) -> np.ndarray:
    """Generalized weighting w_j = w_{j-1} sqrt(I~ / I), both intensities at unit sum."""
    t = normalise(target)
    i = np.maximum(normalise(intensity), IHAT_FLOOR)
    return np.asarray(w, np.float64) * np.sqrt(t / i)


def focused_field(w: np.ndarray, target: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Focal amplitude constraint: w sqrt(I~) exp(i arg Theta), arg(0) = 0."""
    t = normalise(target)
    psi = np.arctan2(theta.imag, theta.real)
    return np.asarray(w, np.float64) * np.sqrt(t) * np.exp(1j * psi)


def camera_step(amplitude, phi, fx, fy, target, w, measured):
    """One cycle of the camera-in-the-loop mode (experiments of the Results and
    discussion section): gsw_step with the calculated intensities replaced by captured
    ones in the weight update; the focused field keeps the phase of the calculated
    Theta (a camera records intensities only).  Returns (phi, w, xi of the
    measurement)."""
    A = np.asarray(amplitude, np.float64)
    theta = forward(pupil_field(A, phi), fx, fy)
    meas = np.asarray(measured, np.float64)
    xi = intensity_accuracy(target, meas)
    w = generalized_weights(w, target, meas)
    field = focused_field(w, target, theta)
    return phase_projection(adjoint(field, fx, fy)), w, xi


# ----------------------------------------------------------- the GSW loop
def gsw_step(amplitude, phi, w, fx, fy, target, weighting=True):
    """One cycle of the method (Results and discussion section: generalized weighting
    with the MTP operator), from the CGH phase phi and the weights w.

    The pupil function A exp(i phi) goes to the foci through the forward operator of
    Eq. 2, giving complex amplitudes Theta and intensities I = |Theta|^2.  With the
    target and calculated intensities the weights are updated, w <- w sqrt(I~/I)
    (generalized weighting; weighting=False keeps them, which is plain GS).  The
    focal-plane amplitude constraint replaces each focus amplitude by
    w sqrt(I~) and keeps the phase of Theta; the inverse operator brings that field
    back to the pupil, where the pupil amplitude constraint keeps only its phase.

    Returns (theta, intensity, xi, w_new, phi_new); xi is the intensity accuracy of
    the forward that starts the cycle.
    """
    theta = forward(pupil_field(amplitude, phi), fx, fy)
    intensity = np.abs(theta) ** 2
    xi = intensity_accuracy(target, intensity)
    w_new = generalized_weights(w, target, intensity) if weighting else np.asarray(w, np.float64)
    back = adjoint(focused_field(w_new, target, theta), fx, fy)
    return theta, intensity, xi, w_new, phase_projection(back)


def gsw(amplitude, phi0, fx, fy, target, n_iter, threshold=None, weighting=True, w0=None,
        record=False):
    """Drive gsw_step from phi0 for n_iter cycles in FP64.

    The run stops early once the intensity accuracy of a cycle's forward exceeds
    `threshold` (that cycle then makes no update), as the method iterates "until the
    intensity accuracy reaches the threshold value".  Returns a dict with the final
    phase 'phi', weights 'w', the accuracy of the forward that started each cycle
    'xi_hist', the cycles completed 'iters', and the statistics of one extra
    forward at the final phase: 'theta', 'intensity', 'xi', 'uniformity'.
    weighting=False is the plain GS loop (w stays 1).
    """
    A = np.asarray(amplitude, np.float64)
    phi = np.asarray(phi0, np.float64).copy()
    K = fx.shape[0]
    w = np.ones(K) if w0 is None else np.asarray(w0, np.float64).copy()
    xi_hist, phis = [], []
    iters = 0
    while iters < int(n_iter):
        _, _, xi, w_next, phi_next = gsw_step(A, phi, w, fx, fy, target, weighting)
        xi_hist.append(xi)
        if threshold is not None and xi > threshold:
            break
        phi, w = phi_next, w_next
        iters += 1
        if record:
            phis.append(phi.copy())
    theta = forward(pupil_field(A, phi), fx, fy)
    intensity = np.abs(theta) ** 2
    out = {"phi": phi, "w": w, "xi_hist": np.asarray(xi_hist), "iters": iters,
           "theta": theta, "intensity": intensity,
           "xi": intensity_accuracy(target, intensity),
           "uniformity": uniformity(target, intensity)}
    if record:
        out["phis"] = phis
    return out


# ------------------------------------------------ gradient (differentiation)
def intensity_loss(target, intensity) -> float:
    """L = sum_k (I_k / sum I - t_k)^2 with t = I~ / sum I~."""
    return float(np.sum((normalise(intensity) - normalise(target)) ** 2))


def intensity_loss_grad_I(target, intensity) -> np.ndarray:
    """dL/dI_k = (2/S) [(Ihat_k - t_k) - sum_j (Ihat_j - t_j) Ihat_j], S = sum I."""
    i = np.asarray(intensity, np.float64)
    S = i.sum()
    ih = i / S
    d = ih - normalise(target)
    return (2.0 / S) * (d - np.sum(d * ih))


def phase_gradient(amplitude, phi, fx, fy, grad_I) -> np.ndarray:
    """dL/dphi for L(I(phi)) given g = dL/dI: 2 Im(conj(E) B), B = adjoint(g * Theta)."""
    E = pupil_field(amplitude, phi)
    theta = forward(E, fx, fy)
    B = adjoint(np.asarray(grad_I, np.float64) * theta, fx, fy)
    return 2.0 * np.imag(np.conj(E) * B)


# ------------------------------------------------ library default inputs
def default_amplitude(nx, ny, pitch_x, pitch_y, waist_frac=0.4) -> np.ndarray:
    """Gaussian beam A = exp(-(u^2/wx^2 + v^2/wy^2)), w = waist_frac * N * p per axis."""
    u = pupil_coords(nx, pitch_x)
    v = pupil_coords(ny, pitch_y)
    wx = waist_frac * nx * pitch_x
    wy = waist_frac * ny * pitch_y
    return np.exp(-(v[:, None] ** 2 / wy ** 2 + u[None, :] ** 2 / wx ** 2))


_MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One splitmix64 output for state x (Steele, Lea and Flood, OOPSLA 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def default_phase(nx, ny, seed) -> np.ndarray:
    """Counter-based initial guess: phi0[i] = 2 pi (splitmix64(seed + i*gamma) >> 11) / 2^53 - pi.

    gamma is splitmix64's increment 0x9E3779B97F4A7C15; i is the row-major
    pixel index.  (The paper leaves the initial guess open.)
    """
    gamma = 0x9E3779B97F4A7C15
    out = np.empty(nx * ny, dtype=np.float64)
    for i in range(nx * ny):
        v = splitmix64((int(seed) + i * gamma) & _MASK64)
        out[i] = (v >> 11) * (1.0 / 9007199254740992.0) * TWO_PI - np.pi
    return out.reshape(ny, nx)
