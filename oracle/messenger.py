"""Algorithm 1 (messenger-field Wiener sampler) and its G -> 0 Wiener-filter variant, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``). The steps follow §2.2 in the paper's order, with
A = I (§3.2) and the messenger covariance T = lambda * tau * I, where tau = min observed noise variance
(Alg. 1 definitions) and N_bar = N - tau * I is kept fixed (the lambda-cooling reading below).

Per sweep (Alg. 1):
  1. pixel space, every pixel i:  t_i = mu_t + sqrt(var_t) * G,
       mu_t  = (T d_i + N_bar_i s_i) / (T + N_bar_i),  var_t = T N_bar_i / (T + N_bar_i)   (observed)
       mu_t  = s_i,                                      var_t = T                         (missing pixel,
       the exact N_bar -> infinity limit of the same formulas; §1.1 treats missing data as infinite noise)
  2. t_hat = U t                                           (unitary 2D DFT)
  3. Fourier space, every mode k:  s_hat_k = mu_s + sqrt(var_s) * zeta_k,
       mu_s = P_k / (P_k + T) * t_hat_k,   var_s = P_k T / (P_k + T)
     (the variance line of Alg. 1 is labelled sigma^t_hat but is the s_hat variance used in the update;
     zeta is the unitary DFT of real white noise so that s stays real)
  4. s = U^dagger s_hat  (real part; the imaginary part is round-off)

G -> 0 (§2.2, after Alg. 1) turns the sweep into a fixed-point iteration whose limit at lambda = 1 is the
Wiener filter of Eq. 2-3. At messenger level lambda its limit is the Wiener filter with noise
N + (lambda - 1) tau I (the joint density with T = lambda tau and fixed N_bar has marginal noise
N_bar + T); the cooling schedule only changes how fast lambda = 1 is reached, not the answer.

Noise layout (identical on the GPU; see ``oracle.philox``):
  * t-draw: stream 0, counter group j = (y*W + x) // 4, variate slot (y*W + x) % 4;
  * s-draw: stream 1. One counter group feeds a mode and its mirror (ky, H - ky) of one column.
    Interior columns kx in (0, W/2): group g = kx*(H/2) + j for j in [0, H/2); group j = 0 feeds the
    modes ky = 0 (z0, z1) and ky = H/2 (z2, z3); group j > 0 feeds ky = j (z0, z1) and ky = H - j
    (z2, z3); zeta = (Re + i Im)/sqrt(2).
    Edge columns kx in {0, W/2} (Hermitian within the column): group g = j for j in (0, H/2) feeds
    zeta = (z0 + i z1)/sqrt(2) at (j, 0) and (z2 + i z3)/sqrt(2) at (j, W/2); the modes H - j take the
    complex conjugates; group 0 feeds the four self-conjugate modes with real, unit-variance zeta:
    z0 -> (0, 0), z1 -> (H/2, 0), z2 -> (0, W/2), z3 -> (H/2, W/2).
    kx > W/2 is the Hermitian image of (H - ky, W - kx).
  * counter step for sweep i of a call is ``start_step + i``; chain id is the third counter word.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

from . import dft
from .philox import STREAM_S, STREAM_T, normals4


# ----------------------------------------------------------------------------------------------
# problem set-up (Alg. 1 definitions of T and N_bar)
# ----------------------------------------------------------------------------------------------
def default_tau(Ndiag: np.ndarray, mask: np.ndarray, Pk: np.ndarray, A=None) -> float:
    """tau = min over observed pixels of N_i / A_i^2 (Alg. 1: T = min((A^-1)^dagger N A^-1) I; A = I by
    default). Pixels with A_i = 0 carry no data and are left out like missing pixels.

    With no observed pixel the data carry no information and any tau > 0 gives a valid sampler;
    this code base then takes tau = max_k P_k (1 if P = 0), which makes each sweep close to an exact
    prior draw.
    """
    obs = np.asarray(mask) == 0
    N = np.asarray(Ndiag, dtype=np.float64)
    if A is not None:
        A = np.asarray(A, dtype=np.float64)
        obs = obs & (A != 0)
        N = N / np.where(obs, A * A, 1.0)
    if np.any(obs):
        return float(np.min(N[obs]))
    pmax = float(np.max(Pk))
    return pmax if pmax > 0 else 1.0


def _fields(d, Ndiag, mask, Pk, A=None):
    d = np.asarray(d, dtype=np.float64)
    N = np.asarray(Ndiag, dtype=np.float64)
    m = np.asarray(mask) != 0
    if A is not None:
        m = m | (np.asarray(A) == 0)   # A_i = 0: no data at pixel i (the A_i^2 > 0 condition of Alg. 1)
    H, W = d.shape
    Pfull = dft.half_to_full(np.asarray(Pk, dtype=np.float64), W)
    return d, N, m, Pfull


def pixel_update(s, d, N, miss, tau, lam, xi=None, A=None):
    """Alg. 1 step 1 with T = lam*tau; ``xi`` = G(0,1) per pixel or None (G -> 0).

    A = I: N_bar = N - tau, mu_t = (T d + N_bar s) / (T + N_bar), var_t = T N_bar / (T + N_bar).
    Diagonal response A (Alg. 1 definitions, pixels with A_i^2 > 0): N_bar = N - A^2 tau,
    mu_t = T A d / (T A^2 + N_bar) + N_bar s / (T A^2 + N_bar), var_t = T N_bar / (T A^2 + N_bar).
    """
    T = lam * tau
    if A is None:
        Nbar = np.where(miss, 0.0, N - tau)
        denom = np.where(miss, 1.0, T + Nbar)
        mu = np.where(miss, s, (T * d + Nbar * s) / denom)
    else:
        A = np.asarray(A, dtype=np.float64)
        # N_bar >= 0 by the definition of T (min of N / A^2); the clamp only removes rounding at the minimum
        Nbar = np.where(miss, 0.0, np.maximum(N - A * A * tau, 0.0))
        denom = np.where(miss, 1.0, T * A * A + Nbar)
        mu = np.where(miss, s, T * A * d / denom + Nbar * s / denom)
    if xi is None:
        return mu
    var = np.where(miss, T, T * Nbar / denom)
    return mu + np.sqrt(var) * xi


def fourier_update(t, Pfull, tau, lam, zeta=None):
    """Alg. 1 steps 2-4: t_hat = U t, s_hat = mu_s + sqrt(var_s) zeta, s = U^dagger s_hat."""
    T = lam * tau
    th = dft.dft2(t)
    sh = Pfull / (Pfull + T) * th
    if zeta is not None:
        sh = sh + np.sqrt(Pfull * T / (Pfull + T)) * zeta
    s = dft.idft2(sh)
    assert np.max(np.abs(s.imag)) <= 1e-9 * max(1.0, float(np.max(np.abs(s.real)))), "lost Hermitian symmetry"
    return s.real


# ----------------------------------------------------------------------------------------------
# Gaussian variates in the counter layout shared with the GPU
# ----------------------------------------------------------------------------------------------
def draw_xi(seed: int, chain: int, step: int, H: int, W: int, stream: int = STREAM_T) -> np.ndarray:
    """Pixel-space G(0,1) field [H][W] for one sweep (stream 0 by default)."""
    groups = np.arange(H * W // 4)
    z = normals4(groups, step, chain, stream, seed)
    return z.reshape(H, W)


@lru_cache(maxsize=None)
def _zeta_layout(H: int, W: int):
    """Index maps of the s-draw layout on the half-spectrum [H][W//2+1] (see module docstring).

    Returns (group, re_slot, im_slot, kind) arrays of shape [H][W//2+1]: the counter group and the
    variate slots for Re and Im of each mode, and kind = 0 complex, 1 self-conjugate (real, Re slot
    only), 2 conjugate image of the mode at H - ky in the same column.
    """
    Hh, Wh = H // 2, W // 2
    group = np.zeros((H, Wh + 1), dtype=np.int64)
    re_slot = np.zeros((H, Wh + 1), dtype=np.int64)
    im_slot = np.zeros((H, Wh + 1), dtype=np.int64)
    kind = np.zeros((H, Wh + 1), dtype=np.int64)
    for kx in range(Wh + 1):
        for ky in range(H):
            if 0 < kx < Wh:                       # interior column: group pairs ky with H - ky
                j = ky if ky < Hh else (0 if ky == Hh else H - ky)
                first = ky < Hh
                group[ky, kx] = kx * Hh + j
                re_slot[ky, kx], im_slot[ky, kx] = (0, 1) if first else (2, 3)
            else:                                 # edge column, Hermitian in ky
                e = 0 if kx == 0 else 1
                if ky == 0 or ky == Hh:
                    group[ky, kx] = 0
                    re_slot[ky, kx] = 2 * e + (0 if ky == 0 else 1)
                    kind[ky, kx] = 1
                elif ky < Hh:
                    group[ky, kx] = ky
                    re_slot[ky, kx], im_slot[ky, kx] = 2 * e, 2 * e + 1
                else:
                    kind[ky, kx] = 2
    for a in (group, re_slot, im_slot, kind):
        a.setflags(write=False)
    return group, re_slot, im_slot, kind


def draw_zeta(seed: int, chain: int, step: int, H: int, W: int, stream: int = STREAM_S) -> np.ndarray:
    """Hermitian complex white noise on the full spectrum [H][W] for one sweep (stream 1 by default)."""
    Hh, Wh = H // 2, W // 2
    group, re_slot, im_slot, kind = _zeta_layout(H, W)
    z = normals4(np.arange(Wh * Hh), step, chain, stream, seed)            # [(W/2)*(H/2), 4]
    re = z[group, re_slot]
    im = z[group, im_slot]
    half = (re + 1j * im) / math.sqrt(2.0)
    half = np.where(kind == 1, re + 0j, half)
    mirror = half[(H - np.arange(H)) % H, :]                # row H - ky of the same column
    half = np.where(kind == 2, np.conj(mirror), half)
    full = np.empty((H, W), dtype=np.complex128)
    full[:, : Wh + 1] = half
    kxs = np.arange(Wh + 1, W)
    full[:, kxs] = np.conj(half[(H - np.arange(H))[:, None] % H, (W - kxs)[None, :]])
    return full


# ----------------------------------------------------------------------------------------------
# Algorithm 1: the sampler
# ----------------------------------------------------------------------------------------------
def sample(d, Ndiag, mask, Pk, n_samples: int, seed: int, *, chain: int = 0, tau: float | None = None,
           start_step: int = 0, burn_in: int = 0, thin: int = 1, init_s=None, A=None) -> np.ndarray:
    """Draw ``n_samples`` posterior samples from one chain -> float64 [n_samples][H][W].

    The chain starts at ``init_s`` (zero if None) and performs burn_in + n_samples*thin sweeps; sample m
    is the state after sweep burn_in + (m+1)*thin. Sweep i uses counter step ``start_step + i``.
    """
    d, N, miss, Pfull = _fields(d, Ndiag, mask, Pk, A)
    H, W = d.shape
    if tau is None:
        tau = default_tau(N, miss, Pk, A)
    s = np.zeros((H, W)) if init_s is None else np.asarray(init_s, dtype=np.float64).copy()
    out = np.empty((n_samples, H, W))
    n_sweeps = burn_in + n_samples * thin
    m = 0
    for i in range(n_sweeps):
        step = start_step + i
        t = pixel_update(s, d, N, miss, tau, 1.0, draw_xi(seed, chain, step, H, W), A)
        s = fourier_update(t, Pfull, tau, 1.0, draw_zeta(seed, chain, step, H, W))
        done = i + 1
        if done > burn_in and (done - burn_in) % thin == 0:
            out[m] = s
            m += 1
    return out


# ----------------------------------------------------------------------------------------------
# G -> 0: Wiener filter with lambda-cooling
# ----------------------------------------------------------------------------------------------
def apply_S(v, Pfull):
    """S v = U^dagger diag(P) U v (Eq. 7: S is diagonal in Fourier space)."""
    return dft.idft2(Pfull * dft.dft2(v)).real


def residual(s, d, Ndiag, mask, Pk, tau: float | None = None, lam: float = 1.0, A=None) -> float:
    """Relative residual of the Wiener-filter equation at messenger level lambda.

    The Wiener filter s_W = S (S + N)^-1 d (Eq. 2-3, A = I) solves (I + S N^-1) s = S N^-1 d, with
    N^-1 = 0 on missing pixels. Returns ||s + S N^-1 (s - d)|| / ||S N^-1 d|| for noise
    N + (lambda - 1) tau I (lambda = 1: the Wiener filter itself). With a diagonal response A the
    equation is (I + S A N^-1 A) s = S A N^-1 d and the level-lambda noise N + (lambda - 1) tau A^2.
    """
    d, N, miss, Pfull = _fields(d, Ndiag, mask, Pk, A)
    if tau is None:
        tau = default_tau(N, miss, Pk, A)
    Av = np.ones_like(d) if A is None else np.asarray(A, dtype=np.float64)
    Ninv = np.where(miss, 0.0, 1.0 / np.where(miss, 1.0, N + (lam - 1.0) * tau * Av * Av))
    s = np.asarray(s, dtype=np.float64)
    b = apply_S(Av * Ninv * d, Pfull)
    r = s + apply_S(Av * Ninv * (Av * s - d), Pfull)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(r) / nb) if nb > 0 else float(np.linalg.norm(r))


class CoolingSchedule:
    """lambda-cooling for the G -> 0 iteration (reading of §2.2; the schedule itself is not in the paper).

    lambda_0 = max(1, max_k P_k / tau); after every ``check`` sweeps at level lambda the level residual
    rho_lambda is measured; the level ends when rho_lambda < ``level_tol`` or after ``level_max`` sweeps,
    and lambda <- max(1, eta * lambda). At lambda = 1 the iteration stops when rho < tol, or at max_iter.
    """

    def __init__(self, eta: float = 0.5, level_tol: float = 1e-2, level_max: int = 64, check: int = 1):
        self.eta = eta
        self.level_tol = level_tol
        self.level_max = level_max
        self.check = check

    def lambda0(self, Pk, tau: float) -> float:
        return max(1.0, float(np.max(Pk)) / tau)


def wf_solve(d, Ndiag, mask, Pk, tau: float | None = None, tol: float = 1e-6, max_iter: int = 100000,
             schedule: CoolingSchedule | None = None, init_s=None, return_history: bool = False, A=None):
    """Wiener filter by the G -> 0 messenger iteration with lambda-cooling.

    Returns (s, iters, rho) with rho the final lambda = 1 relative residual (see :func:`residual`).
    """
    d, N, miss, Pfull = _fields(d, Ndiag, mask, Pk, A)
    H, W = d.shape
    if tau is None:
        tau = default_tau(N, miss, Pk, A)
    sch = schedule or CoolingSchedule()
    lam = sch.lambda0(Pk, tau)
    s = np.zeros((H, W)) if init_s is None else np.asarray(init_s, dtype=np.float64).copy()
    it = 0
    level_it = 0
    hist = []
    rho = residual(s, d, N, miss, Pk, tau, 1.0, A)
    while it < max_iter:
        t = pixel_update(s, d, N, miss, tau, lam, None, A)
        s = fourier_update(t, Pfull, tau, lam)
        it += 1
        level_it += 1
        if level_it % sch.check:
            continue
        if lam > 1.0:
            rl = residual(s, d, N, miss, Pk, tau, lam, A)
            hist.append((it, lam, rl))
            if rl < sch.level_tol or level_it >= sch.level_max:
                lam = max(1.0, sch.eta * lam)
                level_it = 0
        else:
            rho = residual(s, d, N, miss, Pk, tau, 1.0, A)
            hist.append((it, lam, rho))
            if rho < tol:
                break
    if lam > 1.0 or it == 0:
        rho = residual(s, d, N, miss, Pk, tau, 1.0, A)
    if return_history:
        return s, it, rho, hist
    return s, it, rho
