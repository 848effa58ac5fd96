"""Seeded synthetic inputs shaped like the paper's workloads (§3.2, data model of Eq. 1 with A = I).

This module only *makes inputs*: a Gaussian random field with a chosen power spectrum, a spatially
varying noise-variance map, a mask of missing pixels, and the data d = s + n. It contains none of the
messenger-field arithmetic (no Wiener filter, no Gibbs step, no Philox) and imports neither the CUDA
binding nor the oracle, so both sides of every parity test can use it.

Conventions shared by every caller:

* images are row-major float32 ``[H][W]``; the mask is uint8 ``[H][W]`` with 1 = missing pixel;
* ``Pk`` is float32 ``[H][W//2+1]`` on the half-spectrum grid (ky in FFT order, kx = 0..W/2) and holds
  the variance of the *unitary* 2D DFT coefficient of the signal at that mode, so a field with flat
  ``Pk = 1`` has unit pixel variance;
* wavenumbers are in cycles per pixel: ``k = sqrt((ky/H)^2 + (kx/W)^2)`` with ky folded to [-1/2, 1/2);
* the DC mode has ``P = 0`` (zero-mean signal, §1.1);
* randomness comes from ``numpy.random.default_rng(seed)``, independent of the method's Philox draws.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class WFProblem:
    """One image of the data model d = s + n (Eq. 1 with A = I) plus the known covariances."""

    d: np.ndarray          # float32 [H][W], masked pixels set to 0
    Ndiag: np.ndarray      # float32 [H][W], noise variance (ignored where mask = 1)
    mask: np.ndarray       # uint8   [H][W], 1 = missing data (infinite noise, §1.1)
    Pk: np.ndarray         # float32 [H][W//2+1], unitary-DFT signal power
    signal: np.ndarray     # float64 [H][W], the true field the data were drawn from
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.d.shape


def wavenumber_half(H: int, W: int) -> np.ndarray:
    """|k| in cycles/pixel on the ``[H][W//2+1]`` half-spectrum grid (ky in FFT order)."""
    ky = np.fft.fftfreq(H)[:, None]
    kx = (np.arange(W // 2 + 1) / W)[None, :]
    return np.sqrt(ky * ky + kx * kx)


def power_law_pk(H: int, W: int, amp: float = 1.0, slope: float = -2.0, k0: float | None = None) -> np.ndarray:
    """P(k) = amp * (k/k0)^slope on the half-spectrum grid, with P = 0 at k = 0 (§2.1, Eq. 5 form)."""
    if k0 is None:
        k0 = 1.0 / max(H, W)
    k = wavenumber_half(H, W)
    P = np.zeros_like(k)
    nz = k > 0
    P[nz] = amp * (k[nz] / k0) ** slope
    return P.astype(np.float32)


def gaussian_random_field(Pk: np.ndarray, H: int, W: int, rng: np.random.Generator) -> np.ndarray:
    """Real zero-mean GRF whose unitary DFT has variance ``Pk`` per mode (§3.2 recipe).

    Filtering white noise by sqrt(P) in the orthonormal FFT basis is distributionally identical to
    drawing Re, Im of each Hermitian-paired mode with variance P/2 (self-conjugate modes real).
    """
    white = rng.standard_normal((H, W))
    spec = np.fft.rfft2(white, norm="ortho") * np.sqrt(Pk.astype(np.float64))
    return np.fft.irfft2(spec, s=(H, W), norm="ortho")


def _scatter(mask: np.ndarray, count: int, rng: np.random.Generator) -> None:
    free = np.flatnonzero(mask.ravel() == 0)
    pick = rng.choice(free, size=count, replace=False)
    mask.ravel()[pick] = 1


def _finish(signal, Ndiag, mask, Pk, rng, meta) -> WFProblem:
    noise = rng.standard_normal(signal.shape) * np.sqrt(Ndiag.astype(np.float64))
    d = signal + noise
    d[mask == 1] = 0.0
    return WFProblem(d=d.astype(np.float32), Ndiag=Ndiag.astype(np.float32), mask=mask.astype(np.uint8),
                     Pk=Pk.astype(np.float32), signal=signal, meta=meta)


def make_problem(H: int, W: int | None = None, *, seed: int = 0, amp: float = 1.0, slope: float = -2.0,
                 k0: float | None = None, sigma2: tuple[float, float] = (0.05, 0.5),
                 mask_frac: float = 0.1, block: tuple[int, int, int, int] | None = None) -> WFProblem:
    """Generic test problem: power-law GRF, i.i.d. uniform noise variance, scattered mask + optional block.

    ``block`` = (row0, row1, col0, col1), half-open, is masked in addition to ``mask_frac`` of the
    remaining pixels chosen at random.
    """
    W = H if W is None else W
    rng = np.random.default_rng(seed)
    Pk = power_law_pk(H, W, amp, slope, k0)
    signal = gaussian_random_field(Pk, H, W, rng)
    Ndiag = rng.uniform(sigma2[0], sigma2[1], size=(H, W))
    mask = np.zeros((H, W), np.uint8)
    if block is not None:
        r0, r1, c0, c1 = block
        mask[r0:r1, c0:c1] = 1
    n_scatter = int(round(mask_frac * H * W))
    if n_scatter:
        _scatter(mask, n_scatter, rng)
    return _finish(signal, Ndiag, mask, Pk, rng, dict(kind="generic", H=H, W=W, seed=seed, slope=slope))


def config_plain32(seed: int = 0) -> WFProblem:
    """32x32 plain-method case: P = (k/k0)^-2 with k0 = 1/32, sigma^2 ~ U[0.05, 0.5],
    an 8x8 masked block (rows/cols 12..19) plus 5% (51) random pixels outside it."""
    H = W = 32
    rng = np.random.default_rng(seed)
    Pk = power_law_pk(H, W, 1.0, -2.0, 1.0 / 32)
    signal = gaussian_random_field(Pk, H, W, rng)
    Ndiag = rng.uniform(0.05, 0.5, size=(H, W))
    mask = np.zeros((H, W), np.uint8)
    mask[12:20, 12:20] = 1
    _scatter(mask, int(round(0.05 * H * W)), rng)
    return _finish(signal, Ndiag, mask, Pk, rng, dict(kind="plain32", H=H, W=W, seed=seed))


def config_paper128(seed: int = 0) -> WFProblem:
    """128x128 paper-shaped case (§3.2 image size): slope -2 with k0 = 1/32, sigma^2 ~ U[0.01, 1.0],
    mask = two rectangles (rows 16..39 x cols 20..51, rows 80..95 x cols 70..101) plus 358 scattered
    pixels, 1638 pixels in all (10% of the area)."""
    H = W = 128
    rng = np.random.default_rng(seed)
    Pk = power_law_pk(H, W, 1.0, -2.0, 1.0 / 32)
    signal = gaussian_random_field(Pk, H, W, rng)
    Ndiag = rng.uniform(0.01, 1.0, size=(H, W))
    mask = np.zeros((H, W), np.uint8)
    mask[16:40, 20:52] = 1
    mask[80:96, 70:102] = 1
    _scatter(mask, 358, rng)
    return _finish(signal, Ndiag, mask, Pk, rng, dict(kind="paper128", H=H, W=W, seed=seed))


def circular_holes(H: int, W: int, n_holes: int, r_range: tuple[float, float], area_frac: float,
                   rng: np.random.Generator) -> np.ndarray:
    """Mask of ``n_holes`` discs (periodic wrap) with radii in ``r_range`` covering ``area_frac`` of the image.

    Centres are uniform; radii are r_lo + (r_hi - r_lo) u^a with u uniform, and the exponent a is set by
    bisection so that the union of the discs covers ``area_frac`` of the pixels (to within a pixel or so
    of the reachable fractions).
    """
    cy = rng.uniform(0, H, n_holes)
    cx = rng.uniform(0, W, n_holes)
    u = rng.uniform(0.0, 1.0, n_holes)
    r_lo, r_hi = r_range

    def paint(a):
        mask = np.zeros((H, W), np.uint8)
        for y0, x0, r in zip(cy, cx, r_lo + (r_hi - r_lo) * u ** a):
            R = int(np.ceil(r)) + 1
            ys = np.arange(int(np.floor(y0)) - R, int(np.floor(y0)) + R + 1)
            xs = np.arange(int(np.floor(x0)) - R, int(np.floor(x0)) + R + 1)
            inside = (ys[:, None] + 0.5 - y0) ** 2 + (xs[None, :] + 0.5 - x0) ** 2 <= r * r
            yy, xx = np.nonzero(inside)
            mask[ys[yy] % H, xs[xx] % W] = 1
        return mask

    lo, hi = np.log(1e-3), np.log(1e3)           # a small: radii near r_hi (largest cover)
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if paint(np.exp(mid)).mean() > area_frac:
            lo = mid
        else:
            hi = mid
    return paint(np.exp(0.5 * (lo + hi)))


def config_precision(H: int = 1024, seed: int = 0, n_holes: int = 200, r_range: tuple[float, float] = (4.0, 30.0),
                     area_frac: float = 0.25) -> WFProblem:
    """Precision case: P = (k/k0)^-1.5 with k0 = 1/32, sigma^2 ~ U[0.001, 0.1] (noise dynamic range 100), and
    a mask of ``n_holes`` circular holes with radii in ``r_range`` covering ``area_frac`` of the area
    (defaults: the 1024x1024 map with 200 holes of radius 4-30 px over 25%)."""
    W = H
    rng = np.random.default_rng(seed)
    Pk = power_law_pk(H, W, 1.0, -1.5, 1.0 / 32)
    signal = gaussian_random_field(Pk, H, W, rng)
    Ndiag = rng.uniform(0.001, 0.1, size=(H, W))
    mask = circular_holes(H, W, n_holes, r_range, area_frac, rng)
    return _finish(signal, Ndiag, mask, Pk, rng, dict(kind="precision", H=H, W=W, seed=seed))


def batch_class_counts(n_images: int, fractions=((64, 0.40), (128, 0.40), (256, 0.15), (512, 0.05))) -> dict:
    """Images per size by largest-remainder rounding of ``n_images * fraction`` (ties: the first size)."""
    raw = [(H, n_images * f) for H, f in fractions]
    counts = {H: int(np.floor(x)) for H, x in raw}
    left = n_images - sum(counts.values())
    for H, x in sorted(raw, key=lambda t: -(t[1] - np.floor(t[1])))[:left]:
        counts[H] += 1
    return counts


def config_batch(n_images: int = 4096, seed: int = 0, fractions=((64, 0.40), (128, 0.40), (256, 0.15), (512, 0.05))):
    """Mixed-size batch (default: 4096 images, 1639 x 64^2, 1638 x 128^2, 614 x 256^2, 205 x 512^2), in a
    random order. Per image: slope ~ U[-3, -1] with k0 = 1/N; sigma^2 ~ U[a, b] with a ~ U[0.01, 0.1] and
    b = a * U[2, 20]; masked fraction f ~ U[0, 0.2], half of it one random rectangle (periodic wrap) and
    half scattered pixels. Returns a list of WFProblem."""
    rng = np.random.default_rng(seed)
    counts = batch_class_counts(n_images, fractions)
    sizes = np.concatenate([np.full(c, H) for H, c in counts.items()])
    sizes = sizes[rng.permutation(sizes.size)]
    out = []
    for H in sizes:
        H = int(H)
        slope = rng.uniform(-3.0, -1.0)
        Pk = power_law_pk(H, H, 1.0, slope, 1.0 / H)
        signal = gaussian_random_field(Pk, H, H, rng)
        a = rng.uniform(0.01, 0.1)
        b = a * rng.uniform(2.0, 20.0)
        Ndiag = rng.uniform(a, b, size=(H, H))
        mask = np.zeros((H, H), np.uint8)
        f = rng.uniform(0.0, 0.2)
        rect = int(round(0.5 * f * H * H))
        if rect:
            h = int(np.clip(round(np.sqrt(rect * rng.uniform(0.5, 2.0))), 1, H))
            w = int(np.clip(round(rect / h), 1, H))
            y0, x0 = rng.integers(0, H, size=2)
            mask[np.ix_((y0 + np.arange(h)) % H, (x0 + np.arange(w)) % H)] = 1
        n_scatter = int(round(0.5 * f * H * H))
        if n_scatter:
            _scatter(mask, min(n_scatter, int((mask == 0).sum())), rng)
        out.append(_finish(signal, Ndiag, mask, Pk, rng, dict(kind="batch", H=H, W=H, slope=slope)))
    return out


def flat_problem(H: int, W: int | None = None, *, seed: int = 0, P: float = 1.0, sigma2: float = 0.3,
                 all_masked: bool = False) -> WFProblem:
    """Special cases with closed-form answers: flat P (except P0 = 0), homogeneous noise, and either no
    mask or every pixel masked."""
    W = H if W is None else W
    rng = np.random.default_rng(seed)
    Pk = np.full((H, W // 2 + 1), P, np.float32)
    Pk[0, 0] = 0.0
    signal = gaussian_random_field(Pk, H, W, rng)
    Ndiag = np.full((H, W), sigma2)
    mask = np.ones((H, W), np.uint8) if all_masked else np.zeros((H, W), np.uint8)
    return _finish(signal, Ndiag, mask, Pk, rng, dict(kind="flat", H=H, W=W, seed=seed))
