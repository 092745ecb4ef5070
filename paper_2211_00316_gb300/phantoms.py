"""Seeded synthetic inputs: ring geometries, sound-speed phantoms, frequency sweeps, noise.

This module holds no arithmetic of the inversion method itself. It only builds the
inputs that both the CUDA path and the FP64 CPU oracle consume: a grid, a ring of
point transducers, sound-speed maps, an initial model, a frequency list and additive
complex Gaussian noise. The paper's own phantom (a slice of a public digital breast
phantom) and its full-wave k-Wave data are not available; the generators below stand
in for them with the paper's value ranges: water 1500 m/s, tissue 1470-1580 m/s
(Sec. 6.1), a reconstruction mask of 0.9 R (Sec. 6.3) and a peak-based SNR (Sec. 6.3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np
from scipy import ndimage

C_WATER = 1500.0


@dataclass
class Geometry:
    """A centred square grid plus a ring of N point transducers (emitter and receiver each).

    Node (ix, iy) sits at (x0 + ix*dx, y0 + iy*dx); arrays are row-major [iy][ix].
    Transducer e sits at R*(cos(2*pi*e/N), sin(2*pi*e/N)) (Sec. 2.1: elements on a ring), or
    at xducer_xy[e] (N x 2, on the ring, counterclockwise) when that is given.
    """
    nx: int
    ny: int
    dx: float
    n_xducers: int
    ring_radius: float
    c0: float = C_WATER
    mask_frac: float = 0.9          # reconstruction mask radius / ring radius (Sec. 6.3)
    ds_frac: float = 0.5            # ray step / grid spacing
    weight_mode: int = 0            # 0 literal scattering-angle weight, 1 isochron weight
    tau: float = 0.12               # step length (Sec. 6.3.2a); sweeps set step_length(df)
    xducer_xy: np.ndarray | None = field(default=None, repr=False)   # N x 2 positions; None: uniform ring

    @property
    def x0(self) -> float:
        return -(self.nx - 1) * self.dx / 2.0

    @property
    def y0(self) -> float:
        return -(self.ny - 1) * self.dx / 2.0

    @property
    def mask_radius(self) -> float:
        return self.mask_frac * self.ring_radius

    @property
    def ds(self) -> float:
        return self.ds_frac * self.dx

    def coords(self):
        x = self.x0 + self.dx * np.arange(self.nx)
        y = self.y0 + self.dx * np.arange(self.ny)
        return np.meshgrid(x, y)  # X[iy, ix], Y[iy, ix]

    def mask(self) -> np.ndarray:
        X, Y = self.coords()
        return X * X + Y * Y <= self.mask_radius ** 2

    def as_dict(self) -> dict:
        d = asdict(self)
        d.update(x0=self.x0, y0=self.y0, mask_radius=self.mask_radius, ds=self.ds)
        return d


@dataclass
class Workload:
    name: str
    geom: Geometry
    freqs: np.ndarray
    snr_db: float
    c_true: np.ndarray
    c_init: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def dfreq(self) -> float:
        return float(self.freqs[1] - self.freqs[0]) if len(self.freqs) > 1 else 1.0e5


# The paper's sweep: 180 frequencies over 0.2-1.72 MHz, two consecutive frequencies per
# update, step length 0.12 (Sec. 6.3.2a). Its step per unit of frequency band is therefore
# 0.12 over 2 x 8.49 kHz; a sweep of one frequency per update at spacing df takes the step
# that moves the model as far per unit band.
TAU_PAPER = 0.12
DF_PAPER = (1.72e6 - 0.2e6) / 179.0
FREQS_PER_SET_PAPER = 2


def step_length(df: float) -> float:
    """Step length of a one-frequency-per-update sweep at spacing df (Hz)."""
    return TAU_PAPER * FREQS_PER_SET_PAPER * DF_PAPER / df


def _with_step(w: "Workload") -> "Workload":
    w.geom.tau = step_length(w.dfreq)
    return w


def jittered_ring(n_xducers: int, ring_radius: float, jitter: float, seed: int) -> np.ndarray:
    """N x 2 transducer positions on the ring, counterclockwise: element e at angle
    2 pi (e + u_e) / N with u_e uniform in [-jitter, jitter] (jitter < 0.5 keeps the order)."""
    rng = np.random.default_rng(seed)
    th = 2 * math.pi * (np.arange(n_xducers) + rng.uniform(-jitter, jitter, n_xducers)) / n_xducers
    return np.stack([ring_radius * np.cos(th), ring_radius * np.sin(th)], axis=1)


def _disc(X, Y, cx, cy, r):
    return (X - cx) ** 2 + (Y - cy) ** 2 <= r * r


def blur(c: np.ndarray, dx: float, sigma_m: float = 5e-3) -> np.ndarray:
    """Initial model: the true map blurred by a Gaussian of std sigma_m (edges replicated)."""
    return ndimage.gaussian_filter(c, sigma=sigma_m / dx, mode="nearest")


def two_disc_phantom(geom: Geometry, centres_mm=((-15.0, -5.0), (14.0, 10.0)),
                     radius_mm=8.0, contrasts=(0.03, -0.02)) -> np.ndarray:
    """Water with two discs of radius 8 mm at +3 % and -2 % sound speed."""
    X, Y = geom.coords()
    c = np.full((geom.ny, geom.nx), geom.c0)
    for (cx, cy), dc in zip(centres_mm, contrasts):
        c[_disc(X, Y, cx * 1e-3, cy * 1e-3, radius_mm * 1e-3)] = geom.c0 * (1.0 + dc)
    return c


def breast_phantom(geom: Geometry, seed: int) -> np.ndarray:
    """Breast-like slice from a seed.

    Water 1500 m/s; a fat ellipse at 1470 m/s with semi-axes (0.55 R, 0.45 R), random
    rotation and centre within 0.05 R; 3-6 glandular blobs at 1520-1560 m/s of radius
    0.05-0.12 R inside the ellipse; two tumours at 1570 m/s of radius 3-6 mm; and a
    Gaussian random field (std 10 m/s, correlation std 5 mm) added inside the ellipse.
    """
    rng = np.random.default_rng(seed)
    R = geom.ring_radius
    X, Y = geom.coords()
    c = np.full((geom.ny, geom.nx), geom.c0)
    th = rng.uniform(0, math.pi)
    rr = 0.05 * R * math.sqrt(rng.uniform())
    ph = rng.uniform(0, 2 * math.pi)
    ex, ey = rr * math.cos(ph), rr * math.sin(ph)
    ax, ay = 0.55 * R, 0.45 * R
    u = (X - ex) * math.cos(th) + (Y - ey) * math.sin(th)
    v = -(X - ex) * math.sin(th) + (Y - ey) * math.cos(th)
    ell = (u / ax) ** 2 + (v / ay) ** 2 <= 1.0
    c[ell] = 1470.0

    def inside_point(margin):
        while True:
            uu = rng.uniform(-1, 1)
            vv = rng.uniform(-1, 1)
            if uu * uu + vv * vv <= (1.0 - margin) ** 2:
                px = ex + uu * ax * math.cos(th) - vv * ay * math.sin(th)
                py = ey + uu * ax * math.sin(th) + vv * ay * math.cos(th)
                return px, py

    for _ in range(int(rng.integers(3, 7))):
        r = rng.uniform(0.05, 0.12) * R
        px, py = inside_point(0.3)
        c[_disc(X, Y, px, py, r) & ell] = rng.uniform(1520.0, 1560.0)
    for _ in range(2):
        r = rng.uniform(3e-3, 6e-3)
        px, py = inside_point(0.3)
        c[_disc(X, Y, px, py, r) & ell] = 1570.0
    noise = rng.standard_normal((geom.ny, geom.nx))
    grf = ndimage.gaussian_filter(noise, sigma=(5e-3 / math.sqrt(2.0)) / geom.dx, mode="wrap")
    grf *= 10.0 / max(grf[ell].std(), 1e-12)
    c[ell] += grf[ell]
    return c


def absorption_map(c_true: np.ndarray, c0: float = C_WATER, y: float = 1.4) -> np.ndarray:
    """Absorption coefficient alpha0 (Np (rad/s)^-y m^-1) of a breast-like phantom, in the
    paper's range 0-1 dB MHz^-y cm^-1 with water lossless (Sec. 6.1): fat (below c0) 0.4,
    denser tissue 0.5 + 0.5 (c - 1520)/50 clipped to [0.5, 1.0] dB MHz^-y cm^-1."""
    c = np.asarray(c_true, float)
    db = np.where(c < c0 - 1e-9, 0.4, np.clip(0.5 + 0.5 * (c - 1520.0) / 50.0, 0.5, 1.0))
    db = np.where(np.abs(c - c0) <= 1e-9, 0.0, db)
    np_per_m = db * 100.0 / (20.0 * np.log10(np.e))
    return np_per_m / (2 * np.pi * 1e6) ** y


def add_noise(data: np.ndarray, snr_db: float, seed: int) -> np.ndarray:
    """Complex Gaussian noise, E|n|^2 = sigma^2, sigma = 10^(-SNR/20) * max off-diagonal |data|.

    data is [..., N, N] complex (emitter-major); each leading slice gets its own sigma.
    """
    rng = np.random.default_rng(seed)
    out = np.array(data, dtype=np.complex128, copy=True)
    n = out.shape[-1]
    off = ~np.eye(n, dtype=bool)
    flat = out.reshape(-1, n, n)
    for k in range(flat.shape[0]):
        peak = np.abs(flat[k][off]).max()
        sigma = 10.0 ** (-snr_db / 20.0) * peak
        nz = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * (sigma / math.sqrt(2.0))
        nz[~off] = 0.0
        flat[k] += nz
    return flat.reshape(out.shape)


def small_two_disc() -> Workload:
    """64-transducer ring at 45 mm, 96x96 grid at 1 mm, two discs, 200/300/400 kHz, 40 dB."""
    g = Geometry(nx=96, ny=96, dx=1e-3, n_xducers=64, ring_radius=45e-3)
    ct = two_disc_phantom(g)
    return _with_step(Workload("ring64_grid96_two_discs", g, np.array([2e5, 3e5, 4e5]), 40.0, ct, blur(ct, g.dx)))


def breast(n_xducers: int, nx: int, dx: float, ring_radius: float, freqs, seed: int = 0,
           name: str | None = None, snr_db: float = 40.0) -> Workload:
    g = Geometry(nx=nx, ny=nx, dx=dx, n_xducers=n_xducers, ring_radius=ring_radius)
    ct = breast_phantom(g, seed)
    nm = name or f"ring{n_xducers}_grid{nx}_breast_seed{seed}"
    return _with_step(Workload(nm, g, np.asarray(freqs, dtype=float), snr_db, ct, blur(ct, g.dx), {"seed": seed}))


def fp32_ring256() -> Workload:
    """256-transducer ring at 110 mm, 288x288 grid at 0.8 mm, 10 frequencies 0.1-1 MHz."""
    return breast(256, 288, 0.8e-3, 110e-3, np.linspace(1e5, 1e6, 10), seed=0,
                  name="ring256_grid288_breast")


def precision_ring1024() -> Workload:
    """1024-transducer ring at 110 mm, 512x512 grid at 0.45 mm, 20 frequencies 0.1-1.2 MHz."""
    return breast(1024, 512, 0.45e-3, 110e-3, np.linspace(1e5, 1.2e6, 20), seed=0,
                  name="ring1024_grid512_breast")


def batched_slice(seed: int) -> Workload:
    """One slice of the uneven batch: N in {256,512,768,1024}, n in [192,512] step 32,
    dx in [0.45,1.0] mm, R = (n-1) dx / 2 - 5 mm, 10 frequencies 0.1-1 MHz."""
    rng = np.random.default_rng(1000 + seed)
    n_x = int(rng.choice([256, 512, 768, 1024]))
    n = int(rng.choice(np.arange(192, 513, 32)))
    dx = float(rng.uniform(0.45e-3, 1.0e-3))
    R = (n - 1) * dx / 2.0 - 5e-3
    return breast(n_x, n, dx, R, np.linspace(1e5, 1e6, 10), seed=seed,
                  name=f"slice{seed}_ring{n_x}_grid{n}")


def custom(n_xducers: int, nx: int, dx: float, ring_radius: float, kind: str = "water",
           seed: int = 0, freqs=(3e5,), ny: int | None = None) -> Workload:
    """Free-size workloads for tests (ragged sizes, water, discs)."""
    g = Geometry(nx=nx, ny=ny or nx, dx=dx, n_xducers=n_xducers, ring_radius=ring_radius)
    if kind == "water":
        ct = np.full((g.ny, g.nx), g.c0)
    elif kind == "discs":
        s = ring_radius / 45e-3
        ct = two_disc_phantom(g, centres_mm=((-15.0 * s, -5.0 * s), (14.0 * s, 10.0 * s)), radius_mm=8.0 * s)
    else:
        ct = breast_phantom(g, seed)
    return Workload(f"custom_{kind}_ring{n_xducers}_grid{nx}", g, np.asarray(freqs, float), 40.0, ct,
                    blur(ct, g.dx))
