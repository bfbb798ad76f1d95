"""Seeded synthetic inputs for the photo-switching optoacoustic reconstruction.

This module generates *inputs only*: the transducer's per-depth kernel (which
plays the role of the measured spatial/electrical response in the paper,
Sec. 2.3 "Acoustic Model" and Sec. 3.3), tube phantoms, Gaussian noise draws and
the shapes of batched problems.  It holds none of the reconstruction arithmetic
(no switching model, no H, no H^T, no proximal step, no FISTA).  Both the FP64
oracle tests and the CUDA library consume exactly the arrays produced here.

Everything is seeded with ``numpy.random.default_rng``.

Units: lengths in mm, times in microseconds, speed of sound in mm/us.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np

__all__ = [
    "Geometry",
    "Switching",
    "Problem",
    "WORKLOADS",
    "workload",
    "transducer_kernel",
    "eir_taps",
    "spr_image",
    "matched_time_grid",
    "tube_phantom",
    "gaussian",
    "noise_sigma",
    "batch_shapes",
]


@dataclass(frozen=True)
class Geometry:
    """Raster-scan grid and transducer.

    The volume is ``Y x X`` scan positions (lateral pitch ``dx_mm``), ``Z``
    depths (pitch ``dz_mm``) centred on the focal plane, ``T`` time samples
    (pitch ``dt_us``), ``N`` pulses (``pulses_per_cycle`` per OFF-switching
    cycle) and ``P`` species (the last one is the non-switching background).
    ``k`` is the odd lateral support of the per-depth kernel.
    """

    X: int
    Y: int
    Z: int
    T: int
    N: int
    P: int
    k: int
    pulses_per_cycle: int
    dx_mm: float = 0.020
    dz_mm: float = 0.010
    dt_us: float = 0.008
    c_mm_per_us: float = 1.5
    focal_mm: float = 3.0
    aperture_mm: float = 1.5
    n_aperture: int = 256
    eir_mhz: float = 50.0

    @property
    def r(self) -> int:
        return self.k // 2

    @property
    def S(self) -> int:
        return self.X * self.Y

    def c_shape(self):
        return (self.P, self.Y, self.X, self.Z)

    def y_shape(self):
        return (self.N, self.Y, self.X, self.T)

    def k_shape(self):
        return (self.Z, self.k, self.k, self.T)


@dataclass(frozen=True)
class Switching:
    """Photo-switching parameters of the exponential OFF-switching law.

    Per species p: ``eps_bar[p]`` (ON minus OFF extinction), ``eps_off[p]``
    and the kinetic constant ``kappa[p]`` (per pulse interval).  The fluence
    decays with depth as exp(-mu * j * dz).  The background species has
    kappa = 0 and eps_bar = 0, eps_off = 1 (a constant weight).
    """

    kappa: tuple
    eps_bar: tuple
    eps_off: tuple
    mu_per_mm: float = 2.0


def _default_switching(kappas_switchable):
    ks = tuple(float(v) for v in kappas_switchable) + (0.0,)
    eb = tuple(1.0 for _ in kappas_switchable) + (0.0,)
    eo = tuple(0.0 for _ in kappas_switchable) + (1.0,)
    return Switching(kappa=ks, eps_bar=eb, eps_off=eo, mu_per_mm=2.0)


@dataclass(frozen=True)
class Problem:
    """A named workload: geometry, switching, phantom recipe and solve settings."""

    name: str
    geom: Geometry
    sw: Switching
    tubes: int
    tubes_per_species: bool
    iters: int
    lam_l1: float = 1e-3
    lam_tv: float = 1e-3
    inner: int = 10
    snr_db: float = 20.0
    seed: int = 0


WORKLOADS = {
    # 16x16 scan, 24 depths, T=64, 7x7 support, 8 pulses (1 cycle), 2 species.
    "tiny_16x16x24_T64_k7_N8_P2": Problem(
        name="tiny_16x16x24_T64_k7_N8_P2",
        geom=Geometry(X=16, Y=16, Z=24, T=64, N=8, P=2, k=7, pulses_per_cycle=8),
        sw=_default_switching([0.05]),
        tubes=2, tubes_per_species=True, iters=20),
    # 64x64 scan, 64 depths, T=256, 15x15 support, 40 pulses (4 x 10), 2 species.
    "medium_64x64x64_T256_k15_N40_P2": Problem(
        name="medium_64x64x64_T256_k15_N40_P2",
        geom=Geometry(X=64, Y=64, Z=64, T=256, N=40, P=2, k=15, pulses_per_cycle=10),
        sw=_default_switching([0.05]),
        tubes=40, tubes_per_species=False, iters=200),
    # 128x128 scan, 96 depths, T=512, 31x31 support, 60 pulses (6 x 10), 3 species.
    "large_128x128x96_T512_k31_N60_P3": Problem(
        name="large_128x128x96_T512_k31_N60_P3",
        geom=Geometry(X=128, Y=128, Z=96, T=512, N=60, P=3, k=31, pulses_per_cycle=10),
        sw=_default_switching([0.03, 0.08]),
        tubes=60, tubes_per_species=False, iters=100),
}


def workload(name: str) -> Problem:
    return WORKLOADS[name]


def eir_taps(geom: Geometry) -> np.ndarray:
    """Gaussian-derivative electrical impulse response v[s], s in [-J, J].

    sigma = 1/(2 pi f_c) puts the spectral peak of the derivative of a
    Gaussian at f_c; J = ceil(4 sigma / dt); the taps are scaled so that
    max |v| = 1.
    """
    sigma = 1.0 / (2.0 * math.pi * geom.eir_mhz)
    J = int(math.ceil(4.0 * sigma / geom.dt_us))
    s = np.arange(-J, J + 1, dtype=np.float64)
    tau = s * geom.dt_us
    v = -(tau / sigma ** 2) * np.exp(-(tau ** 2) / (2.0 * sigma ** 2))
    return v / np.max(np.abs(v))


def aperture_points(geom: Geometry, seed: int = 0) -> np.ndarray:
    """Area-uniform points on the spherical cap of the focused transducer.

    The cap has radius ``focal_mm`` around the focus F = (0, 0, focal_mm)
    (depth axis pointing into the sample) and rim radius ``aperture_mm``.
    Returns an (n, 3) array of (x, y, depth) in mm.
    """
    rng = np.random.default_rng(seed)
    f = geom.focal_mm
    cos_max = math.cos(math.asin(geom.aperture_mm / f))
    u = rng.random(geom.n_aperture)
    v = rng.random(geom.n_aperture)
    cos_t = 1.0 - u * (1.0 - cos_max)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t ** 2))
    phi = 2.0 * math.pi * v
    px = f * sin_t * np.cos(phi)
    py = f * sin_t * np.sin(phi)
    pz = f - f * cos_t
    return np.stack([px, py, pz], axis=1)


def transducer_kernel(geom: Geometry, seed: int = 0) -> np.ndarray:
    """Per-depth lateral-shift-invariant kernel K[z][dy][dx][t] (FP64).

    For a point source at lateral offset (dx, dy) * dx_mm from the transducer
    axis and depth z_j = f + (j - (Z-1)/2) dz, each aperture point contributes
    a spherical-spreading weight 1/(4 pi d) / n_aperture at the time sample
    round(d / (c dt)) - t_gate, with t_gate = round(f / (c dt)) - T/2 so that
    the focal arrival lands at sample T/2.  Samples outside [0, T) are
    dropped.  The result is then convolved along t with the electrical
    impulse response (full convolution truncated to [0, T)).
    """
    f = geom.focal_mm
    r = geom.r
    cdt = geom.c_mm_per_us * geom.dt_us
    t_gate = int(np.rint(f / cdt)) - geom.T // 2
    pts = aperture_points(geom, seed)
    q = np.zeros(geom.k_shape(), dtype=np.float64)
    for j in range(geom.Z):
        zj = f + (j - (geom.Z - 1) / 2.0) * geom.dz_mm
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                ddx = pts[:, 0] - dx * geom.dx_mm
                ddy = pts[:, 1] - dy * geom.dx_mm
                ddz = pts[:, 2] - zj
                d = np.sqrt(ddx * ddx + ddy * ddy + ddz * ddz)
                bins = np.rint(d / cdt).astype(np.int64) - t_gate
                w = 1.0 / (4.0 * math.pi * d) / geom.n_aperture
                ok = (bins >= 0) & (bins < geom.T)
                np.add.at(q[j, dy + r, dx + r], bins[ok], w[ok])
    v = eir_taps(geom)
    J = (len(v) - 1) // 2
    K = np.zeros_like(q)
    for si, s in enumerate(range(-J, J + 1)):
        # K[..., t] += q[..., t - s] * v[s]
        if s >= 0:
            K[..., s:] += q[..., : geom.T - s] * v[si]
        else:
            K[..., : geom.T + s] += q[..., -s:] * v[si]
    return K


def matched_time_grid(geom: Geometry) -> Geometry:
    """The same geometry with the time pitch set so that one sample of
    travel distance equals one depth pitch (c dt = dz), the matched
    measurement and image grids of the paper's discretised acoustic model."""
    return replace(geom, dt_us=geom.dz_mm / geom.c_mm_per_us)


def spr_image(geom: Geometry, seed: int = 0) -> np.ndarray:
    """Synthetic spatial response eta[z][dy][dx] (FP64) of a focused
    transducer about its focus, standing in for the measured SPR image that
    the paper uses and does not publish: a Gaussian beam whose width grows
    away from the focal plane (w(z) = w0 sqrt(1 + (z / zR)^2), w0 from the
    aperture's numerical aperture), with a seeded multiplicative ripple of
    a few per cent.  Depth z is measured from the focal plane (depths
    centred on it, as in ``transducer_kernel``)."""
    rng = np.random.default_rng(seed)
    r = geom.r
    na = geom.aperture_mm / geom.focal_mm
    lam = geom.c_mm_per_us / geom.eir_mhz          # wavelength at the centre frequency
    w0 = max(0.5 * lam / na, 0.5 * geom.dx_mm)
    zr = math.pi * w0 * w0 / lam
    z = (np.arange(geom.Z) - (geom.Z - 1) / 2.0) * geom.dz_mm
    w = w0 * np.sqrt(1.0 + (z / zr) ** 2)
    lat = np.arange(-r, r + 1) * geom.dx_mm
    rho2 = lat[None, :, None] ** 2 + lat[None, None, :] ** 2
    eta = np.exp(-rho2 / (2.0 * w[:, None, None] ** 2)) * (w0 / w)[:, None, None]
    eta *= 1.0 + 0.03 * rng.standard_normal(eta.shape)
    return eta


def _segment_distance(p, a, b):
    ab = b - a
    denom = float(ab @ ab)
    t = ((p - a) @ ab) / denom if denom > 0 else np.zeros(p.shape[0])
    t = np.clip(t, 0.0, 1.0)
    proj = a[None, :] + t[:, None] * ab[None, :]
    return np.sqrt(((p - proj) ** 2).sum(axis=1))


def tube_phantom(geom: Geometry, tubes: int, seed: int = 0,
                 per_species: bool = False) -> np.ndarray:
    """Random vessel-like tubes; returns c[P][Y][X][Z] (FP64).

    Each tube is the set of voxels within a radius U[1, 3] (in units of the
    lateral pitch) of a segment between two uniform random points of the
    volume (distances in physical units, so voxels are anisotropic).  The
    tube value is U(0.5, 1) and its species is uniform over the P species,
    or, with ``per_species``, ``tubes`` tubes are drawn for every species.
    Overlapping tubes keep the maximum.
    """
    rng = np.random.default_rng(seed)
    c = np.zeros(geom.c_shape(), dtype=np.float64)
    yy, xx, zz = np.meshgrid(np.arange(geom.Y), np.arange(geom.X),
                             np.arange(geom.Z), indexing="ij")
    pos = np.stack([yy.ravel() * geom.dx_mm, xx.ravel() * geom.dx_mm,
                    zz.ravel() * geom.dz_mm], axis=1)
    ext = np.array([(geom.Y - 1) * geom.dx_mm, (geom.X - 1) * geom.dx_mm,
                    (geom.Z - 1) * geom.dz_mm])
    if per_species:
        species = [p for p in range(geom.P) for _ in range(tubes)]
    else:
        species = [int(rng.integers(0, geom.P)) for _ in range(tubes)]
    for sp in species:
        a = rng.random(3) * ext
        b = rng.random(3) * ext
        rad = rng.uniform(1.0, 3.0) * geom.dx_mm
        val = rng.uniform(0.5, 1.0)
        dist = _segment_distance(pos, a, b)
        inside = (dist <= rad).reshape(geom.Y, geom.X, geom.Z)
        c[sp] = np.where(inside, np.maximum(c[sp], val), c[sp])
    return c


def gaussian(shape, seed: int) -> np.ndarray:
    """Standard normal draws N(0, 1) in FP64."""
    return np.random.default_rng(seed).standard_normal(shape)


def noise_sigma(clean: np.ndarray, snr_db: float) -> float:
    """Noise standard deviation for a power signal-to-noise ratio in dB."""
    power = float(np.mean(np.asarray(clean, dtype=np.float64) ** 2))
    return math.sqrt(power / (10.0 ** (snr_db / 10.0)))


def batch_shapes(count: int = 16, seed: int = 0):
    """Shapes of ``count`` uneven independent problems (seeded).

    Scan sides from {32, 48, 64, 96, 128}, depths 48-128, T 128-512 (multiple
    of 16), pulses 20-80 (whole cycles of 10), 2-3 species and odd lateral
    supports 11-31.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(rng.choice([32, 48, 64, 96, 128]))
        Z = int(rng.integers(48, 129))
        T = int(rng.integers(128 // 16, 512 // 16 + 1)) * 16
        N = int(rng.integers(2, 9)) * 10
        P = int(rng.integers(2, 4))
        k = int(rng.choice(np.arange(11, 32, 2)))
        kap = [0.03, 0.08][: P - 1] if P == 3 else [0.05]
        out.append(Problem(
            name=f"batch{i}", seed=i,
            geom=Geometry(X=side, Y=side, Z=Z, T=T, N=N, P=P, k=k,
                          pulses_per_cycle=10),
            sw=_default_switching(kap), tubes=max(4, side // 2),
            tubes_per_species=False, iters=100))
    return out


def small_variant(prob: Problem, **geom_changes) -> Problem:
    """The same problem with some geometry fields replaced."""
    return replace(prob, geom=replace(prob.geom, **geom_changes))
