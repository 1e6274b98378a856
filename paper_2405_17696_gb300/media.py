"""Seeded synthetic inputs: velocity media, absorbing-layer profiles, sources.

This module builds the *inputs* of the Helmholtz solves (Sec. 3.1, Eq. 3.1-3.3
and Sec. 4.1) and nothing else: it contains none of the solver's arithmetic.
The CUDA path and the CPU oracle both receive the arrays made here.

The paper runs on the SEG/EAGE salt model (608x304) and on Marmousi (544x272)
(Sec. 5.2, Sec. 5.5); neither dataset is available, so the media below are
seeded stand-ins with the same shapes and statistics: 2:1 aspect, layered
sediments between 1.5 and 4.5 km/s, salt-like high-velocity bodies, sources
and receivers on the top rows, about 10 grid points per wavelength.

Conventions used throughout the library:
  * fields are ``[nz][nx]`` arrays, x contiguous (row-major), z pointing down;
  * ``kappa = 1/c`` in s/m, so the squared slowness of Eq. 3.1 is m = kappa^2;
  * a point source is a discrete delta of unit integral, e_s / (hx * hz).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# random streams
# --------------------------------------------------------------------------

#: Seeds of the four random streams: true model, sources/noise, CNN
#: initialisation and training-data generation.
SEED_MODEL, SEED_SOURCES, SEED_CNN, SEED_DATAGEN = 0, 1, 2, 3


def rng(seed: int) -> np.random.Generator:
    """A reproducible numpy generator (PCG64) for one seed."""
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# counter-based splitmix64 streams (the draws the library makes itself when it
# builds training data, reproduced here from the generator's published definition:
# Steele, Lea and Flood, OOPSLA 2014)
# --------------------------------------------------------------------------
_SM_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def _sm_mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _sm_uniform(key, n):
    """u in (0, 1) from counter n of the stream with key `key`."""
    with np.errstate(over="ignore"):
        z = _sm_mix(np.uint64(key) + np.asarray(n, dtype=np.uint64) * _SM_GAMMA)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def splitmix_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        return _sm_mix(np.uint64(seed) + np.uint64(stream) * _SM_GAMMA)


def splitmix_complex_normal(first: int, n: int, npts: int, seed: int) -> np.ndarray:
    """x ~ CN(0, 1) of pairs first .. first + n - 1 (npts nodes each) of the training-data
    stream (stream 1): Box-Muller on the uniforms of counters 2q + 1 and 2q + 2, q = i npts + p."""
    key = splitmix_key(seed, 1)
    q = np.arange(first * npts, (first + n) * npts, dtype=np.uint64)
    u1 = _sm_uniform(key, np.uint64(2) * q + np.uint64(1))
    u2 = _sm_uniform(key, np.uint64(2) * q + np.uint64(2))
    rho = np.sqrt(-np.log(u1))
    x = (rho * np.cos(2.0 * np.pi * u2) + 1j * rho * np.sin(2.0 * np.pi * u2)).astype(np.complex64)
    return x.reshape(n, npts)


def splitmix_step_counts(n: int, seed: int, kmax: int) -> np.ndarray:
    """GMRES step counts 1 + floor(u kmax) of pairs 0 .. n - 1 (stream 2, counter i + 1)."""
    u = _sm_uniform(splitmix_key(seed, 2), np.arange(1, n + 1, dtype=np.uint64))
    return np.minimum(1 + np.floor(u * kmax).astype(np.int64), kmax).astype(np.int32)


# --------------------------------------------------------------------------
# smoothing used to shape the media (input construction only)
# --------------------------------------------------------------------------

def gaussian_smooth(a: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian filter with edge replication (truncated at 4 sigma)."""
    if sigma <= 0:
        return np.array(a, dtype=np.float64, copy=True)
    r = int(math.ceil(4.0 * sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-0.5 * (t / sigma) ** 2)
    w /= w.sum()
    out = np.asarray(a, dtype=np.float64)
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (r, r)
        p = np.pad(out, pad, mode="edge")
        acc = np.zeros_like(out)
        n = out.shape[axis]
        for k, wk in enumerate(w):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(k, k + n)
            acc += wk * p[tuple(sl)]
        out = acc
    return out


# --------------------------------------------------------------------------
# velocity media (m/s)
# --------------------------------------------------------------------------

def constant_velocity(nx: int, nz: int, c: float = 1500.0) -> np.ndarray:
    return np.full((nz, nx), float(c))


def linear_slowness_velocity(nx: int, nz: int, c_top: float, c_bot: float) -> np.ndarray:
    """Velocity whose squared slowness m = 1/c^2 is linear in depth between
    the values at the top and bottom rows (the training media of Sec. 4.1)."""
    m_top, m_bot = 1.0 / c_top ** 2, 1.0 / c_bot ** 2
    t = np.linspace(0.0, 1.0, nz)[:, None]
    m = (1.0 - t) * m_top + t * m_bot
    return np.broadcast_to(1.0 / np.sqrt(m), (nz, nx)).copy()


def random_linear_velocity(nx: int, nz: int, seed: int) -> np.ndarray:
    """A random training medium: c_top ~ U(1.5, 2.0) km/s, c_bot ~ U(3.0, 4.5)
    km/s, squared slowness linear in depth."""
    g = rng(seed)
    c_top = g.uniform(1500.0, 2000.0)
    c_bot = g.uniform(3000.0, 4500.0)
    return linear_slowness_velocity(nx, nz, c_top, c_bot)


def layered_velocity(nx: int, nz: int, seed: int = SEED_MODEL, n_layers: int = 12,
                     c_min: float = 1500.0, c_max: float = 4500.0,
                     noise_std: float = 100.0, sigma: float = 3.0) -> np.ndarray:
    """Layered sediments with sinusoidally perturbed interfaces.

    Layer k (0-based, top to bottom) has velocity c_min + (c_max-c_min) k/(L-1).
    Its top interface sits at depth k*nz/L + A_k sin(2 pi x / Lambda_k + phi_k)
    with A_k ~ U(0, nz/(4L)), Lambda_k ~ U(0.25, 1) nx, phi_k ~ U(0, 2 pi).
    i.i.d. N(0, noise_std) noise is added, then smoothed by a Gaussian of
    ``sigma`` cells; the result is clipped to [c_min - 100, c_max + 100].
    """
    g = rng(seed)
    x = np.arange(nx, dtype=np.float64)
    z = np.arange(nz, dtype=np.float64)[:, None]
    c = np.full((nz, nx), c_min)
    for k in range(1, n_layers):
        amp = g.uniform(0.0, 0.25 * nz / n_layers)
        lam = g.uniform(0.25, 1.0) * nx
        phi = g.uniform(0.0, 2.0 * math.pi)
        top = k * nz / n_layers + amp * np.sin(2.0 * math.pi * x / lam + phi)
        ck = c_min + (c_max - c_min) * k / (n_layers - 1)
        c = np.where(z >= top[None, :], ck, c)
    c = c + g.normal(0.0, noise_std, size=c.shape)
    c = gaussian_smooth(c, sigma)
    return np.clip(c, c_min - 100.0, c_max + 100.0)


def fault_salt_velocity(nx: int, nz: int, seed: int = SEED_MODEL,
                        n_faults: int = 3, salt_c: float = 4500.0) -> np.ndarray:
    """Layered model cut by vertical faults with a salt-like ellipse.

    Each fault at a seeded column shifts everything to its right down by a
    seeded throw of 10..40 cells (scaled with nz/1024); the ellipse has
    semi-axes (300, 120) cells scaled with (nx/2048, nz/1024).
    """
    base = layered_velocity(nx, nz, seed=seed)
    g = rng(seed + 1000)
    c = base.copy()
    for _ in range(n_faults):
        xf = int(g.uniform(0.15, 0.85) * nx)
        throw = max(1, int(round(g.uniform(10, 40) * nz / 1024)))
        shifted = np.empty_like(c[:, xf:])
        shifted[throw:] = c[:-throw, xf:]
        shifted[:throw] = c[:1, xf:]
        c[:, xf:] = shifted
    ax, az = 300.0 * nx / 2048, 120.0 * nz / 1024
    cx, cz = g.uniform(0.35, 0.65) * nx, g.uniform(0.45, 0.6) * nz
    X, Z = np.meshgrid(np.arange(nx), np.arange(nz))
    inside = ((X - cx) / ax) ** 2 + ((Z - cz) / az) ** 2 <= 1.0
    c[inside] = salt_c
    return c


def kappa_of(c: np.ndarray) -> np.ndarray:
    """kappa = 1/c (s/m) as float32, the medium input of the solver."""
    return (1.0 / np.asarray(c, dtype=np.float64)).astype(np.float32)


# --------------------------------------------------------------------------
# absorbing layer (Sec. 4.1: gamma goes from 0 to 1 towards the boundaries,
# except the top, which is allowed to reflect)
# --------------------------------------------------------------------------

def abl_gamma(nx: int, nz: int, width: int, gamma_max: float = 1.0,
              top: bool = False) -> np.ndarray:
    """Quadratic absorbing-layer profile gamma(x), float32 ``[nz][nx]``.

    In a layer of ``width`` cells a cell at depth d cells into it (d = width
    at the outermost cell, 1 at the innermost) gets gamma_max (d/width)^2;
    where layers overlap the larger value wins; the interior is 0.  ``top``
    adds a layer along the top edge too (used for free-space tests).
    """
    def ramp(n: int, lo: bool, hi: bool) -> np.ndarray:
        i = np.arange(n, dtype=np.float64)
        d = np.zeros(n)
        if lo:
            d = np.maximum(d, width - i)
        if hi:
            d = np.maximum(d, i - (n - 1 - width))
        d = np.clip(d, 0.0, None)
        return gamma_max * (d / width) ** 2

    gx = ramp(nx, True, True)[None, :]
    gz = ramp(nz, top, True)[:, None]
    return np.maximum(gx, gz).astype(np.float32)


# --------------------------------------------------------------------------
# right-hand sides
# --------------------------------------------------------------------------

def point_source_rhs(nx: int, nz: int, positions, hx: float, hz: float) -> np.ndarray:
    """complex64 ``[len(positions)][nz][nx]``: one discrete delta e_s/(hx hz)
    per (iz, ix) position (Eq. 3.1: g is a discretised delta)."""
    out = np.zeros((len(positions), nz, nx), dtype=np.complex64)
    for s, (iz, ix) in enumerate(positions):
        out[s, iz, ix] = 1.0 / (hx * hz)
    return out


def complex_normal(shape, seed: int) -> np.ndarray:
    """complex64 samples of CN(0, 1): real and imaginary parts ~ N(0, 1/2)."""
    g = rng(seed)
    re = g.normal(0.0, math.sqrt(0.5), size=shape)
    im = g.normal(0.0, math.sqrt(0.5), size=shape)
    return (re + 1j * im).astype(np.complex64)


def top_row_positions(nx: int, n: int, iz: int = 2, step: int = 8, offset: int = 4):
    return [(iz, offset + step * s) for s in range(n) if offset + step * s < nx]


# --------------------------------------------------------------------------
# workload recipes (the configurations the tests and the benchmark use)
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    nx: int
    nz: int
    h: float
    freqs_hz: list
    kappa: np.ndarray = field(repr=False)
    gamma: np.ndarray = field(repr=False)
    positions: list = field(repr=False)

    @property
    def omegas(self):
        return [2.0 * math.pi * f for f in self.freqs_hz]

    def rhs(self) -> np.ndarray:
        """All (frequency, source) right-hand sides, frequency-major."""
        g = point_source_rhs(self.nx, self.nz, self.positions, self.h, self.h)
        return np.concatenate([g] * len(self.freqs_hz), axis=0)

    def freq_index(self) -> np.ndarray:
        ns = len(self.positions)
        return np.repeat(np.arange(len(self.freqs_hz), dtype=np.int32), ns)


def workload_small() -> Workload:
    """128x128 interior plus a 16-cell absorbing layer on all four sides
    (160x160), h = 25 m, c = 1.5 km/s, f = 6 Hz (10 points per wavelength),
    one source at the top centre of the interior."""
    n = 160
    c = constant_velocity(n, n, 1500.0)
    return Workload("helmholtz_160x160_1rhs", n, n, 25.0, [6.0], kappa_of(c),
                    abl_gamma(n, n, 16, 1.0, top=True), [(16, 80)])


def workload_batched(n_src: int = 64) -> Workload:
    """512x256 layered medium, h = 20 m, 32-cell absorbing layer on the left,
    right and bottom, 64 sources on row 2, f in {3, 4.5, 6} Hz -> 192 RHS."""
    nx, nz = 512, 256
    c = layered_velocity(nx, nz, seed=SEED_MODEL)
    return Workload(f"helmholtz_512x256_{3 * n_src}rhs", nx, nz, 20.0, [3.0, 4.5, 6.0],
                    kappa_of(c), abl_gamma(nx, nz, 32), top_row_positions(nx, n_src))


def workload_cnn(n_src: int = 128) -> Workload:
    """1024x512 layered medium, h = 12.5 m, f = 8 Hz, n_src (128) sources on row 2."""
    nx, nz = 1024, 512
    c = layered_velocity(nx, nz, seed=SEED_MODEL)
    return Workload(f"helmholtz_1024x512_{n_src}rhs", nx, nz, 12.5, [8.0],
                    kappa_of(c), abl_gamma(nx, nz, 32), top_row_positions(nx, n_src))


def crop_workload(nx: int = 64, nz: int = 32, h: float = 20.0, freqs=(6.0,),
                  seed: int = SEED_MODEL, width: int = 8) -> Workload:
    """A small layered medium for oracle-speed tests."""
    c = layered_velocity(nx, nz, seed=seed)
    return Workload(f"helmholtz_{nx}x{nz}", nx, nz, h, list(freqs), kappa_of(c),
                    abl_gamma(nx, nz, width), top_row_positions(nx, max(1, nx // 8), iz=2,
                                                                   step=8, offset=4))


def medium_sequence(c_true: np.ndarray, steps: int = 8, sigma: float = 10.0):
    """The squared-slowness path m_t = (1 - t/T) G_sigma(m_true) + (t/T) m_true, t = 0..T, from a
    Gaussian-smoothed model to the true one (a stand-in for the models an FWI visits), as
    kappa = sqrt(m_t) float32 arrays."""
    m_true = 1.0 / np.asarray(c_true, dtype=np.float64) ** 2
    m_s = gaussian_smooth(m_true, sigma)
    out = []
    for t in range(steps + 1):
        m = (1.0 - t / steps) * m_s + (t / steps) * m_true
        out.append(np.sqrt(m).astype(np.float32))
    return out
