"""Seeded synthetic microlens fields (inputs only; none of the method's arithmetic).

Both the CUDA path and the FP64 oracle draw their inputs from here, so a field is the
same bytes on both sides.  Random numbers come from SplitMix64 (Steele, Lea & Flood
2014): output k >= 1 of a stream with seed s is mix(s + k * 0x9E3779B97F4A7C15), and a
uniform double in [0, 1) is the top 53 bits times 2^-53.

Fields follow the paper's set-up (Sec. 2): N point masses placed uniformly in a disc of
radius R sized for a microlens convergence kappa_* = pi * sum(m) / (pi R^2), i.e.
R = sqrt(sum(m) / kappa_*), with theta_* = 1.  Positions are r = R sqrt(u),
theta = 2 pi v.  Mass functions: unit, log-uniform on [a, b] (optionally rescaled to mean
1), or a Kroupa-like broken power law dN/dm ~ m^-1.3 on [0.08, 0.5), m^-2.3 on [0.5, 1.5].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset+1 .. offset+count of the SplitMix64 stream with the given seed."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64 outputs."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def stream_seed(config_seed: int, index: int, lane: int = 0) -> int:
    """Independent stream per (config, field/request index, lane)."""
    return ((config_seed & 0xFFFF) << 48) ^ ((index & 0xFFFFFFFF) << 8) ^ (lane & 0xFF)


@dataclasses.dataclass
class Field:
    """A microlens field: star positions/masses (FP64) and the macro-model."""
    x: np.ndarray
    y: np.ndarray
    m: np.ndarray
    kappa_star: float
    kappa_s: float
    gamma: float
    radius: float
    seed: int
    c1: float = 0.0  # rectangular field: half-width and half-height (0 for a disc)
    c2: float = 0.0

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_roots(self) -> int:
        return 2 * self.n


def masses(kind: str, n: int, seed: int, lo: float = 0.08, hi: float = 1.0, normalise: bool = False) -> np.ndarray:
    if kind == "unit":
        return np.ones(n)
    u = uniform(seed, n)
    if kind == "loguniform":
        mm = lo * np.exp(u * math.log(hi / lo))
        if normalise:
            mm = mm / mm.mean()
        return mm
    if kind == "kroupa":
        # dN/dm = c m^-1.3 on [0.08, 0.5), c 0.5 m^-2.3 on [0.5, 1.5] (continuous at 0.5).
        a, b, c = 0.08, 0.5, 1.5
        w1 = (b ** -0.3 - a ** -0.3) / -0.3
        w2 = 0.5 * (c ** -1.3 - b ** -1.3) / -1.3
        p1 = w1 / (w1 + w2)
        out = np.empty(n)
        low = u < p1
        t = u[low] / p1
        out[low] = (a ** -0.3 + t * (b ** -0.3 - a ** -0.3)) ** (1.0 / -0.3)
        t = (u[~low] - p1) / (1.0 - p1)
        out[~low] = (b ** -1.3 + t * (c ** -1.3 - b ** -1.3)) ** (1.0 / -1.3)
        return out
    raise ValueError(f"unknown mass function {kind!r}")


def disc_field(n: int, kappa_star: float, kappa_s: float, gamma: float, seed: int,
               mass_kind: str = "unit", mass_lo: float = 0.08, mass_hi: float = 1.0,
               normalise: bool = False) -> Field:
    """N stars uniform in a disc of radius sqrt(sum(m)/kappa_*) (Sec. 2)."""
    mm = masses(mass_kind, n, seed ^ 0x5A5A5A5A, mass_lo, mass_hi, normalise)
    radius = math.sqrt(float(mm.sum()) / kappa_star)
    u = uniform(seed, 2 * n)
    r = radius * np.sqrt(u[0::2])
    th = 2.0 * math.pi * u[1::2]
    return Field(r * np.cos(th), r * np.sin(th), mm, kappa_star, kappa_s, gamma, radius, seed)


def rect_field(n: int, kappa_star: float, kappa_s: float, gamma: float, seed: int, aspect: float = 1.0,
               mass_kind: str = "unit", mass_lo: float = 0.08, mass_hi: float = 1.0,
               normalise: bool = False) -> Field:
    """N stars uniform in the rectangle |x| <= c1, |y| <= c2 = aspect c1 whose area
    4 c1 c2 = sum(m) / kappa_* (the rectangular field of Sec. 4.2)."""
    mm = masses(mass_kind, n, seed ^ 0x5A5A5A5A, mass_lo, mass_hi, normalise)
    c1 = math.sqrt(float(mm.sum()) / (4.0 * kappa_star * aspect))
    c2 = aspect * c1
    u = uniform(seed, 2 * n)
    return Field(c1 * (2.0 * u[0::2] - 1.0), c2 * (2.0 * u[1::2] - 1.0), mm, kappa_star, kappa_s, gamma,
                 math.hypot(c1, c2), seed, c1, c2)


# --------------------------------------------------------------------------------------
# Workloads (synthetic stand-ins for the paper's random star fields)
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    fields: list
    msteps: int
    map_extent: float = 0.0
    map_pixels: int = 0


def workload_small() -> Workload:
    """N=10 unit masses, kappa_*=0.3, kappa_s=0, gamma=0.2, seed 0; m=1000; 256^2 map over +-3."""
    f = disc_field(10, 0.3, 0.0, 0.2, stream_seed(0, 0))
    return Workload("n10_m1000_map256", [f], 1000, 3.0, 256)


def workload_n1000() -> Workload:
    """N=1000 log-uniform masses in [0.08, 1] rescaled to mean 1, kappa_*=0.4, kappa_s=0,
    gamma=0.4; m=10^4; 4096^2 crossing and distance maps over +-10."""
    f = disc_field(1000, 0.4, 0.0, 0.4, stream_seed(1, 0), "loguniform", 0.08, 1.0, normalise=True)
    return Workload("n1000_m10000_map4096", [f], 10000, 10.0, 4096)


def workload_n20000() -> Workload:
    """N=20000 Kroupa-like masses in [0.08, 1.5], kappa_*=0.2, kappa_s=0.3, gamma=0.3;
    m=2x10^4; 8192^2 map over +-10."""
    f = disc_field(20000, 0.2, 0.3, 0.3, stream_seed(2, 0), "kroupa")
    return Workload("n20000_m20000_map8192", [f], 20000, 10.0, 8192)


def _batched_params(config_seed: int, index: int, n_lo: int, n_hi: int, ks_hi: float):
    """Per-field (N, kappa_*, gamma, kappa_s), resampled while |1 - kappa_s - gamma| < 0.01
    (a root runs to infinity at phi = 0 when gamma = 1 - kappa_s)."""
    draw = 0
    while True:
        u = uniform(stream_seed(config_seed, index, 1), 4, offset=4 * draw)
        n = int(round(math.exp(math.log(n_lo) + u[0] * math.log(n_hi / n_lo))))
        ks = 0.1 + 0.7 * u[1]
        g = 0.8 * u[2]
        kss = ks_hi * u[3]
        if abs(1.0 - kss - g) >= 0.01:
            return n, ks, g, kss
        draw += 1


def workload_batched(count: int = 256, msteps: int = 5000) -> Workload:
    """Many independent fields: N log-uniform in [50, 5000], kappa_* ~ U[0.1, 0.8],
    gamma ~ U[0, 0.8], kappa_s ~ U[0, 0.3], unit masses; m = 5000."""
    fields = []
    for i in range(count):
        n, ks, g, kss = _batched_params(3, i, 50, 5000, 0.3)
        fields.append(disc_field(n, ks, kss, g, stream_seed(3, i)))
    return Workload(f"batched{count}_m{msteps}", fields, msteps)


def served_requests(count: int = 500, rate_hz: float = 50.0):
    """Poisson arrivals (rate_hz) of requests with N log-uniform in [100, 20000],
    kappa_* ~ U[0.1, 0.8], gamma ~ U[0, 0.8], kappa_s = 0, log-uniform masses in
    [0.08, 1]; m = 200, 1024^2 crossing maps over +-10.  Returns [(t_arrival, Field)]."""
    gaps = -np.log1p(-uniform(stream_seed(4, 0, 2), count)) / rate_hz
    t = np.cumsum(gaps)
    out = []
    for i in range(count):
        n, ks, g, _ = _batched_params(4, i, 100, 20000, 0.0)
        out.append((float(t[i]), disc_field(n, ks, 0.0, g, stream_seed(4, i), "loguniform", 0.08, 1.0)))
    return out
