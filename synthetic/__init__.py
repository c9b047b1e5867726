"""Seeded synthetic inputs for the 2D parallel-beam reconstruction workloads.

This module is shared by the oracle's tests and by the GPU path's tests and
benchmark. It holds none of the reconstruction arithmetic (no projection, no
wavelet transform, no solver): only random draws, phantom rasterisation and the
catalogue of workload shapes.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the state advances by the golden
gamma 0x9E3779B97F4A7C15 and each output is the state passed through the
two-multiply finaliser. A uniform double is (x >> 11) * 2^-53 in [0, 1).
Gaussian draws use the Box-Muller transform.

Phantoms stand in for the paper's "Shepp-Logan type" 160x160 test object
(Section 4.1): a sum of seeded ellipses that lie inside the inscribed circle
of the unit square [-1/2, 1/2]^2, as the paper's object does. The pixel value
is the sum of the densities of the ellipses that contain the pixel centre.
Image storage is row-major, x[iy * n + ix], with iy = 0 at y = -1/2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
SEED_BASE = 0x5EED0000


def seed_for(config_index: int, problem_index: int = 0) -> int:
    """Seed of problem `problem_index` of workload `config_index`."""
    return SEED_BASE + 1000 * config_index + problem_index


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Sequential splitmix64 stream; `next_u64(k)` returns the next k outputs."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self, k: int) -> np.ndarray:
        steps = np.arange(1, k + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + steps * np.uint64(GAMMA)
            out = _mix(z)
        self.state = (self.state + k * GAMMA) & MASK64
        return out

    def uniform(self, k: int) -> np.ndarray:
        """k doubles in [0, 1)."""
        return (self.next_u64(k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform_in(self, lo: float, hi: float, k: int) -> np.ndarray:
        return lo + (hi - lo) * self.uniform(k)

    def normal(self, k: int) -> np.ndarray:
        """k standard normal draws (Box-Muller, cosine branch)."""
        u1 = 1.0 - self.uniform(k)  # (0, 1]: log is finite
        u2 = self.uniform(k)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


@dataclass(frozen=True)
class Ellipse:
    cx: float
    cy: float
    a: float
    b: float
    phi: float
    rho: float


def draw_ellipses(rng: SplitMix64, count: int) -> list[Ellipse]:
    """Seeded ellipses: centre ~ U(-0.3, 0.3)^2, semi-axes ~ U(0.03, 0.2),
    rotation ~ U(0, pi), density ~ U(0, 1); rejected until
    |centre| + max(a, b) <= 0.45 so the object sits inside the inscribed circle."""
    out: list[Ellipse] = []
    while len(out) < count:
        cx, cy, a, b, phi, rho = rng.uniform(6)
        cx = -0.3 + 0.6 * cx
        cy = -0.3 + 0.6 * cy
        a = 0.03 + 0.17 * a
        b = 0.03 + 0.17 * b
        phi = math.pi * phi
        if math.hypot(cx, cy) + max(a, b) <= 0.45:
            out.append(Ellipse(cx, cy, a, b, phi, rho))
    return out


def rasterise(ellipses: list[Ellipse], n: int) -> np.ndarray:
    """Image (n*n, float64): per pixel, the summed density of the ellipses that
    contain its centre."""
    h = 1.0 / n
    centres = -0.5 + (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(centres, centres)  # X varies along ix (columns), Y along iy
    img = np.zeros((n, n))
    for e in ellipses:
        dx, dy = X - e.cx, Y - e.cy
        cp, sp = math.cos(e.phi), math.sin(e.phi)
        u = (dx * cp + dy * sp) / e.a
        v = (-dx * sp + dy * cp) / e.b
        img += np.where(u * u + v * v <= 1.0, e.rho, 0.0)
    return img.reshape(-1)


def phantom(n: int, count: int, seed: int, texture: float = 0.0) -> np.ndarray:
    """Seeded ellipse phantom, optionally plus a per-pixel texture
    texture * U(-1, 1) over the whole image."""
    rng = SplitMix64(seed)
    img = rasterise(draw_ellipses(rng, count), n)
    if texture:
        img = img + texture * rng.uniform_in(-1.0, 1.0, n * n)
    return img


def noise_draws(M: int, seed: int) -> np.ndarray:
    """M standard-normal draws for the additive sinogram noise of a problem.
    A separate stream from the phantom's (seed offset by 2^32)."""
    return SplitMix64(seed + (1 << 32)).normal(M)


def uniform_noise_draws(M: int, seed: int) -> np.ndarray:
    """M draws from U(-1, 1): the paper's white-noise model (Section 4.3)."""
    return SplitMix64(seed + (1 << 32)).uniform_in(-1.0, 1.0, M)


def detectors_for(n: int) -> int:
    """ceil(sqrt(2) * n) bins of one pixel width: covers the image diagonal."""
    return math.isqrt(2 * n * n - 1) + 1


def levels_for(n: int, min_leaf: int = 12) -> int:
    """WMG level count l = L + 1 with L = max{L : 2^L | n, n / 2^L >= min_leaf}."""
    L = 0
    while n % (1 << (L + 1)) == 0 and n // (1 << (L + 1)) >= min_leaf:
        L += 1
    return L + 1


@dataclass(frozen=True)
class Problem:
    """One reconstruction problem: geometry, phantom recipe and noise level."""
    n: int
    m: int
    D: int
    levels: int
    ellipses: int
    noise: float          # sigma = noise * max|W x|
    seed: int
    texture: float = 0.0

    @property
    def N(self) -> int:
        return self.n * self.n

    @property
    def M(self) -> int:
        return self.m * self.D

    def image(self) -> np.ndarray:
        return phantom(self.n, self.ellipses, self.seed, self.texture)

    def noise_unit(self) -> np.ndarray:
        return noise_draws(self.M, self.seed)


@dataclass(frozen=True)
class Workload:
    name: str
    problems: tuple[Problem, ...] = field(default_factory=tuple)
    note: str = ""


def workload_small() -> Workload:
    """64x64 image, 90 angles, 91 bins, 10 ellipses, no noise, 3 levels."""
    return Workload("64x64_90ang_91det_noiseless",
                    (Problem(64, 90, 91, 3, 10, 0.0, seed_for(0)),))


def workload_mid(count: int = 1) -> Workload:
    """256x256 image, 180 angles, 363 bins, 20 ellipses, 1% Gaussian noise,
    5 levels; `count` independent phantoms of the same geometry."""
    return Workload("256x256_180ang_363det_noise1pct",
                    tuple(Problem(256, 180, 363, 5, 20, 0.01, seed_for(1, i))
                          for i in range(count)))


def workload_large() -> Workload:
    """1024x1024 image, 1024 angles, 1449 bins, 50 ellipses + 0.05 texture,
    0.5% Gaussian noise, 7 levels."""
    return Workload("1024x1024_1024ang_1449det_noise0.5pct",
                    (Problem(1024, 1024, 1449, 7, 50, 0.005, seed_for(2), 0.05),))


def workload_batched(count: int = 64) -> Workload:
    """Uneven batch: n ~ U{128,192,256,384,512}, m ~ U[60,360],
    D = ceil(sqrt(2) n), levels by the leaf-side rule, 10 + n/32 ellipses,
    1% noise."""
    rng = SplitMix64(seed_for(3, 999))
    sizes = (128, 192, 256, 384, 512)
    probs = []
    for i in range(count):
        n = sizes[int(rng.uniform(1)[0] * len(sizes))]
        m = 60 + int(rng.uniform(1)[0] * 301)
        probs.append(Problem(n, m, detectors_for(n), levels_for(n), 10 + n // 32,
                             0.01, seed_for(3, i)))
    return Workload("batched64_n128-512_m60-360", tuple(probs))


def workload_serving(count: int = 2000) -> tuple[Workload, np.ndarray]:
    """Request stream: n ~ U{128,256,512,1024,2048}, m ~ U[90,720], 1% noise.
    Returns the workload and the unit-rate exponential inter-arrival draws
    (scale them by 1/rate to get Poisson arrival gaps)."""
    rng = SplitMix64(seed_for(4, 999))
    sizes = (128, 256, 512, 1024, 2048)
    probs = []
    for i in range(count):
        n = sizes[int(rng.uniform(1)[0] * len(sizes))]
        m = 90 + int(rng.uniform(1)[0] * 631)
        probs.append(Problem(n, m, detectors_for(n), levels_for(n), 10 + n // 32,
                             0.01, seed_for(4, i)))
    gaps = -np.log(1.0 - rng.uniform(count))
    return Workload("serving2000_n128-2048_m90-720", tuple(probs)), gaps
