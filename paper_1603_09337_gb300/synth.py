"""Seeded synthetic binary images shaped like the paper's workload.

The paper measures on 512 x 512 binary images of noisy shapes (Sec. 4.3) that
are not published; these generators stand in for them.  Everything here is
integer arithmetic on a SplitMix64 stream, so x86 and Arm hosts produce the
same bytes for the same seed.  The module holds none of the filter's own
arithmetic: it only draws inputs, which both the CUDA library and the CPU
oracle then receive unchanged.

Image recipe (``shapes_image``): the union of discs and ellipses (semi-axes
uniform in a range, orientation uniform), minus a few disc-shaped holes
centred on object pixels, then a random boundary jitter (each pixel copies the
pixel at a random offset in [-j, j]^2, outside = background), then
salt-and-pepper noise (each pixel flipped with probability k / 1000).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
BASE_SEED = 0x160309337


def image_seed(config: int, index: int) -> int:
    """Seed of image `index` of workload `config`."""
    return (BASE_SEED ^ (config << 40) ^ index) & MASK64


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood 2014): state += gamma, then mix."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    @staticmethod
    def _mix_scalar(z: int) -> int:
        z = ((z ^ (z >> 30)) * _M1) & MASK64
        z = ((z ^ (z >> 27)) * _M2) & MASK64
        return z ^ (z >> 31)

    def next(self) -> int:
        self.state = (self.state + GAMMA) & MASK64
        return self._mix_scalar(self.state)

    def block(self, n: int) -> np.ndarray:
        """The next n outputs as a uint64 array (same values as n calls of next())."""
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + idx * np.uint64(GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * GAMMA) & MASK64
        return z

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive), by 32-bit multiply-shift."""
        span = hi - lo + 1
        return lo + (((self.next() >> 32) * span) >> 32)

    def direction(self, radius: int = 64) -> tuple[int, int]:
        """A non-zero integer vector drawn uniformly from the disc of the given radius."""
        while True:
            u = self.randint(-radius, radius)
            v = self.randint(-radius, radius)
            if 0 < u * u + v * v <= radius * radius:
                return u, v


def _paint_ellipse(img: np.ndarray, cx: int, cy: int, a: int, b: int, u: int, v: int, val: int):
    """Set img to val on the integer points of an ellipse with semi-axes a, b whose
    a-axis points along (u, v).  Exact integer inside-test."""
    h, w = img.shape
    R = max(a, b)
    x0, x1 = max(0, cx - R), min(w - 1, cx + R)
    y0, y1 = max(0, cy - R), min(h - 1, cy + R)
    if x0 > x1 or y0 > y1:
        return
    dx = np.arange(x0, x1 + 1, dtype=np.int64)[None, :] - cx
    dy = np.arange(y0, y1 + 1, dtype=np.int64)[:, None] - cy
    p = dx * u + dy * v
    q = -dx * v + dy * u
    inside = (b * b) * p * p + (a * a) * q * q <= (a * a) * (b * b) * (u * u + v * v)
    sub = img[y0:y1 + 1, x0:x1 + 1]
    sub[inside] = val


def shapes_image(seed: int, w: int, h: int, n_shapes: int, axis_lo: int, axis_hi: int,
                 n_holes: int = 0, hole_lo: int = 5, hole_hi: int = 20, jitter: int = 2,
                 noise_permille: int = 50) -> np.ndarray:
    """A w x h uint8 0/1 image following the recipe in the module docstring."""
    rng = SplitMix64(seed)
    img = np.zeros((h, w), np.uint8)
    for _ in range(n_shapes):
        cx = rng.randint(0, w - 1)
        cy = rng.randint(0, h - 1)
        a = rng.randint(axis_lo, axis_hi)
        if rng.next() >> 63:           # ellipse
            b = rng.randint(axis_lo, axis_hi)
            u, v = rng.direction()
        else:                          # disc
            b, u, v = a, 1, 0
        _paint_ellipse(img, cx, cy, a, b, u, v, 1)
    for _ in range(n_holes):
        obj = np.flatnonzero(img)
        if obj.size == 0:
            break
        at = int(obj[rng.randint(0, obj.size - 1)])
        rad = rng.randint(hole_lo, hole_hi)
        _paint_ellipse(img, at % w, at // w, rad, rad, 1, 0, 0)
    if jitter > 0:
        span = 2 * jitter + 1
        z = rng.block(w * h).reshape(h, w)
        ox = ((z >> np.uint64(32)) % np.uint64(span)).astype(np.int64) - jitter
        oy = ((z & np.uint64(0xFFFFFFFF)) % np.uint64(span)).astype(np.int64) - jitter
        ys, xs = np.mgrid[0:h, 0:w]
        sx, sy = xs + ox, ys + oy
        ok = (sx >= 0) & (sx < w) & (sy >= 0) & (sy < h)
        out = np.zeros_like(img)
        out[ok] = img[sy[ok], sx[ok]]
        img = out
    if noise_permille > 0:
        thresh = np.uint64((noise_permille << 32) // 1000)
        z = rng.block(w * h).reshape(h, w)
        flip = (z >> np.uint64(32)) < thresh
        img = img ^ flip.astype(np.uint8)
    return img


def constraint_points(seed: int, X: np.ndarray, count: int) -> np.ndarray:
    """A 0/1 image holding `count` object pixels of X drawn uniformly without replacement."""
    rng = SplitMix64(seed ^ 0xC0C0C0C0)
    obj = np.flatnonzero(X)
    C = np.zeros(X.size, np.uint8)
    count = min(count, obj.size)
    pool = obj.copy()
    for i in range(count):                  # partial Fisher-Yates shuffle
        j = rng.randint(i, pool.size - 1)
        pool[i], pool[j] = pool[j], pool[i]
        C[pool[i]] = 1
    return C.reshape(X.shape)


@dataclass
class Job:
    """One image to smooth: X (h, w) uint8 0/1, optional constraint C, order rmax."""

    X: np.ndarray
    rmax: int
    C: np.ndarray | None = None
    D: np.ndarray | None = None
    conn: int = 8
    meta: dict = field(default_factory=dict)


# --- the five workloads -------------------------------------------------------

def single_512(index: int = 0) -> Job:
    """One 512 x 512 image: 12 discs/ellipses (semi-axes 20-90), 6 holes, 2-px
    jitter, 5 % salt-and-pepper; rmax = 3, no constraint."""
    seed = image_seed(0, index)
    X = shapes_image(seed, 512, 512, 12, 20, 90, n_holes=6, jitter=2, noise_permille=50)
    return Job(X, 3, meta={"seed": seed})


def batch_512(n: int = 256, first: int = 0) -> list[Job]:
    """n images as single_512 with noise uniform in 2-10 %, rmax = 5, and a
    constraint set of 50 object pixels each."""
    jobs = []
    for i in range(first, first + n):
        seed = image_seed(1, i)
        noise = SplitMix64(seed ^ 0x5A5A).randint(20, 100)
        X = shapes_image(seed, 512, 512, 12, 20, 90, n_holes=6, jitter=2, noise_permille=noise)
        C = constraint_points(seed, X, 50)
        jobs.append(Job(X, 5, C=C, meta={"seed": seed, "noise_permille": noise}))
    return jobs


def large_image(side: int, index: int = 0) -> Job:
    """One side x side image of 2,000 discs/ellipses (semi-axes 5-200), 3 %
    noise, no holes; rmax = 10."""
    seed = image_seed(2, (side << 8) ^ index)
    X = shapes_image(seed, side, side, 2000, 5, 200, n_holes=0, jitter=0, noise_permille=30)
    return Job(X, 10, meta={"seed": seed})


def ragged_batch(n: int = 1024, first: int = 0, lo: int = 128, hi: int = 2048) -> list[Job]:
    """n images with width and height each uniform in [lo, hi]; shape and hole
    counts scaled to area; 5 % noise; rmax uniform in 1-8."""
    jobs = []
    for i in range(first, first + n):
        seed = image_seed(3, i)
        rng = SplitMix64(seed ^ 0x3333)
        w = rng.randint(lo, hi)
        h = rng.randint(lo, hi)
        rmax = rng.randint(1, 8)
        area = w * h
        n_shapes = max(1, (12 * area + 131072) // 262144)
        n_holes = (6 * area + 131072) // 262144
        ahi = max(20, min(90, min(w, h) // 3))
        X = shapes_image(seed, w, h, n_shapes, 20, ahi, n_holes=n_holes, jitter=2,
                         noise_permille=50)
        jobs.append(Job(X, rmax, meta={"seed": seed}))
    return jobs


def volume(seed: int, d: int, h: int, w: int, n_balls: int, rlo: int, rhi: int,
           noise_permille: int) -> np.ndarray:
    """A (d, h, w) 0/1 volume: union of n_balls balls (centre uniform in the box,
    radius uniform in [rlo, rhi], exact integer inside test), then each voxel
    flipped with probability noise_permille / 1000."""
    rng = SplitMix64(seed)
    V = np.zeros((d, h, w), np.uint8)
    for _ in range(n_balls):
        cz, cy, cx = rng.randint(0, d - 1), rng.randint(0, h - 1), rng.randint(0, w - 1)
        r = rng.randint(rlo, rhi)
        z0, z1 = max(0, cz - r), min(d, cz + r + 1)
        y0, y1 = max(0, cy - r), min(h, cy + r + 1)
        x0, x1 = max(0, cx - r), min(w, cx + r + 1)
        zz, yy, xx = np.ogrid[z0:z1, y0:y1, x0:x1]
        inside = (zz - cz) ** 2 + (yy - cy) ** 2 + (xx - cx) ** 2 <= r * r
        V[z0:z1, y0:y1, x0:x1] |= inside.astype(np.uint8)
    flip = (rng.block(d * h * w) % np.uint64(1000)) < np.uint64(noise_permille)
    return V ^ flip.reshape(d, h, w).astype(np.uint8)


def volume_batch(n: int = 16, side: int = 128, first: int = 0) -> list[Job]:
    """n volumes of side^3 voxels: balls of radius 4-16 (about 40 per 128^3,
    scaled to volume), 3 % noise; rmax = 4.  Job.X has shape (d, h, w)."""
    jobs = []
    nb = max(1, (40 * side ** 3 + (1 << 20)) // (1 << 21))
    for i in range(first, first + n):
        seed = image_seed(5, i)
        jobs.append(Job(volume(seed, side, side, side, nb, 4, 16, 30), 4, meta={"seed": seed}))
    return jobs


def small_random(seed: int, w: int, h: int, density_permille: int = 500) -> np.ndarray:
    """Independent Bernoulli pixels (for tiny brute-force checks)."""
    rng = SplitMix64(seed)
    z = rng.block(w * h).reshape(h, w)
    return ((z >> np.uint64(32)) < np.uint64((density_permille << 32) // 1000)).astype(np.uint8)
