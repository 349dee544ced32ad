"""Seeded synthetic inputs shared by the tests, ``bench.py`` and the oracle checks.

This module holds no TaylorGrid arithmetic: no field evaluation, no loss, no
optimizer and no compositing. It only draws numbers and builds the synthetic
shapes, points, rays and scenes that stand in for the paper's datasets
(Stanford / Thingi10K / Synthetic Indoor Scene SDFs of Sec. 4.1 and
Synthetic-NeRF of Sec. 4.2, none of which is available here).

Counter-based generator
-----------------------
Every random number is a pure function of ``(seed, stream, index)``:

    mix(z)  = splitmix64 finaliser of z + 0x9E3779B97F4A7C15
              (Steele, Lea & Flood, "Fast splittable pseudorandom number
              generators", OOPSLA 2014; constants as published by Vigna)
    key     = mix(mix(mix(seed) + stream) + index)          (mod 2^64)
    U[0,1)  = (key >> 40) * 2^-24                            (exact in FP32)
    N(0,1)  = sqrt(-2 ln(1 - U_a)) * cos(2 pi U_b),
              U_a = U(seed, stream, 2i), U_b = U(seed, stream, 2i+1)

The CUDA library implements the same definition on the device (for the
device-side samplers of the fit jobs and the stratified ray samples); the
uniforms are bit-identical on both sides, the normals agree to FP32 rounding.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "splitmix64", "counter_u64", "uniform", "normal",
    "STREAM_INIT", "STREAM_QUERY", "STREAM_UPSTREAM", "STREAM_EVAL",
    "init_coefs", "uniform_points", "Shape", "sphere_shape", "union_shape",
    "sdf_points", "n_coefs", "blob_scene", "camera_rays", "random_rays",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream ids of the fixed draws (documented so that other implementations of
# the generator can reproduce the same inputs).
STREAM_INIT = 0xC0EF          # grid coefficient initialisation N(0, std)
STREAM_QUERY = 3              # query-only points U[0,1]^D
STREAM_UPSTREAM = 4           # upstream gradients dL/df ~ N(0,1)
STREAM_EVAL = 2               # fixed evaluation points of a fit
SLOTS = 16                    # draws reserved per sampled point


def n_coefs(dim: int, order: int) -> int:
    """Coefficients per vertex per channel: C(dim + order, order)."""
    return math.comb(dim + order, order)


def splitmix64(z) -> np.ndarray:
    """splitmix64 finaliser applied to ``z + golden`` (vectorised, wraps mod 2^64)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def counter_u64(seed: int, stream, index) -> np.ndarray:
    s = splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    with np.errstate(over="ignore"):
        k = splitmix64(s + np.asarray(stream, dtype=np.uint64))
        return splitmix64(k + np.asarray(index, dtype=np.uint64))


def uniform(seed: int, stream, index) -> np.ndarray:
    """U[0,1) with 24 random bits, returned as float32 (exactly representable)."""
    k = counter_u64(seed, stream, index)
    return ((k >> np.uint64(40)).astype(np.float64) * (1.0 / (1 << 24))).astype(np.float32)


def normal(seed: int, stream, index) -> np.ndarray:
    """N(0,1) by Box-Muller on the uniform pair (2i, 2i+1); float64 result."""
    index = np.asarray(index, dtype=np.uint64)
    ua = uniform(seed, stream, index * np.uint64(2)).astype(np.float64)
    ub = uniform(seed, stream, index * np.uint64(2) + np.uint64(1)).astype(np.float64)
    return np.sqrt(-2.0 * np.log1p(-ua)) * np.cos(2.0 * math.pi * ub)


def init_coefs(dim: int, res: int, order: int, channels: int, seed: int, std: float) -> np.ndarray:
    """Grid coefficients N(0, std) in the exchange layout [vertex][channel][k], float32."""
    n = res ** dim * channels * n_coefs(dim, order)
    return (normal(seed, STREAM_INIT, np.arange(n, dtype=np.uint64)) * std).astype(np.float32)


def uniform_points(seed: int, n: int, dim: int = 3, stream: int = STREAM_QUERY) -> np.ndarray:
    """n points U[0,1)^dim, row-major (n, dim) float32."""
    idx = np.arange(n * dim, dtype=np.uint64)
    return uniform(seed, stream, idx).reshape(n, dim)


# --------------------------------------------------------------------------
# Synthetic SDF targets (stand-ins for the paper's scanned shapes)
# --------------------------------------------------------------------------
@dataclass
class Shape:
    """Union of spheres (cx, cy, cz, r) and axis-aligned boxes (cx, cy, cz, hx, hy, hz)."""
    spheres: np.ndarray     # (S, 4) float32
    boxes: np.ndarray       # (B, 6) float32

    def sdf(self, x: np.ndarray) -> np.ndarray:
        """Ground-truth signed distance (float64), used only to build the samplers."""
        x = np.asarray(x, dtype=np.float64)
        d = np.full(x.shape[0], np.inf)
        for cx, cy, cz, r in self.spheres.astype(np.float64):
            d = np.minimum(d, np.linalg.norm(x - [cx, cy, cz], axis=1) - r)
        for cx, cy, cz, hx, hy, hz in self.boxes.astype(np.float64):
            q = np.abs(x - [cx, cy, cz]) - [hx, hy, hz]
            out = np.linalg.norm(np.maximum(q, 0.0), axis=1)
            d = np.minimum(d, out + np.minimum(q.max(axis=1), 0.0))
        return d

    def areas(self) -> np.ndarray:
        a = [4.0 * math.pi * float(r) ** 2 for r in self.spheres[:, 3]]
        a += [8.0 * (float(hx) * hy + float(hx) * hz + float(hy) * hz) for hx, hy, hz in self.boxes[:, 3:]]
        return np.asarray(a, dtype=np.float64)

    def area_cdf(self) -> np.ndarray:
        """Cumulative area fractions (float32), last entry forced to 1."""
        a = self.areas()
        c = np.cumsum(a) / a.sum()
        c[-1] = 1.0
        return c.astype(np.float32)


def sphere_shape(center=(0.5, 0.5, 0.5), radius: float = 0.3) -> Shape:
    return Shape(np.asarray([[*center, radius]], dtype=np.float32), np.zeros((0, 6), np.float32))


def union_shape(seed: int, n_spheres: int = 24, n_boxes: int = 8) -> Shape:
    """Seeded union: radii U[0.05,0.2], centres U[r,1-r]^3; box half-extents U[0.05,0.15]."""
    u = lambda i: float(uniform(seed, 0x5EED, i))
    sph = []
    i = 0
    for _ in range(n_spheres):
        r = 0.05 + 0.15 * u(i); i += 1
        c = [r + (1.0 - 2.0 * r) * u(i + k) for k in range(3)]; i += 3
        sph.append([*c, r])
    box = []
    for _ in range(n_boxes):
        h = [0.05 + 0.10 * u(i + k) for k in range(3)]; i += 3
        c = [h[k] + (1.0 - 2.0 * h[k]) * u(i + k) for k in range(3)]; i += 3
        box.append([*c, *h])
    return Shape(np.asarray(sph, np.float32).reshape(-1, 4), np.asarray(box, np.float32).reshape(-1, 6))


def _surface_candidates(shape: Shape, seed: int, stream, j: np.ndarray) -> np.ndarray:
    """One area-weighted surface point per index in j (slots 0, 1, 8, 9 of each point)."""
    base = j.astype(np.uint64) * np.uint64(SLOTS)
    u0 = uniform(seed, stream, base + np.uint64(0)).astype(np.float64)
    u1 = uniform(seed, stream, base + np.uint64(1)).astype(np.float64)
    u8 = uniform(seed, stream, base + np.uint64(8))
    u9 = uniform(seed, stream, base + np.uint64(9)).astype(np.float64)
    cdf = shape.area_cdf()
    prim = np.minimum(np.searchsorted(cdf, u8, side="right"), len(cdf) - 1)
    out = np.zeros((j.shape[0], 3))
    ns = shape.spheres.shape[0]
    for p in np.unique(prim):
        m = prim == p
        if p < ns:
            cx, cy, cz, r = shape.spheres[p].astype(np.float64)
            z = 1.0 - 2.0 * u0[m]
            s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
            ph = 2.0 * math.pi * u1[m]
            out[m] = np.stack([cx + r * s * np.cos(ph), cy + r * s * np.sin(ph), cz + r * z], 1)
        else:
            cx, cy, cz, hx, hy, hz = shape.boxes[p - ns].astype(np.float64)
            c = np.array([cx, cy, cz]); h = np.array([hx, hy, hz])
            fa = np.array([h[1] * h[2], h[0] * h[2], h[0] * h[1]])   # face areas / 4 per axis
            fcdf = np.cumsum(np.repeat(fa, 2)) / (2.0 * fa.sum())
            face = np.minimum(np.searchsorted(fcdf, u9[m], side="right"), 5)
            ax = face // 2
            sgn = np.where(face % 2 == 0, -1.0, 1.0)
            a1 = (ax + 1) % 3; a2 = (ax + 2) % 3
            pt = np.tile(c, (m.sum(), 1))
            rows = np.arange(m.sum())
            pt[rows, ax] = c[ax] + sgn * h[ax]
            pt[rows, a1] = c[a1] + (2.0 * u0[m] - 1.0) * h[a1]
            pt[rows, a2] = c[a2] + (2.0 * u1[m] - 1.0) * h[a2]
            out[m] = pt
    return out


def sdf_points(shape: Shape, seed: int, step: int, n: int, jitter: float = 0.01,
               attempts: int = 8) -> np.ndarray:
    """Fit batch: first half U[0,1]^3, second half near-surface points, float32 (n, 3).

    Near-surface point j: an area-weighted surface point (attempt a draws from
    stream step*256 + a), kept if it lies on the union's boundary
    (union SDF > -1e-6, i.e. not inside another primitive); after ``attempts``
    rejections the point falls back to a uniform one. Then N(0, jitter^2) noise
    per axis (normals 8j+2..8j+4, i.e. uniform slots 4..9 of stream step*256 + 255), clamped to [0,1]^3.
    """
    n_uni = n // 2
    pts = np.zeros((n, 3), dtype=np.float64)
    j = np.arange(n, dtype=np.uint64)
    base_stream = np.uint64(step) * np.uint64(256)
    uni = uniform(seed, base_stream + np.uint64(255), (j[:, None] * np.uint64(SLOTS) + np.arange(3, dtype=np.uint64)))
    pts[:n_uni] = uni[:n_uni]
    js = j[n_uni:]
    done = np.zeros(js.shape[0], bool)
    surf = uni[n_uni:].astype(np.float64).copy()
    for a in range(attempts):
        if done.all():
            break
        todo = np.nonzero(~done)[0]
        cand = _surface_candidates(shape, seed, base_stream + np.uint64(a), js[todo])
        ok = shape.sdf(cand) > -1e-6
        surf[todo[ok]] = cand[ok]
        done[todo[ok]] = True
    if jitter > 0:
        noise = normal(seed, base_stream + np.uint64(255),
                       (js[:, None] * np.uint64(SLOTS // 2) + np.uint64(2) + np.arange(3, dtype=np.uint64)))
        surf = surf + jitter * noise
    pts[n_uni:] = surf
    return np.clip(pts, 0.0, 1.0).astype(np.float32)


# --------------------------------------------------------------------------
# Synthetic radiance scene (stand-in for Synthetic-NeRF, Sec. 4.2)
# --------------------------------------------------------------------------
def _random_rotation(u: np.ndarray) -> np.ndarray:
    """Uniform random rotation from three uniforms (Shoemake's quaternion method)."""
    u1, u2, u3 = (float(v) for v in u)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                  math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3),
                  math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def blob_scene(seed: int, n_blobs: int = 64):
    """Anisotropic Gaussian blobs: returns (mu (B,3), inv_cov (B,3,3), amp (B,), rgb (B,3)), float64."""
    u = lambda i, k=1: uniform(seed, 0xB10B, np.arange(i, i + k, dtype=np.uint64)).astype(np.float64)
    mu, icov, amp, rgb = [], [], [], []
    i = 0
    for _ in range(n_blobs):
        mu.append(0.2 + 0.6 * u(i, 3)); i += 3
        s = 0.02 + 0.06 * u(i, 3); i += 3
        R = _random_rotation(u(i, 3)); i += 3
        icov.append(R @ np.diag(1.0 / s ** 2) @ R.T)
        amp.append(20.0 + 80.0 * u(i)[0]); i += 1
        rgb.append(u(i, 3)); i += 3
    return np.array(mu), np.array(icov), np.array(amp), np.array(rgb)


def camera_rays(n_cams: int, width: int, height: int, radius: float = 1.5, fov_deg: float = 50.0,
                center=(0.5, 0.5, 0.5), cams=None):
    """Pinhole cameras on a Fibonacci sphere looking at the centre; rays through pixel centres.

    Returns (origins (M,3), unit directions (M,3)) float32 for the selected cameras.
    """
    c = np.asarray(center, np.float64)
    cams = range(n_cams) if cams is None else cams
    golden = math.pi * (3.0 - math.sqrt(5.0))
    f = 0.5 * height / math.tan(math.radians(fov_deg) / 2.0)
    js, is_ = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    px = (is_ + 0.5 - width / 2.0) / f
    py = -(js + 0.5 - height / 2.0) / f
    O, Dd = [], []
    for k in cams:
        zc = 1.0 - 2.0 * (k + 0.5) / n_cams
        rr = math.sqrt(max(0.0, 1.0 - zc * zc))
        eye = c + radius * np.array([rr * math.cos(golden * k), rr * math.sin(golden * k), zc])
        fwd = (c - eye) / np.linalg.norm(c - eye)
        up0 = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) < 0.99 else np.array([0.0, 1.0, 0.0])
        right = np.cross(fwd, up0); right /= np.linalg.norm(right)
        up = np.cross(right, fwd)
        d = fwd[None, None] + px[..., None] * right + py[..., None] * up
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        O.append(np.broadcast_to(eye, d.shape).reshape(-1, 3))
        Dd.append(d.reshape(-1, 3))
    return np.concatenate(O).astype(np.float32), np.concatenate(Dd).astype(np.float32)


def random_rays(seed: int, n: int, radius: float = 1.5, center=(0.5, 0.5, 0.5), spread: float = 0.35):
    """n rays from random points on a sphere towards jittered points near the centre (float32)."""
    j = np.arange(n, dtype=np.uint64)
    u = lambda s: uniform(seed, 0x7A75, j * np.uint64(8) + np.uint64(s)).astype(np.float64)
    z = 1.0 - 2.0 * u(0)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ph = 2.0 * math.pi * u(1)
    c = np.asarray(center)
    o = c + radius * np.stack([r * np.cos(ph), r * np.sin(ph), z], 1)
    tgt = c + spread * (2.0 * np.stack([u(2), u(3), u(4)], 1) - 1.0)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)
