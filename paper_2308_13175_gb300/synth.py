"""Seeded synthetic inputs: point clouds, query batches and grid values.

This module only draws inputs. It holds none of the fitting arithmetic (no cell
lookup, interpolation, loss, nearest-neighbour search or optimiser), so that the
CUDA path and the FP64 oracle can both consume the same inputs without sharing
any of the method's code.

The clouds stand in for the shape and scene benchmarks of the paper (Sec. 4,
"Datasets and Metrics"), which are not available here:

* ``sphere_cloud``       - 5,000 points on a radius-0.5 sphere (small parity case).
* ``object_cloud``       - union of 3 random ellipsoids and a torus (single object).
* ``room_cloud``         - a 10 x 8 x 3 m room with 60 boxes and cylinders (scene).
* ``superquadric_cloud`` - union of 10 random superquadrics (large single object).
* ``shape_collection``   - many small unions of ellipsoids, boxes and tori.

Every surface is sampled uniformly by area (rejection on the area element of a
parametrisation); for unions only the surface points that lie outside all other
primitives are kept.  All coordinates are returned as float32 in [-1, 1]^3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    qv = rng.normal(size=4)
    qv /= np.linalg.norm(qv)
    w, x, y, z = qv
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


# ---------------------------------------------------------------- primitives
@dataclass
class Primitive:
    kind: str            # "ellipsoid" | "torus" | "box" | "cylinder" | "superquadric"
    center: np.ndarray   # (3,)
    rot: np.ndarray      # (3,3) local -> world
    params: tuple

    def to_local(self, x: np.ndarray) -> np.ndarray:
        return (x - self.center) @ self.rot

    def inside(self, x: np.ndarray) -> np.ndarray:
        p = self.to_local(x)
        if self.kind == "ellipsoid":
            a = np.asarray(self.params)
            return np.sum((p / a) ** 2, axis=1) < 1.0
        if self.kind == "torus":
            big, small = self.params
            rho = np.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2)
            return (rho - big) ** 2 + p[:, 2] ** 2 < small * small
        if self.kind == "box":
            half = np.asarray(self.params)
            return np.all(np.abs(p) < half, axis=1)
        if self.kind == "cylinder":
            radius, half_h = self.params
            return (p[:, 0] ** 2 + p[:, 1] ** 2 < radius * radius) & (np.abs(p[:, 2]) < half_h)
        if self.kind == "superquadric":
            a, b, c, e1, e2 = self.params
            with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
                xy = np.abs(p[:, 0] / a) ** (2.0 / e2) + np.abs(p[:, 1] / b) ** (2.0 / e2)
                val = xy ** (e2 / e1) + np.abs(p[:, 2] / c) ** (2.0 / e1)
            return val < 1.0
        raise ValueError(self.kind)

    # Parametrisation (u, v) in [0,1]^2 -> local surface point; used with
    # rejection on the numerical area element to get area-uniform samples.
    def _param(self, u: np.ndarray, v: np.ndarray) -> np.ndarray:
        if self.kind == "ellipsoid":
            a = np.asarray(self.params)
            th = np.arccos(1.0 - 2.0 * u)
            ph = 2.0 * math.pi * v
            return np.stack([a[0] * np.sin(th) * np.cos(ph), a[1] * np.sin(th) * np.sin(ph),
                             a[2] * np.cos(th)], axis=1)
        if self.kind == "torus":
            big, small = self.params
            th = 2.0 * math.pi * u
            ph = 2.0 * math.pi * v
            rr = big + small * np.cos(ph)
            return np.stack([rr * np.cos(th), rr * np.sin(th), small * np.sin(ph)], axis=1)
        if self.kind == "superquadric":
            a, b, c, e1, e2 = self.params
            eta = (u - 0.5) * math.pi
            om = (v * 2.0 - 1.0) * math.pi

            def spow(t, e):
                return np.sign(t) * np.abs(t) ** e
            ce, se = spow(np.cos(eta), e1), spow(np.sin(eta), e1)
            co, so = spow(np.cos(om), e2), spow(np.sin(om), e2)
            return np.stack([a * ce * co, b * ce * so, c * se], axis=1)
        raise ValueError(self.kind)

    def sample_surface(self, n: int, rng: np.random.Generator) -> np.ndarray:
        if self.kind in ("box", "cylinder"):
            return self._sample_flat(n, rng)
        if self.kind == "superquadric":
            # Its area element is too peaked for rejection: draw 3n parameter
            # pairs and resample n of them in proportion to the area element.
            eps = 1e-4
            m = max(3 * n, 4096)
            u, v = rng.random(m), rng.random(m)
            dens = self._area_element(u, v, eps)
            idx = rng.choice(m, size=n, p=dens / dens.sum())
            return self._param(np.clip(u[idx], eps, 1 - eps), np.clip(v[idx], eps, 1 - eps)) @ self.rot.T + self.center
        out = []
        got = 0
        eps = 1e-4
        # Estimate the maximum area element once.
        u0, v0 = rng.random(4096), rng.random(4096)
        dens_max = self._area_element(u0, v0, eps).max() * 1.25
        while got < n:
            m = max(2 * (n - got), 1024)
            u, v = rng.random(m), rng.random(m)
            dens = self._area_element(u, v, eps)
            keep = rng.random(m) * dens_max < dens
            pts = self._param(u[keep], v[keep])
            out.append(pts)
            got += len(pts)
        loc = np.concatenate(out)[:n]
        return loc @ self.rot.T + self.center

    def _area_element(self, u, v, eps):
        u = np.clip(u, eps, 1 - eps)
        v = np.clip(v, eps, 1 - eps)
        du = (self._param(u + eps, v) - self._param(u - eps, v)) / (2 * eps)
        dv = (self._param(u, v + eps) - self._param(u, v - eps)) / (2 * eps)
        return np.linalg.norm(np.cross(du, dv), axis=1)

    def _sample_flat(self, n, rng):
        if self.kind == "box":
            hx, hy, hz = self.params
            areas = np.array([hy * hz, hy * hz, hx * hz, hx * hz, hx * hy, hx * hy])
            face = rng.choice(6, size=n, p=areas / areas.sum())
            p = (rng.random((n, 3)) * 2 - 1) * np.array([hx, hy, hz])
            axis = face // 2
            sign = np.where(face % 2 == 0, -1.0, 1.0)
            half = np.array([hx, hy, hz])
            p[np.arange(n), axis] = sign * half[axis]
        else:
            radius, half_h = self.params
            a_side = 2 * math.pi * radius * 2 * half_h
            a_cap = math.pi * radius * radius
            part = rng.choice(3, size=n, p=np.array([a_side, a_cap, a_cap]) / (a_side + 2 * a_cap))
            th = 2 * math.pi * rng.random(n)
            rr = radius * np.sqrt(rng.random(n))
            z = (rng.random(n) * 2 - 1) * half_h
            p = np.stack([rr * np.cos(th), rr * np.sin(th), z], axis=1)
            side = part == 0
            p[side, 0] = radius * np.cos(th[side])
            p[side, 1] = radius * np.sin(th[side])
            p[part == 1, 2] = -half_h
            p[part == 2, 2] = half_h
        return p @ self.rot.T + self.center

    def bound(self) -> float:
        """Radius of a ball around the centre that holds the whole primitive
        (inside() is False beyond it); infinite when there is none."""
        if self.kind == "ellipsoid":
            return float(max(self.params))
        if self.kind == "torus":
            return float(self.params[0] + self.params[1])
        if self.kind in ("box", "superquadric"):
            return float(np.linalg.norm(self.params[:3]))
        if self.kind == "cylinder":
            return float(math.hypot(self.params[0], self.params[1]))
        return math.inf

    def area(self, rng: np.random.Generator) -> float:
        if self.kind == "box":
            hx, hy, hz = self.params
            return 8 * (hx * hy + hy * hz + hx * hz)
        if self.kind == "cylinder":
            radius, half_h = self.params
            return 2 * math.pi * radius * 2 * half_h + 2 * math.pi * radius * radius
        u, v = rng.random(20000), rng.random(20000)
        return float(self._area_element(u, v, 1e-4).mean())


def union_surface(prims: list, n: int, rng: np.random.Generator,
                  open_inside: Primitive | None = None) -> np.ndarray:
    """Area-uniform points on the boundary of a union of primitives."""
    areas = np.array([p.area(rng) for p in prims])
    chunks = []
    got = 0
    while got < n:
        m = int((n - got) * 1.3) + 256
        counts = rng.multinomial(m, areas / areas.sum())
        for i, (p, c) in enumerate(zip(prims, counts)):
            if c == 0:
                continue
            pts = p.sample_surface(int(c), rng)
            keep = np.ones(len(pts), dtype=bool)
            for k, other in enumerate(prims):
                if k != i and other.kind != "room":
                    # Only points within the other primitive's bounding ball can lie inside it.
                    near = np.flatnonzero(np.sum((pts - other.center) ** 2, axis=1) < other.bound() ** 2)
                    if len(near):
                        keep[near] &= ~other.inside(pts[near])
            chunks.append(pts[keep])
            got += int(keep.sum())
    pts = np.concatenate(chunks)
    pts = pts[rng.permutation(len(pts))[:n]]
    return pts


def _finish(pts: np.ndarray, noise_std: float, rng: np.random.Generator) -> np.ndarray:
    if noise_std > 0:
        pts = pts + rng.normal(scale=noise_std, size=pts.shape)
    return np.clip(pts, -1.0, 1.0).astype(np.float32)


# ------------------------------------------------------------------- clouds
def sphere_cloud(n: int = 5000, radius: float = 0.5, seed: int = 0,
                 center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Points uniform on a sphere (area-uniform via normalised Gaussians)."""
    rng = _rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return (np.asarray(center) + radius * d).astype(np.float32)


def object_primitives(seed: int) -> list:
    rng = _rng(seed + 1000)
    prims = []
    for _ in range(3):
        prims.append(Primitive("ellipsoid", rng.uniform(-0.4, 0.4, 3), _random_rotation(rng),
                               tuple(rng.uniform(0.1, 0.4, 3))))
    prims.append(Primitive("torus", rng.uniform(-0.3, 0.3, 3), _random_rotation(rng), (0.3, 0.08)))
    return prims


def object_cloud(n: int = 100_000, seed: int = 1, noise_std: float = 0.001) -> np.ndarray:
    """Union of 3 random ellipsoids (semi-axes U[0.1,0.4]) and a torus (R=0.3, r=0.08)."""
    rng = _rng(seed)
    return _finish(union_surface(object_primitives(seed), n, rng), noise_std, rng)


def room_cloud(n: int = 10_000_000, seed: int = 2, noise_std_m: float = 0.002) -> np.ndarray:
    """A 10 x 8 x 3 m room (floor, ceiling, 4 walls) with 60 random boxes and
    cylinders (sizes U[0.2, 1.5] m) standing on the floor, scaled by 0.2 about
    the room centre so that it spans [-1,1] x [-0.8,0.8] x [-0.3,0.3]."""
    rng = _rng(seed)
    room = (10.0, 8.0, 3.0)
    objs = []
    for _ in range(60):
        size = rng.uniform(0.2, 1.5, 3)
        size[2] = min(size[2], 2.9)
        c = np.array([rng.uniform(size[0] / 2, room[0] - size[0] / 2),
                      rng.uniform(size[1] / 2, room[1] - size[1] / 2), size[2] / 2])
        yaw = rng.uniform(0, 2 * math.pi)
        rot = np.array([[math.cos(yaw), -math.sin(yaw), 0], [math.sin(yaw), math.cos(yaw), 0], [0, 0, 1]])
        if rng.random() < 0.5:
            objs.append(Primitive("box", c, rot, tuple(size / 2)))
        else:
            objs.append(Primitive("cylinder", c, rot, (size[0] / 2, size[2] / 2)))
    # Room shell: six faces of the room box, sampled by area.
    shell = Primitive("box", np.array(room) / 2, np.eye(3), tuple(np.array(room) / 2))
    shell_area = shell.area(rng)
    obj_areas = np.array([o.area(rng) for o in objs])
    total = shell_area + obj_areas.sum()
    chunks = []
    got = 0
    while got < n:
        m = int((n - got) * 1.2) + 256
        counts = rng.multinomial(m, np.concatenate([[shell_area], obj_areas]) / total)
        for i, c in enumerate(counts):
            if c == 0:
                continue
            src = shell if i == 0 else objs[i - 1]
            pts = src.sample_surface(int(c), rng)
            keep = np.ones(len(pts), dtype=bool)
            for k, o in enumerate(objs):
                if k != i - 1:
                    keep &= ~o.inside(pts)
            chunks.append(pts[keep])
            got += int(keep.sum())
    pts = np.concatenate(chunks)
    pts = pts[rng.permutation(len(pts))[:n]]
    pts = pts + rng.normal(scale=noise_std_m, size=pts.shape)
    pts = (pts - np.array(room) / 2) * 0.2
    return np.clip(pts, -1.0, 1.0).astype(np.float32)


def superquadric_cloud(n: int = 2_000_000, seed: int = 4, noise_std: float = 0.001) -> np.ndarray:
    """Union of 10 superquadrics (exponents U[0.3,3], scales U[0.1,0.4], centres U[-0.5,0.5]^3)."""
    rng = _rng(seed)
    prims = []
    for _ in range(10):
        a, b, c = rng.uniform(0.1, 0.4, 3)
        e1, e2 = rng.uniform(0.3, 3.0, 2)
        prims.append(Primitive("superquadric", rng.uniform(-0.5, 0.5, 3), _random_rotation(rng),
                               (a, b, c, e1, e2)))
    return _finish(union_surface(prims, n, rng), noise_std, rng)


def shape_collection(n_shapes: int = 64, seed: int = 3, j_min: int = 5000, j_max: int = 500_000,
                     resolutions=(128, 256, 512), noise_std: float = 0.001):
    """Many independent shapes of uneven size: each a union of 1-5 ellipsoids,
    boxes or tori, with a log-uniform point count and a random resolution."""
    rng = _rng(seed)
    shapes = []
    for k in range(n_shapes):
        n_prim = int(rng.integers(1, 6))
        prims = []
        for _ in range(n_prim):
            kind = ("ellipsoid", "box", "torus")[int(rng.integers(0, 3))]
            c = rng.uniform(-0.4, 0.4, 3)
            rot = _random_rotation(rng)
            if kind == "ellipsoid":
                prims.append(Primitive(kind, c, rot, tuple(rng.uniform(0.1, 0.4, 3))))
            elif kind == "box":
                prims.append(Primitive(kind, c, rot, tuple(rng.uniform(0.08, 0.35, 3))))
            else:
                big = rng.uniform(0.15, 0.35)
                prims.append(Primitive(kind, c, rot, (big, rng.uniform(0.04, 0.4 * big))))
        j = int(round(math.exp(rng.uniform(math.log(j_min), math.log(j_max)))))
        res = int(resolutions[int(rng.integers(0, len(resolutions)))])
        pts = _finish(union_surface(prims, j, rng), noise_std, rng)
        shapes.append((pts, res))
    return shapes


# ------------------------------------------------------------ query batches
def gaussian_queries(points: np.ndarray, n: int, sigma, seed: int):
    """Queries q = s_j + sigma_j * N(0, I) around uniformly chosen points j.

    Returns (q float32 (n,3), j int64 (n,)).  ``sigma`` is a scalar or a per-point
    array.  Used for parity inputs; the fitting loop draws its own queries with
    the counter-based sampler of the library."""
    rng = _rng(seed)
    j = rng.integers(0, len(points), size=n)
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (len(points),))[j]
    q = points[j].astype(np.float64) + sig[:, None] * rng.normal(size=(n, 3))
    return q.astype(np.float32), j


def sphere_field(coords_ijk: np.ndarray, R: int, radius: float, noise_std: float, seed: int,
                 center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Grid values |v - c| - radius + noise at integer vertex coordinates.

    The noise of a vertex depends only on (seed, vertex): one normal draw per
    vertex of the whole (R+1)^3 grid, indexed by i + (R+1)(j + (R+1)k), so the
    same vertex gets the same value whichever subset of vertices is asked for."""
    h = 2.0 / R
    ijk = np.asarray(coords_ijk, dtype=np.int64)
    v = -1.0 + h * ijk.astype(np.float64)
    d = np.linalg.norm(v - np.asarray(center), axis=1) - radius
    if noise_std > 0:
        n1 = R + 1
        noise = _rng(seed).standard_normal(n1 ** 3, dtype=np.float32)
        key = ijk[:, 0] + n1 * (ijk[:, 1] + n1 * ijk[:, 2])
        d = d + noise_std * noise[key].astype(np.float64)
    return d.astype(np.float32)


def all_vertices(R: int) -> np.ndarray:
    """Integer coordinates of every vertex of the (R+1)^3 grid, key order."""
    n1 = R + 1
    k = np.arange(n1 ** 3, dtype=np.int64)
    return np.stack([k % n1, (k // n1) % n1, k // (n1 * n1)], axis=1)


def random_field(coords_ijk: np.ndarray, scale: float, seed: int) -> np.ndarray:
    """Independent uniform values in [-scale, scale] per vertex (stress input)."""
    return (_rng(seed).uniform(-scale, scale, size=len(coords_ijk))).astype(np.float32)
