"""Synthetic spinning-LiDAR frames (ray-cast street scene + snow / outliers).

Recipe for one frame (``lidar_frame``), all randomness from PCG64 seeded RNGs:

* Sensor at (0, 0, 1.8 m); ``beams`` elevation channels evenly spaced over
  [-25 deg, +15 deg]; 0.2 deg azimuth steps (1,800 columns); ranges above 80 m
  are dropped; Gaussian range noise sigma = 2 cm along each ray.
* Scene: ground plane z = 0; 10-30 boxes ("cars", about 4.5 x 1.8 x 1.5 m,
  +-10 % per dimension, random yaw, 5-60 m from the sensor) and 20-60 vertical
  cylinders ("poles", radius 0.1-0.3 m, height 3-8 m, 3-70 m away).
* One sweep has at most beams x 1,800 rays, so a frame accumulates S sweeps
  with the azimuth phase offset by 0.2/S deg per sweep; S is the smallest count
  whose hits cover the frame's target size, and the surface hits are then
  subsampled to exactly the surface share of the target.
* Snow (label 2): a fraction of the target, uniform in direction over the
  vertical field of view (uniform in sin(elevation)) with volumetric density
  proportional to 1/r for r in [0.5, 15] m, i.e. a radial pdf proportional to r;
  flakes below the ground plane are redrawn.
* Uniform outliers (label 1): uniform in the surface bounding box scaled 1.2x.

``lidar_batch`` reproduces the 64-frame batching workload (32 beams, target
U[60k, 130k] points, snow 5-20 %, seeds 1000 + i).  ``serving_stream`` builds
the Poisson request stream of the serving workload from a small pool of
ray-cast scenes, re-posed and re-noised per request so that 2,000 requests do
not need 2,000 ray casts.
"""

from __future__ import annotations

import dataclasses

import numpy as np

SENSOR_Z = 1.8
MAX_RANGE = 80.0
AZ_STEP_DEG = 0.2


@dataclasses.dataclass
class _Scene:
    boxes: np.ndarray      # [B, 7]: cx, cy, yaw, hx, hy, hz(height), unused
    cyls: np.ndarray       # [C, 4]: cx, cy, radius, height


def _make_scene(rng) -> _Scene:
    nb = int(rng.integers(10, 31))
    nc = int(rng.integers(20, 61))
    r = rng.uniform(5.0, 60.0, nb)
    a = rng.uniform(0.0, 2 * np.pi, nb)
    dims = np.array([4.5, 1.8, 1.5]) * rng.uniform(0.9, 1.1, size=(nb, 3))
    boxes = np.stack([r * np.cos(a), r * np.sin(a), rng.uniform(0.0, np.pi, nb),
                      dims[:, 0] / 2, dims[:, 1] / 2, dims[:, 2], np.zeros(nb)], axis=1)
    rc = rng.uniform(3.0, 70.0, nc)
    ac = rng.uniform(0.0, 2 * np.pi, nc)
    cyls = np.stack([rc * np.cos(ac), rc * np.sin(ac), rng.uniform(0.1, 0.3, nc),
                     rng.uniform(3.0, 8.0, nc)], axis=1)
    return _Scene(boxes, cyls)


def _ray_dirs(beams: int, phase_deg: float):
    el = np.deg2rad(np.linspace(-25.0, 15.0, beams))
    az = np.deg2rad(np.arange(int(round(360.0 / AZ_STEP_DEG))) * AZ_STEP_DEG + phase_deg)
    E, A = np.meshgrid(el, az, indexing="ij")
    d = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], axis=-1)
    return d.reshape(-1, 3)


def _cast(scene: _Scene, d: np.ndarray) -> np.ndarray:
    """Nearest hit distance per ray (inf if none within range)."""
    t = np.full(d.shape[0], np.inf)
    down = d[:, 2] < 0
    t[down] = -SENSOR_Z / d[down, 2]
    ox, oy, oz = 0.0, 0.0, SENSOR_Z
    chunk = 16384
    for s in range(0, d.shape[0], chunk):
        dd = d[s:s + chunk]
        tc = t[s:s + chunk]
        # boxes: slab test in the box frame
        b = scene.boxes
        cy_, sy_ = np.cos(b[:, 2]), np.sin(b[:, 2])
        px, py = ox - b[:, 0], oy - b[:, 1]
        lox = cy_ * px + sy_ * py
        loy = -sy_ * px + cy_ * py
        dx = dd[:, None, 0] * cy_ + dd[:, None, 1] * sy_
        dy = -dd[:, None, 0] * sy_ + dd[:, None, 1] * cy_
        dz = np.repeat(dd[:, None, 2], len(b), axis=1)
        with np.errstate(divide="ignore", invalid="ignore"):
            tx1, tx2 = (-b[:, 3] - lox) / dx, (b[:, 3] - lox) / dx
            ty1, ty2 = (-b[:, 4] - loy) / dy, (b[:, 4] - loy) / dy
            tz1, tz2 = (0.0 - oz) / dz, (b[:, 5] - oz) / dz
            tmin = np.maximum.reduce([np.minimum(tx1, tx2), np.minimum(ty1, ty2), np.minimum(tz1, tz2)])
            tmax = np.minimum.reduce([np.maximum(tx1, tx2), np.maximum(ty1, ty2), np.maximum(tz1, tz2)])
        hit = (tmax >= tmin) & (tmin > 0)
        tb = np.where(hit, tmin, np.inf).min(axis=1)
        # cylinders
        c = scene.cyls
        qx, qy = ox - c[:, 0], oy - c[:, 1]
        aa = dd[:, None, 0] ** 2 + dd[:, None, 1] ** 2
        bb = 2 * (dd[:, None, 0] * qx + dd[:, None, 1] * qy)
        cc = qx ** 2 + qy ** 2 - c[:, 2] ** 2
        disc = bb * bb - 4 * aa * cc
        with np.errstate(invalid="ignore", divide="ignore"):
            tcyl = (-bb - np.sqrt(disc)) / (2 * aa)
        zc = oz + tcyl * dd[:, None, 2]
        ok = (disc > 0) & (tcyl > 0) & (zc >= 0) & (zc <= c[:, 3])
        tcy = np.where(ok, tcyl, np.inf).min(axis=1)
        t[s:s + chunk] = np.minimum(tc, np.minimum(tb, tcy))
    t[t > MAX_RANGE] = np.inf
    return t


def _surface_hits(rng, scene, beams, sweeps):
    pts = []
    for s in range(sweeps):
        d = _ray_dirs(beams, AZ_STEP_DEG * s / sweeps)
        t = _cast(scene, d)
        ok = np.isfinite(t)
        tt = t[ok] + rng.normal(scale=0.02, size=int(ok.sum()))
        p = d[ok] * tt[:, None]
        p[:, 2] += SENSOR_Z
        pts.append(p)
    return np.concatenate(pts, axis=0)


def _snow(rng, count):
    """Snow flakes above the ground (samples below z = 0 are redrawn)."""
    out = np.empty((0, 3))
    while len(out) < count:
        m = 2 * (count - len(out)) + 16
        r = np.sqrt(rng.uniform(0.5 ** 2, 15.0 ** 2, m))
        az = rng.uniform(0, 2 * np.pi, m)
        sel = rng.uniform(np.sin(np.deg2rad(-25.0)), np.sin(np.deg2rad(15.0)), m)
        cel = np.sqrt(1 - sel ** 2)
        p = np.stack([r * cel * np.cos(az), r * cel * np.sin(az), SENSOR_Z + r * sel], axis=1)
        out = np.concatenate([out, p[p[:, 2] >= 0.0]])
    return out[:count]


def lidar_frame(seed: int, beams: int = 32, target=None, snow_frac=None,
                outlier_frac: float = 0.0, scene_seed=None):
    """One accumulated spinning-LiDAR frame.

    ``target`` (total points) defaults to U[60k, 130k]; ``snow_frac`` to
    U[0.05, 0.20].  ``outlier_frac`` adds uniform outliers on top (share of the
    target).  Returns ``(xyz float32 [N,3], labels uint8 [N])``.
    """
    rng = np.random.default_rng(seed)
    scene = _make_scene(np.random.default_rng(scene_seed) if scene_seed is not None else rng)
    if target is None:
        target = int(rng.integers(60_000, 130_001))
    if snow_frac is None:
        snow_frac = float(rng.uniform(0.05, 0.20))
    n_snow = int(round(snow_frac * target))
    n_out = int(round(outlier_frac * target))
    need = target - n_snow - n_out
    one = _surface_hits(rng, scene, beams, 1)
    sweeps = max(1, int(np.ceil(need / max(1, len(one)))))
    surf = one if sweeps == 1 else _surface_hits(rng, scene, beams, sweeps)
    if len(surf) > need:
        surf = surf[np.sort(rng.choice(len(surf), size=need, replace=False))]
    parts, labels = [surf], [np.zeros(len(surf))]
    if n_snow:
        parts.append(_snow(rng, n_snow))
        labels.append(np.full(n_snow, 2))
    if n_out:
        lo, hi = surf.min(axis=0), surf.max(axis=0)
        c, h = 0.5 * (lo + hi), 0.6 * (hi - lo)
        parts.append(rng.uniform(c - h, c + h, size=(n_out, 3)))
        labels.append(np.ones(n_out))
    xyz = np.concatenate(parts).astype(np.float32)
    lab = np.concatenate(labels).astype(np.uint8)
    perm = rng.permutation(len(xyz))
    return np.ascontiguousarray(xyz[perm]), np.ascontiguousarray(lab[perm])


def lidar_batch(n_frames: int = 64, base_seed: int = 1000, beams: int = 32):
    """The batching workload: ``n_frames`` frames of 60k-130k points with 5-20 % snow."""
    return [lidar_frame(base_seed + i, beams=beams) for i in range(n_frames)]


def _yaw(xyz, ang):
    c, s = np.cos(ang), np.sin(ang)
    out = xyz.copy()
    out[:, 0] = c * xyz[:, 0] - s * xyz[:, 1]
    out[:, 1] = s * xyz[:, 0] + c * xyz[:, 1]
    return out


@dataclasses.dataclass
class Request:
    t_arrival: float        # seconds since stream start
    kind: str               # "dense" (128 beams) or "sparse" (32 beams)
    seed: int


class serving_stream:
    """Poisson request stream mixing dense 128-beam and sparse 32-beam frames.

    ``requests`` lists arrival times (exponential gaps at ``rate_hz``) and the
    kind of each frame (Bernoulli(0.5)).  ``frame(req)`` returns the frame: a
    base scene from a small pool (``pool`` per kind, ray-cast once), rotated by
    a random yaw and given fresh range jitter and fresh noise points, with the
    kind's noise recipe (dense: 10 % uniform outliers; sparse: 15 % near-range
    snow).  ``dense_points`` / ``sparse_points`` set the frame sizes.
    """

    def __init__(self, seed: int = 7, n_frames: int = 2000, rate_hz: float = 20.0,
                 dense_points: int = 1_000_000, sparse_points: int = 100_000, pool: int = 2, bases=None):
        rng = np.random.default_rng(seed)
        gaps = rng.exponential(1.0 / rate_hz, n_frames)
        kinds = np.where(rng.uniform(size=n_frames) < 0.5, "dense", "sparse")
        self.requests = [Request(float(t), str(k), int(seed * 100_003 + i))
                         for i, (t, k) in enumerate(zip(np.cumsum(gaps), kinds))]
        self.seed = seed
        self.pool = pool
        self.sizes = {"dense": dense_points, "sparse": sparse_points}
        self._base = dict(bases or {})

    def bases(self) -> dict:
        """The ray-cast base scenes of the pool (built on first use); pass them to
        another ``serving_stream`` of the same seed (``bases=``) to skip the ray casting."""
        for kind in ("dense", "sparse"):
            for slot in range(self.pool):
                self._base_frame(kind, slot)
        return dict(self._base)

    def _base_frame(self, kind, slot):
        key = (kind, slot)
        if key not in self._base:
            s = self.seed * 1000 + slot + (500 if kind == "dense" else 0)
            if kind == "dense":
                surf, lab = lidar_frame(s, beams=128, target=self.sizes["dense"], snow_frac=0.0)
            else:
                surf, lab = lidar_frame(s, beams=32, target=self.sizes["sparse"], snow_frac=0.0)
            self._base[key] = surf
        return self._base[key]

    def frame(self, req: Request):
        rng = np.random.default_rng(req.seed)
        base = self._base_frame(req.kind, int(rng.integers(0, self.pool)))
        surf = _yaw(base.astype(np.float64), rng.uniform(0, 2 * np.pi))
        rr = np.linalg.norm(surf - np.array([0, 0, SENSOR_Z]), axis=1, keepdims=True)
        surf = surf + (surf - np.array([0, 0, SENSOR_Z])) / np.maximum(rr, 1e-9) * \
            rng.normal(scale=0.02, size=(len(surf), 1))
        n = len(surf)
        if req.kind == "dense":
            n_noise = int(round(0.10 / 0.90 * n))
            lo, hi = surf.min(axis=0), surf.max(axis=0)
            c, h = 0.5 * (lo + hi), 0.6 * (hi - lo)
            noise, nl = rng.uniform(c - h, c + h, size=(n_noise, 3)), 1
        else:
            n_noise = int(round(0.15 / 0.85 * n))
            noise, nl = _snow(rng, n_noise), 2
        xyz = np.concatenate([surf, noise]).astype(np.float32)
        lab = np.concatenate([np.zeros(n), np.full(n_noise, nl)]).astype(np.uint8)
        perm = rng.permutation(len(xyz))
        return np.ascontiguousarray(xyz[perm]), np.ascontiguousarray(lab[perm])
