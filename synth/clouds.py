"""Object-scale synthetic clouds: sphere + torus, and a union of superquadrics.

Recipes (all randomness from ``numpy.random.default_rng(seed)``, PCG64):

* ``object_cloud`` (sphere + attached torus, 36,750 points at the defaults):
  unit sphere at the origin plus a torus with axis z, major radius R=0.6, minor
  radius r=0.15, centred at (0, 0, 0.8) so that its centre circle lies on the
  sphere.  35,000 surface points are split between the two in proportion to
  their areas (4*pi vs 4*pi^2*R*r); torus samples are area-weighted by
  (R + r cos theta).  Gaussian jitter sigma=0.005 per axis, then 5 % (of the
  surface count) uniform outliers in the clean bounding box scaled 1.2x about
  its centre.

* ``superquadric_scan`` (560,000 points at the defaults): 8 superquadrics with
  largest diameter U[0.1, 1.0], axis ratios U[0.5, 1], shape exponents
  U[0.3, 1.5], uniform random rotation and centre U[-1, 1]^3; 500,000
  area-weighted surface points, Gaussian jitter of 0.5 % of the clean bounding
  box diagonal, 10 % uniform outliers in the 1.2x box and 2 % clustered noise in
  20 Gaussian blobs (sigma=0.01, centres uniform in the clean box).
"""

from __future__ import annotations

import numpy as np


def _finish(rng, parts, labels):
    xyz = np.concatenate(parts, axis=0).astype(np.float32)
    lab = np.concatenate(labels, axis=0).astype(np.uint8)
    perm = rng.permutation(xyz.shape[0])
    return np.ascontiguousarray(xyz[perm]), np.ascontiguousarray(lab[perm])


def _uniform_box(rng, lo, hi, count, scale=1.2):
    c = 0.5 * (lo + hi)
    half = 0.5 * (hi - lo) * scale
    return rng.uniform(c - half, c + half, size=(count, 3))


def object_cloud(seed: int = 0, n_surface: int = 35_000, outlier_frac: float = 0.05,
                 jitter: float = 0.005):
    """Sphere plus attached torus with uniform outliers (labels 0/1)."""
    rng = np.random.default_rng(seed)
    R, r, zc = 0.6, 0.15, 0.8
    a_sph = 4.0 * np.pi
    a_tor = 4.0 * np.pi ** 2 * R * r
    n_sph = int(round(n_surface * a_sph / (a_sph + a_tor)))
    n_tor = n_surface - n_sph

    v = rng.normal(size=(n_sph, 3))
    sph = v / np.linalg.norm(v, axis=1, keepdims=True)

    # torus: accept theta with probability (R + r cos theta) / (R + r)
    th = np.empty(0)
    while th.size < n_tor:
        cand = rng.uniform(0.0, 2.0 * np.pi, size=2 * n_tor)
        keep = rng.uniform(0.0, 1.0, size=cand.size) < (R + r * np.cos(cand)) / (R + r)
        th = np.concatenate([th, cand[keep]])
    th = th[:n_tor]
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n_tor)
    tor = np.stack([(R + r * np.cos(th)) * np.cos(ph),
                    (R + r * np.cos(th)) * np.sin(ph),
                    zc + r * np.sin(th)], axis=1)

    surf = np.concatenate([sph, tor], axis=0)
    surf = surf + rng.normal(scale=jitter, size=surf.shape)
    lo, hi = surf.min(axis=0), surf.max(axis=0)
    n_out = int(round(outlier_frac * n_surface))
    out = _uniform_box(rng, lo, hi, n_out)
    return _finish(rng, [surf, out], [np.zeros(len(surf)), np.ones(n_out)])


def _signed_pow(v, e):
    return np.sign(v) * np.abs(v) ** e


def _superquadric_points(eta, omega, ax, e1, e2):
    ce, se = np.cos(eta), np.sin(eta)
    co, so = np.cos(omega), np.sin(omega)
    x = ax[0] * _signed_pow(ce, e1) * _signed_pow(co, e2)
    y = ax[1] * _signed_pow(ce, e1) * _signed_pow(so, e2)
    z = ax[2] * _signed_pow(se, e1)
    return np.stack([x, y, z], axis=-1)


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _superquadric_area_grid(ax, e1, e2, n_eta=256, n_om=512):
    """Area element on a parameter grid (finite differences), for resampling."""
    eta = np.linspace(-np.pi / 2, np.pi / 2, n_eta + 1)
    om = np.linspace(-np.pi, np.pi, n_om + 1)
    E, O = np.meshgrid(eta, om, indexing="ij")
    P = _superquadric_points(E, O, ax, e1, e2)
    du = P[1:, :-1] - P[:-1, :-1]
    dv = P[:-1, 1:] - P[:-1, :-1]
    area = np.linalg.norm(np.cross(du, dv), axis=-1)
    return eta, om, area


def superquadric_scan(seed: int = 1, n_surface: int = 500_000, n_shapes: int = 8,
                      outlier_frac: float = 0.10, blob_frac: float = 0.02,
                      n_blobs: int = 20, blob_sigma: float = 0.01,
                      jitter_frac: float = 0.005):
    """Union of random superquadrics with uniform outliers and Gaussian blobs (labels 0/1/2)."""
    rng = np.random.default_rng(seed)
    shapes = []
    for _ in range(n_shapes):
        size = rng.uniform(0.1, 1.0)
        ratios = rng.uniform(0.5, 1.0, size=3)
        ax = 0.5 * size * ratios / ratios.max()
        e1, e2 = rng.uniform(0.3, 1.5, size=2)
        rot = _random_rotation(rng)
        centre = rng.uniform(-1.0, 1.0, size=3)
        eta, om, area = _superquadric_area_grid(ax, e1, e2)
        shapes.append((ax, e1, e2, rot, centre, eta, om, area))
    tot = np.array([s[7].sum() for s in shapes])
    counts = np.floor(n_surface * tot / tot.sum()).astype(np.int64)
    counts[: n_surface - counts.sum()] += 1

    parts = []
    for (ax, e1, e2, rot, centre, eta, om, area), cnt in zip(shapes, counts):
        p = (area / area.sum()).ravel()
        cell = rng.choice(p.size, size=int(cnt), p=p)
        i, j = np.divmod(cell, area.shape[1])
        e = eta[i] + rng.uniform(0, 1, cnt) * (eta[i + 1] - eta[i])
        o = om[j] + rng.uniform(0, 1, cnt) * (om[j + 1] - om[j])
        pts = _superquadric_points(e, o, ax, e1, e2) @ rot.T + centre
        parts.append(pts)
    surf = np.concatenate(parts, axis=0)
    lo, hi = surf.min(axis=0), surf.max(axis=0)
    diag = float(np.linalg.norm(hi - lo))
    surf = surf + rng.normal(scale=jitter_frac * diag, size=surf.shape)

    n_out = int(round(outlier_frac * n_surface))
    out = _uniform_box(rng, lo, hi, n_out)
    n_blob_total = int(round(blob_frac * n_surface))
    per = n_blob_total // n_blobs
    centres = rng.uniform(lo, hi, size=(n_blobs, 3))
    blobs = [c + rng.normal(scale=blob_sigma, size=(per, 3)) for c in centres]
    blob = np.concatenate(blobs, axis=0)
    return _finish(rng, [surf, out, blob],
                   [np.zeros(len(surf)), np.ones(n_out), np.full(len(blob), 2)])


def noise_labels_to_binary(labels: np.ndarray) -> np.ndarray:
    """1 for any noise point (uniform outlier, blob or snow), 0 for surface."""
    return (np.asarray(labels) != 0).astype(np.uint8)
