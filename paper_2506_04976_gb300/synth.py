"""Seeded synthetic inputs shaped like the paper's simulation and brain workloads.

This module generates INPUTS only: phantoms, attenuation maps, crystal
sensitivities, michelogram plane lists, background sinograms and Poisson counts.
It holds none of the reconstruction method's arithmetic: expected counts come from
exact, continuous line integrals of ellipsoids (and, for TOF, of an untruncated
Gaussian timing kernel), not from the discretised Joseph operator, the truncated
TOF model, the KL term or the prior.  Both the CUDA path and the FP64 oracle consume
what it returns.

Randomness is a counter-based generator (splitmix64 of seed, stream and index), so
the same seed gives the same arrays on every machine and numpy version.

Workloads (paper Sec. 3.1 describes the simulated scanner and phantoms; the sizes
below are those of the five benchmark configurations):
  c1  2D 64x64 at 2 mm, 96 radial x 90 views, 1e5 counts, 10% uniform background.
  c2  3D 128x128x47 at 2x2x2.8 mm, 250 radial x 168 views x 109 planes, 1e7 counts.
  c3  c2 with 11 TOF bins (FWHM 390 ps), 1e6 counts.
  c4  32 instances 96..192 pixels, 1..35 slices (see ``batch_specs``).
  c5  215x215x71 at 1.3x1.3x2.0 mm, 357 radial x 224 views x 1293 planes x 13 TOF.
"""
from __future__ import annotations

import math

import numpy as np

C_MM_PER_NS = 299.792458
FWHM_TO_SIGMA = 1.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


# --------------------------------------------------------------------------- RNG
def _mix64(z):
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0,1) from splitmix64(seed, stream, index)."""
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = np.uint64((seed * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03) & 0xFFFFFFFFFFFFFFFF)
        z = _mix64(base + (idx + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller from two uniform streams."""
    u1 = uniform(seed, stream, n)
    u2 = uniform(seed, stream + 7919, n)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def poisson(lam: np.ndarray, seed: int, stream: int) -> np.ndarray:
    """Poisson counts: CDF inversion for lam < 40, rounded normal approximation above."""
    lam = np.asarray(lam, np.float64).ravel()
    out = np.zeros(lam.size, np.int64)
    u = uniform(seed, stream, lam.size)
    small = lam < 40.0
    ls = lam[small]
    us = u[small]
    k = np.zeros(ls.size, np.int64)
    p = np.exp(-ls)
    cdf = p.copy()
    active = us > cdf
    kk = 0
    while active.any():
        kk += 1
        p = np.where(active, p * ls / kk, p)
        cdf = np.where(active, cdf + p, cdf)
        k = np.where(active, kk, k)
        active = active & (us > cdf) & (kk < 200)
    out[small] = k
    if (~small).any():
        z = normal(seed, stream + 104729, lam.size)[~small]
        lb = lam[~small]
        out[~small] = np.maximum(0, np.rint(lb + np.sqrt(lb) * z)).astype(np.int64)
    return out


# ------------------------------------------------------------------ plane lists
def planes_2d():
    return np.zeros(1), np.zeros(1)


def planes_span3_segments(nrings: int, pitch: float, oblique: bool = True):
    """Michelogram planes: segment 0 (ring differences -1..1 merged, 2*nrings-1 planes
    at half-ring steps) plus, when the scanner has enough rings, the span-3 segments of
    mean ring difference +9 and -9 (differences 8..10 merged), planes at half-ring steps.
    With 24 rings this gives 47 + 2*31 = 109 planes."""
    zr = lambda pos: (pos - 0.5 * (nrings - 1)) * pitch
    z1, z2 = [], []
    for m in range(2 * nrings - 1):
        z = zr(0.5 * m)
        z1.append(z)
        z2.append(z)
    if oblique and nrings >= 10:
        for sign in (+1, -1):
            half = sign * 9 * pitch / 2.0
            pos = 4.0
            while pos <= (nrings - 1) - 4.0 + 1e-9:
                zc = zr(pos)
                z1.append(zc - half)
                z2.append(zc + half)
                pos += 0.5
    return np.array(z1), np.array(z2)


def planes_span1(nrings: int, pitch: float, keep: int | None = None):
    """Span-1 michelogram, planes ordered by |ring difference|, then segment sign
    (+ before -), then first ring.  ``keep`` truncates the list."""
    zr = lambda k: (k - 0.5 * (nrings - 1)) * pitch
    z1, z2 = [], []
    for d in range(nrings):
        if d == 0:
            for r in range(nrings):
                z1.append(zr(r)); z2.append(zr(r))
            continue
        for r in range(nrings - d):
            z1.append(zr(r)); z2.append(zr(r + d))
        for r in range(nrings - d):
            z1.append(zr(r + d)); z2.append(zr(r))
    z1, z2 = np.array(z1), np.array(z2)
    if keep is not None:
        z1, z2 = z1[:keep], z2[:keep]
    return z1, z2


def tof_sigma_mm(fwhm_ps: float = 390.0) -> float:
    """Spatial sigma along the LOR of a coincidence timing FWHM (Sec. 3.1: 390 ps)."""
    return C_MM_PER_NS * fwhm_ps * 1e-3 / 2.0 * FWHM_TO_SIGMA


# ------------------------------------------------------------- LOR endpoints
def lor_endpoints(geom, views=None):
    """Endpoints (E1, E2), each (V, P, R, 3), of the scanner's LORs (data generation)."""
    V, R = geom["nview"], geom["nrad"]
    views = np.arange(V) if views is None else np.asarray(views)
    phi = views * math.pi / V
    s = (np.arange(R) - 0.5 * (R - 1)) * geom["drad"]
    h = np.sqrt(geom["rdet"] ** 2 - s ** 2)
    c, sn = np.cos(phi)[:, None], np.sin(phi)[:, None]
    mx, my = s[None, :] * c, s[None, :] * sn
    ux, uy = -sn, c
    P = len(geom["z1"])
    e1 = np.empty((len(views), P, R, 3))
    e2 = np.empty((len(views), P, R, 3))
    e1[..., 0] = (mx - h * ux)[:, None, :]
    e1[..., 1] = (my - h * uy)[:, None, :]
    e2[..., 0] = (mx + h * ux)[:, None, :]
    e2[..., 1] = (my + h * uy)[:, None, :]
    e1[..., 2] = np.asarray(geom["z1"])[None, :, None]
    e2[..., 2] = np.asarray(geom["z2"])[None, :, None]
    return e1, e2


# ------------------------------------------------------------------ ellipsoids
# An ellipsoid is (cx, cy, cz, ax, ay, az, theta, value): centre (mm), semi-axes
# (mm), rotation about z (rad), additive value.
def voxelise(ellipsoids, shape, spacing):
    nz, ny, nx = shape
    dx, dy, dz = spacing
    x = (np.arange(nx) - 0.5 * (nx - 1)) * dx
    y = (np.arange(ny) - 0.5 * (ny - 1)) * dy
    z = (np.arange(nz) - 0.5 * (nz - 1)) * dz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    img = np.zeros(shape)
    for (cx, cy, cz, ax, ay, az, th, val) in ellipsoids:
        ct, st = math.cos(th), math.sin(th)
        xr = (X - cx) * ct + (Y - cy) * st
        yr = -(X - cx) * st + (Y - cy) * ct
        inside = (xr / ax) ** 2 + (yr / ay) ** 2 + ((Z - cz) / az) ** 2 <= 1.0
        img[inside] += val
    return img


def _chords(ellipsoid, e1, d):
    """Parameters (lam1, lam2) in [0,1] of the chord of the segment e1 + lam d."""
    cx, cy, cz, ax, ay, az, th, _ = ellipsoid
    ct, st = math.cos(th), math.sin(th)
    px, py, pz = e1[..., 0] - cx, e1[..., 1] - cy, e1[..., 2] - cz
    qx = (px * ct + py * st) / ax
    qy = (-px * st + py * ct) / ay
    qz = pz / az
    vx = (d[..., 0] * ct + d[..., 1] * st) / ax
    vy = (-d[..., 0] * st + d[..., 1] * ct) / ay
    vz = d[..., 2] / az
    A = vx * vx + vy * vy + vz * vz
    B = 2.0 * (qx * vx + qy * vy + qz * vz)
    Cc = qx * qx + qy * qy + qz * qz - 1.0
    disc = B * B - 4.0 * A * Cc
    ok = disc > 0
    sq = np.sqrt(np.where(ok, disc, 0.0))
    l1 = np.where(ok, (-B - sq) / (2.0 * A), 0.0)
    l2 = np.where(ok, (-B + sq) / (2.0 * A), 0.0)
    return np.clip(l1, 0.0, 1.0), np.clip(l2, 0.0, 1.0)


def _Phi(u):
    from scipy.special import ndtr
    return ndtr(u)


def _Psi(u):
    """Antiderivative of the standard normal CDF: u*Phi(u) + phi(u)."""
    return u * _Phi(u) + np.exp(-0.5 * u * u) / math.sqrt(2.0 * math.pi)


def line_integrals(ellipsoids, e1, e2, tof=None):
    """Exact line integrals of a sum of ellipsoids along segments e1->e2.

    tof=None: returns (...,) integrals.  tof=(T, sigma, width): returns (..., T), the
    integral of value times the probability that an untruncated Gaussian of std sigma
    around the emission point falls in bin b = [c_b - w/2, c_b + w/2],
    c_b = (b - (T-1)/2) w, positions measured from the segment midpoint toward e2."""
    d = e2 - e1
    L = np.sqrt((d * d).sum(-1))
    if tof is None:
        out = np.zeros(e1.shape[:-1])
    else:
        T, sig, w = tof
        out = np.zeros(e1.shape[:-1] + (T,))
        edges = (np.arange(T + 1) - 0.5 * T) * w
    for ell in ellipsoids:
        l1, l2 = _chords(ell, e1, d)
        seg = l2 > l1
        if not seg.any():
            continue
        val = ell[7]
        if tof is None:
            out += np.where(seg, val * (l2 - l1) * L, 0.0)
        else:
            idx = np.nonzero(seg)
            t1 = (l1[idx] - 0.5) * L[idx]
            t2 = (l2[idx] - 0.5) * L[idx]
            # int_{t1}^{t2} Phi((e - t)/sig) dt = sig * (Psi((e-t1)/sig) - Psi((e-t2)/sig))
            F = np.stack([sig * (_Psi((e - t1) / sig) - _Psi((e - t2) / sig)) for e in edges], -1)
            out[idx] += val * (F[:, 1:] - F[:, :-1])
    return out


# ------------------------------------------------------------------ phantoms
def ellipse_phantom_2d(seed: int):
    """2D ellipse phantom: background ellipse (value 1) with 4-6 ellipses of value
    0 (cold) to 4 (hot) inside; ellipses are long cylinders along z."""
    u = uniform(seed, 11, 64)
    th0 = (u[0] - 0.5) * math.radians(60)
    base = (0.0, 0.0, 0.0, 50.0, 40.0, 1e4, th0, 1.0)
    ells = [base]
    nles = 4 + int(u[1] * 3)
    j = 2
    placed = []
    tries = 0
    while len(placed) < nles and tries < 200:
        tries += 1
        a = 5.0 + 7.0 * u[j % 64]; b = 5.0 + 7.0 * u[(j + 1) % 64]
        r = 30.0 * math.sqrt(u[(j + 2) % 64]); ang = 2 * math.pi * u[(j + 3) % 64]
        cx, cy = r * math.cos(ang), r * math.sin(ang)
        act = 4.0 * u[(j + 4) % 64]
        th = math.pi * u[(j + 5) % 64]
        j += 6
        if j > 58:
            u = uniform(seed, 12 + tries, 64); j = 0
        # keep lesions inside the base ellipse and apart from each other
        ct, st = math.cos(th0), math.sin(th0)
        xr, yr = cx * ct + cy * st, -cx * st + cy * ct
        if ((abs(xr) + max(a, b)) / 50.0) ** 2 + ((abs(yr) + max(a, b)) / 40.0) ** 2 > 1.0:
            continue
        if any(math.hypot(cx - px, cy - py) < max(a, b) + pr + 2.0 for px, py, pr in placed):
            continue
        placed.append((cx, cy, max(a, b)))
        ells.append((cx, cy, 0.0, a, b, 1e4, th, act - 1.0))
    mu = [(0.0, 0.0, 0.0, 60.0, 60.0, 1e4, 0.0, 0.0096)]
    return ells, mu, 1.0


def brain_phantom_3d(seed: int, scale_xy: float = 1.0, scale_z: float = 1.0):
    """Brain-like phantom: grey cortex (4) around white matter (1), two deep grey
    nuclei, five hot spheres (6-8 x white, radius 4-8 mm); water-like tissue
    attenuation 0.0096/mm inside a 5 mm bone shell of 0.0143/mm."""
    sx, sz = scale_xy, scale_z
    grey = (0.0, 0.0, 0.0, 66 * sx, 81 * sx, 55 * sz, 0.0, 4.0)
    white = (0.0, 0.0, 0.0, 58 * sx, 72 * sx, 47 * sz, 0.0, -3.0)
    nuc = [(s * 22 * sx, 5 * sx, 0.0, 8 * sx, 12 * sx, 10 * sz, 0.0, 3.0) for s in (-1, 1)]
    ells = [grey, white] + nuc
    u = uniform(seed, 21, 256)
    spheres = []
    j = 0
    while len(spheres) < 5 and j + 5 < 256:
        rad = (4.0 + 4.0 * u[j]) * min(sx, 1.0)
        cx = (u[j + 1] - 0.5) * 2 * 45 * sx
        cy = (u[j + 2] - 0.5) * 2 * 58 * sx
        cz = (u[j + 3] - 0.5) * 2 * 32 * sz
        val = 6.0 + 2.0 * u[j + 4]
        j += 5
        inside = (abs(cx) + rad) ** 2 / (58 * sx) ** 2 + (abs(cy) + rad) ** 2 / (72 * sx) ** 2 \
            + (abs(cz) + rad) ** 2 / (47 * sz) ** 2 < 1.0
        clear_nuc = all(math.hypot(cx - n[0], cy - n[1]) > rad + 14 * sx for n in nuc)
        clear = all(math.dist((cx, cy, cz), s[:3]) > rad + s[3] + 2.0 for s in spheres)
        if inside and clear_nuc and clear:
            spheres.append((cx, cy, cz, rad))
            ells.append((cx, cy, cz, rad, rad, rad, 0.0, val - 1.0))
    mu = [(0.0, 0.0, 0.0, 73 * sx, 88 * sx, 62 * sz, 0.0, 0.0143),
          (0.0, 0.0, 0.0, 68 * sx, 83 * sx, 57 * sz, 0.0, 0.0096 - 0.0143)]
    return ells, mu, 1.0


# ------------------------------------------------------------------ problems
def crystal_sensitivity(geom, seed: int):
    """Per-LOR sensitivity eps_a * eps_b of the crystals nearest to the endpoints, with
    per-crystal efficiencies clip(N(1, 0.05), 0.8, 1.2), 2V crystals per ring."""
    V = geom["nview"]
    nc = 2 * V
    ring_z = np.asarray(geom.get("ring_z", [0.0]))
    eff = np.clip(1.0 + 0.05 * normal(seed, 31, nc * len(ring_z)), 0.8, 1.2).reshape(len(ring_z), nc)
    e1, e2 = lor_endpoints(geom)

    def crystal(e):
        ang = np.mod(np.arctan2(e[..., 1], e[..., 0]), 2 * math.pi)
        ci = np.mod(np.rint(ang / (2 * math.pi) * nc).astype(np.int64), nc)
        ri = np.abs(e[..., 2][..., None] - ring_z[None, None, None, :]).argmin(-1)
        return eff[ri, ci]

    return crystal(e1) * crystal(e2)


def _smooth(a, sigma):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(a, sigma, mode="nearest")


# Smaller 3D workloads for convergence studies (the c2 brain and scanner at half the
# resolution in every direction: 64x64x23 voxels of 4x4x5.7 mm, 125 radial bins x 84
# views, 21 subsets of 4 views), with the relative prior strength 4 ("c2s"), 1 or 16,
# and the TOF workload c3 (11 bins, 1e6 counts) at the same half resolution ("c3s"); the
# 2D workload with priors 50 and 500 times stronger than its own ("c1b5", "c1b50") and the
# half-resolution 3D one with beta = 50 ("c2sb50"), where the prior's curvature term of the
# harmonic preconditioner (eq. 8) reaches ~10% and ~100% of the sensitivity A^T 1.
STUDY_WORKLOADS = {"c2s": dict(nx=64, nz=23, nrad=125, nview=84, nsub=21),
                   "c2s1": dict(nx=64, nz=23, nrad=125, nview=84, nsub=21, beta=1 * 2e-4 * 1e7 / 3e7),
                   "c2s16": dict(nx=64, nz=23, nrad=125, nview=84, nsub=21, beta=16 * 2e-4 * 1e7 / 3e7),
                   "c3s": dict(base="c3", nx=64, nz=23, nrad=125, nview=84, nsub=21),
                   "c2sb50": dict(nx=64, nz=23, nrad=125, nview=84, nsub=21, beta=50.0),
                   "c1b5": dict(base="c1", beta=5.0),
                   "c1b50": dict(base="c1", beta=50.0)}


def _setup(name: str, seed: int, **over):
    """Geometry, phantom and reconstruction parameters of a workload (no data)."""
    if name in STUDY_WORKLOADS:
        w = dict(STUDY_WORKLOADS[name])
        return _setup(w.pop("base", "c2"), seed, **{**w, **over})
    if name == "c1":
        nx = over.get("nx", 64)
        geom = dict(nx=nx, ny=nx, nz=1, dx=2.0 * 64 / nx, dy=2.0 * 64 / nx, dz=2.0,
                    nrad=over.get("nrad", 96), nview=over.get("nview", 90),
                    drad=over.get("drad", 2.0 * 96 / over.get("nrad", 96)), rdet=300.0, ntof=1,
                    tof_sigma=1.0, tof_bin=1.0)
        geom["z1"], geom["z2"] = planes_2d()
        geom["ring_z"] = np.zeros(1)
        ells, mu_ells, bgval = ellipse_phantom_2d(seed)
        counts, frac, smooth = over.get("counts", 1e5), 0.1, False
        params = dict(nsub=over.get("nsub", 6), beta=over.get("beta", 0.1), gamma=2.0, eps=1e-3)
    elif name in ("c2", "c3"):
        nx = over.get("nx", 128)
        nz = over.get("nz", 47)
        nrings = (nz + 1) // 2
        dxy = 2.0 * 128 / nx
        pitch = 5.6 * 47.0 / nz if over.get("nz") else 5.6
        dz = pitch / 2.0
        tof = name == "c3"
        T = over.get("ntof", 11 if tof else 1)
        geom = dict(nx=nx, ny=nx, nz=nz, dx=dxy, dy=dxy, dz=dz,
                    nrad=over.get("nrad", 250), nview=over.get("nview", 168),
                    drad=over.get("drad", 2.0 * 250 / over.get("nrad", 250)), rdet=300.0, ntof=T,
                    tof_sigma=tof_sigma_mm(390.0),
                    tof_bin=float(math.ceil(math.hypot(nx * dxy, nx * dxy) / T)) if T > 1 else 1.0)
        geom["z1"], geom["z2"] = planes_span3_segments(nrings, pitch)
        geom["ring_z"] = (np.arange(nrings) - 0.5 * (nrings - 1)) * pitch
        ells, mu_ells, bgval = brain_phantom_3d(seed, nx * dxy / 256.0, nz * dz / (47 * 2.8))
        counts = over.get("counts", 1e6 if tof else 1e7)
        frac, smooth = 0.2, True
        params = dict(nsub=over.get("nsub", 21), beta=over.get("beta", None), gamma=2.0, eps=1e-3)
    elif name == "c5":
        nx = over.get("nx", 215)
        nz = over.get("nz", 71)
        nrings = (nz + 1) // 2
        dxy = 1.3 * 215 / nx
        pitch = 4.0 * 71.0 / nz if over.get("nz") else 4.0
        T = over.get("ntof", 13)
        geom = dict(nx=nx, ny=nx, nz=nz, dx=dxy, dy=dxy, dz=pitch / 2.0,
                    nrad=over.get("nrad", 357), nview=over.get("nview", 224),
                    drad=1.3 * 357 / over.get("nrad", 357), rdet=300.0, ntof=T,
                    tof_sigma=tof_sigma_mm(390.0),
                    tof_bin=float(math.ceil(math.hypot(nx * dxy, nx * dxy) / T)))
        keep = over.get("nplane", 1293 if nrings == 36 else None)
        geom["z1"], geom["z2"] = planes_span1(nrings, pitch, keep)
        geom["ring_z"] = (np.arange(nrings) - 0.5 * (nrings - 1)) * pitch
        ells, mu_ells, bgval = brain_phantom_3d(seed, nx * dxy / 256.0, nz * pitch / 2 / (47 * 2.8))
        counts, frac, smooth = over.get("counts", 3e8), 0.2, True
        params = dict(nsub=over.get("nsub", 25), beta=over.get("beta", None), gamma=2.0, eps=1e-3)
    else:
        raise ValueError(name)

    shape = (geom["nz"], geom["ny"], geom["nx"])
    spacing = (geom["dx"], geom["dy"], geom["dz"])
    x_phantom = voxelise(ells, shape, spacing)
    mu = voxelise(mu_ells, shape, spacing)
    from scipy.ndimage import binary_dilation
    mask = binary_dilation(x_phantom > 0, np.ones((3, 3, 3) if geom["nz"] > 1 else (1, 3, 3), bool))
    bgmask = (x_phantom == bgval)
    if params["beta"] is None:
        # beta scaled with the count level as in Sec. 3.1 (relative strength 4)
        params["beta"] = 4.0 * 2e-4 * counts / 3e7
    return dict(name=name, seed=seed, geom=geom, mu=mu, mask=mask.astype(np.uint8),
                bg=bgmask.astype(np.uint8), _ells=ells, _mu_ells=mu_ells, _x_phantom=x_phantom,
                _counts=counts, _frac=frac, _smooth=smooth, **params)


def make_problem(name: str = "c1", seed: int = 0, **over):
    """Returns a dict describing one reconstruction problem (geometry, phantom, data).

    Keys: geom (for both the CUDA plan and the oracle), x_true (nz,ny,nx), mu
    (nz,ny,nx), sens (V,P,R), y (V,P,R,T) integer counts, r (V,P,R,T), mask and bg
    (NRMSE masks), and the reconstruction parameters nsub, beta, gamma, eps.
    Overrides shrink a workload (nx, nz, nrad, nview, nrings, ...) for quick tests."""
    base = _setup(name, seed, **over)
    geom = base["geom"]
    ells, mu_ells = base["_ells"], base["_mu_ells"]
    x_phantom = base["_x_phantom"]
    counts, frac, smooth = base["_counts"], base["_frac"], base["_smooth"]

    sens = crystal_sensitivity(geom, seed) if geom["nz"] > 1 or name != "c1" else np.ones(
        (geom["nview"], len(geom["z1"]), geom["nrad"]))
    T = geom["ntof"] if geom["ntof"] > 1 else 1
    tof = (T, geom["tof_sigma"], geom["tof_bin"]) if T > 1 else None

    V, P, R = geom["nview"], len(geom["z1"]), geom["nrad"]
    lam = np.zeros((V, P, R, T))
    att = np.zeros((V, P, R))
    chunk = max(1, int(2e6 // (P * R)))
    for v0 in range(0, V, chunk):
        vs = np.arange(v0, min(V, v0 + chunk))
        e1, e2 = lor_endpoints(geom, vs)
        li = line_integrals(ells, e1, e2, tof)
        att[vs] = np.exp(-line_integrals(mu_ells, e1, e2))
        lam[vs] = li.reshape(len(vs), P, R, T)
    lam *= (sens * att)[..., None]
    if smooth:
        bg = _smooth(lam.sum(-1), (0, 2.0, 20.0))
        bg = np.repeat(bg[..., None] / T, T, -1)
    else:
        bg = np.ones_like(lam)
    s = (1.0 - frac) * counts / lam.sum()
    r = frac * counts * bg / bg.sum()
    lam_s = s * lam
    y = poisson(lam_s + r, seed, 41).reshape(lam.shape)
    ydt = np.uint16 if y.max() < 65536 else np.uint32
    out = {k: v for k, v in base.items() if not k.startswith("_")}
    out.update(x_true=s * x_phantom, sens=sens, y=y.astype(ydt), r=r.astype(np.float32))
    return out


def batch_specs(seed: int = 0, count: int = 32):
    """Per-instance sizes of the batched workload: Nx = Ny uniform in [96, 192] (multiple
    of 8), Nz odd in [1, 35], R = round(1.95 Nx), n uniform in [8, 28],
    V = n round(1.31 Nx / n), beta log-uniform in [0.01, 1], counts log-uniform in
    [1e5, 1e8].  Each entry is a keyword set for make_problem."""
    u = uniform(seed, 71, 8 * count).reshape(count, 8)
    out = []
    for i in range(count):
        nx = 96 + 8 * int(u[i, 0] * 13)
        nz = 1 + 2 * int(u[i, 1] * 18)
        n = 8 + int(u[i, 2] * 21)
        nview = n * max(1, int(round(1.31 * nx / n)))
        beta = float(10 ** (-2 + 2 * u[i, 3]))
        counts = float(10 ** (5 + 3 * u[i, 4]))
        name = "c1" if nz == 1 else "c2"
        spec = dict(name=name, nx=nx, nrad=int(round(1.95 * nx)), nview=nview, nsub=n, beta=beta,
                    counts=counts)
        if nz > 1:
            spec["nz"] = nz
        out.append(spec)
    return out


def random_sinogram_like(geom, seed: int, lo=0.5, hi=1.5):
    """Uniform random positive sinogram (V,P,R,T), for adjointness checks."""
    T = geom["ntof"] if geom["ntof"] > 1 else 1
    shape = (geom["nview"], len(geom["z1"]), geom["nrad"], T)
    return lo + (hi - lo) * uniform(seed, 51, int(np.prod(shape))).reshape(shape)


def random_image_like(geom, seed: int, lo=0.0, hi=1.0):
    shape = (geom["nz"], geom["ny"], geom["nx"])
    return lo + (hi - lo) * uniform(seed, 61, int(np.prod(shape))).reshape(shape)


# ------------------------------------------------------------- device generator
def make_problem_device(name: str = "c5", seed: int = 0, device="cuda", views_per_chunk: int = 8, **over):
    """As make_problem, but builds the expected counts, background and Poisson counts
    with torch on `device` (for workloads too large for the host generator, e.g. c5:
    1.34 G TOF bins).  Same phantom, scanner and physics (exact ellipsoid chords, the
    closed-form untruncated-Gaussian TOF integral, crystal efficiencies, smooth
    background); counts come from torch's seeded Poisson sampler, so they differ from
    the host generator's draws.  Returns torch tensors for y (int16 holding uint16 or
    int32), r (float32), sens (float32) and numpy arrays for the image-domain fields."""
    import torch
    base = _setup(name, seed, **over)
    geom = base["geom"]
    V, P, R = geom["nview"], len(geom["z1"]), geom["nrad"]
    T = geom["ntof"] if geom["ntof"] > 1 else 1
    dev = torch.device(device)
    f64 = torch.float64
    ells, mu_ells = base["_ells"], base["_mu_ells"]
    z1 = torch.tensor(np.asarray(geom["z1"]), dtype=f64, device=dev)
    z2 = torch.tensor(np.asarray(geom["z2"]), dtype=f64, device=dev)
    s_r = (torch.arange(R, dtype=f64, device=dev) - 0.5 * (R - 1)) * geom["drad"]
    h = torch.sqrt(geom["rdet"] ** 2 - s_r ** 2)
    ring_z = torch.tensor(np.asarray(geom["ring_z"]), dtype=f64, device=dev)
    nc = 2 * V
    eff = np.clip(1.0 + 0.05 * normal(seed, 31, nc * len(geom["ring_z"])), 0.8, 1.2).reshape(-1, nc)
    eff = torch.tensor(eff, dtype=f64, device=dev)
    lam = torch.empty((V, P, R, T), dtype=torch.float32, device=dev)
    att = torch.empty((V, P, R), dtype=torch.float32, device=dev)
    sens = torch.empty((V, P, R), dtype=torch.float32, device=dev)
    if T > 1:
        edges = (torch.arange(T + 1, dtype=f64, device=dev) - 0.5 * T) * geom["tof_bin"]
        sig = geom["tof_sigma"]
    inv_sqrt2pi = 1.0 / math.sqrt(2.0 * math.pi)

    def Psi(u):
        return u * 0.5 * torch.erfc(-u / math.sqrt(2.0)) + torch.exp(-0.5 * u * u) * inv_sqrt2pi

    for v0 in range(0, V, views_per_chunk):
        vs = torch.arange(v0, min(V, v0 + views_per_chunk), dtype=f64, device=dev)
        phi = vs * math.pi / V
        c, sn = torch.cos(phi)[:, None, None], torch.sin(phi)[:, None, None]
        mx, my = s_r[None, None, :] * c, s_r[None, None, :] * sn
        ux, uy = -sn, c
        hh = h[None, None, :]
        e1 = torch.stack([(mx - hh * ux).expand(-1, P, -1), (my - hh * uy).expand(-1, P, -1),
                          z1[None, :, None].expand(len(vs), -1, R)], -1)
        e2 = torch.stack([(mx + hh * ux).expand(-1, P, -1), (my + hh * uy).expand(-1, P, -1),
                          z2[None, :, None].expand(len(vs), -1, R)], -1)
        d = e2 - e1
        L = torch.sqrt((d * d).sum(-1))

        def chords(ell):
            cx, cy, cz, ax, ay, az, th, _ = ell
            ct, st = math.cos(th), math.sin(th)
            px, py, pz = e1[..., 0] - cx, e1[..., 1] - cy, e1[..., 2] - cz
            qx = (px * ct + py * st) / ax
            qy = (-px * st + py * ct) / ay
            qz = pz / az
            vx = (d[..., 0] * ct + d[..., 1] * st) / ax
            vy = (-d[..., 0] * st + d[..., 1] * ct) / ay
            vz = d[..., 2] / az
            A = vx * vx + vy * vy + vz * vz
            B = 2.0 * (qx * vx + qy * vy + qz * vz)
            Cc = qx * qx + qy * qy + qz * qz - 1.0
            disc = B * B - 4.0 * A * Cc
            ok = disc > 0
            sq = torch.sqrt(torch.clamp(disc, min=0.0))
            l1 = torch.where(ok, (-B - sq) / (2.0 * A), torch.zeros_like(A)).clamp(0.0, 1.0)
            l2 = torch.where(ok, (-B + sq) / (2.0 * A), torch.zeros_like(A)).clamp(0.0, 1.0)
            return l1, l2

        mu_int = torch.zeros_like(L)
        for ell in mu_ells:
            l1, l2 = chords(ell)
            mu_int += ell[7] * (l2 - l1).clamp(min=0.0) * L
        acc = torch.zeros(L.shape + (T,), dtype=f64, device=dev)
        for ell in ells:
            l1, l2 = chords(ell)
            seg = l2 > l1
            if T == 1:
                acc[..., 0] += torch.where(seg, ell[7] * (l2 - l1) * L, torch.zeros_like(L))
            else:
                t1 = ((l1 - 0.5) * L)[..., None]
                t2 = ((l2 - 0.5) * L)[..., None]
                F = sig * (Psi((edges - t1) / sig) - Psi((edges - t2) / sig))
                acc += torch.where(seg[..., None], ell[7] * (F[..., 1:] - F[..., :-1]), torch.zeros_like(acc))

        def crystal(ex, ey, ez):
            ang = torch.remainder(torch.atan2(ey, ex), 2 * math.pi)
            ci = torch.remainder(torch.round(ang / (2 * math.pi) * nc).long(), nc)
            ri = (ez[..., None] - ring_z).abs().argmin(-1)
            return eff[ri, ci]

        sl = slice(v0, v0 + len(vs))
        se = crystal(e1[..., 0], e1[..., 1], e1[..., 2]) * crystal(e2[..., 0], e2[..., 1], e2[..., 2])
        a = torch.exp(-mu_int)
        sens[sl] = se.float()
        att[sl] = a.float()
        lam[sl] = (acc * (se * a)[..., None]).float()
    counts = base["_counts"]
    frac = base["_frac"]
    lam_sum = float(lam.double().sum())
    s_scale = (1.0 - frac) * counts / lam_sum
    lam *= s_scale
    # smooth background: Gaussian-smoothed noise-free data (planes sigma 2, radial sigma 20)
    bg = lam.sum(-1)
    for dim, sg in ((1, 2.0), (2, 20.0)):
        rad = int(4 * sg)
        k = torch.exp(-0.5 * (torch.arange(-rad, rad + 1, device=dev, dtype=torch.float32) / sg) ** 2)
        k = (k / k.sum()).view(1, 1, -1)
        x = bg.movedim(dim, -1)
        shp = x.shape
        xp = torch.nn.functional.pad(x.reshape(-1, 1, shp[-1]), (rad, rad), mode="replicate")
        x = torch.nn.functional.conv1d(xp, k).reshape(shp)
        bg = x.movedim(-1, dim)
    r = (frac * counts / float(bg.double().sum())) * (bg[..., None] / T)
    r = r.expand(-1, -1, -1, T).contiguous()
    g = torch.Generator(device=dev).manual_seed(seed)
    y = torch.poisson(lam + r, generator=g)
    del lam
    ymax = float(y.max())
    y = y.to(torch.int32)
    if ymax < 65536:  # uint16 counts carried in an int16 tensor (same bit pattern)
        y = (y - 65536 * (y >= 32768).to(torch.int32)).to(torch.int16)
    out = {k: v for k, v in base.items() if not k.startswith("_")}
    out.update(y=y, r=r, sens=sens, x_true=s_scale * base["_x_phantom"], counts=counts)
    return out
