"""Seeded synthetic inputs for the Barnes-Hut treecode Monte Carlo.

This module only draws charges and positions; it holds none of the method's
arithmetic (no images, no energies, no tree).  It is the one module that both
the CUDA path and the CPU oracle's tests consume.

Workloads (all lengths in the same unit as the Bjerrum length l_B):

* ``plain``   -- N point charges, half +1 and half -1, uniform in the cube
  [-10, 10)^3; root cube [-16, 16)^3; theta = 0.5, p = 4, leaf capacity 8.
* ``colloid`` -- a fixed macroion of charge Z at the origin (radius R), N
  monovalent ions: |Z| counterions plus (N - |Z|)/2 salt pairs, radii drawn from
  the density proportional to exp(-(r - R)/2) + 0.05 on [R + 0.5, r_max],
  directions uniform; ions confined to R + 0.5 <= |r| <= r_max; each ion carries
  a point image (position R^2 r/|r|^2, charge -0.3 q R/|r|).  This mirrors the
  electric double layer around a spherical macroion of Sec. 4 of the paper
  (which uses counterions only, a hard-core diameter and l_B = 7.14).  The
  macroion is fixed at the centre and, by default (``fixed_direct``), held
  outside the tree: the tree holds the 2N ions and images, and the macroion's
  interactions are exact.
* ``batch``   -- replicas of ``colloid`` with N drawn uniformly from
  [2000, 50000] (N - |Z| even).
* ``uniform`` -- N charges of alternating sign uniform in [-50, 50)^3.
"""
from __future__ import annotations

import math

import numpy as np


def base_params(**kw) -> dict:
    p = dict(lB=1.0, beta=1.0, theta=0.5, p=4, N0=0, C=8, Dmax=20,
             root_lo=(-16.0, -16.0, -16.0), root_side=32.0, shell=None, image=None)
    p.update(kw)
    return p


def _unit_vectors(rng, n):
    cost = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sint = np.sqrt(np.maximum(0.0, 1.0 - cost * cost))
    return np.stack([sint * np.cos(phi), sint * np.sin(phi), cost], axis=1)


def _radii(rng, n, rmin, rmax, R, decay=2.0, floor=0.05):
    """Inverse-CDF draws from the mixture exp(-(r-R)/decay) + floor on [rmin, rmax]."""
    w_exp = decay * (math.exp(-(rmin - R) / decay) - math.exp(-(rmax - R) / decay))
    w_uni = floor * (rmax - rmin)
    pick_exp = rng.uniform(0.0, 1.0, n) < w_exp / (w_exp + w_uni)
    u = rng.uniform(0.0, 1.0, n)
    ea = math.exp(-(rmin - R) / decay)
    eb = math.exp(-(rmax - R) / decay)
    r_exp = R - decay * np.log(ea - u * (ea - eb))
    r_uni = rmin + u * (rmax - rmin)
    r = np.where(pick_exp, r_exp, r_uni)
    return np.clip(r, rmin, rmax)


def plain(n: int = 2000, seed: int = 1, theta: float = 0.5, p: int = 4, C: int = 8) -> dict:
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-10.0, 10.0, (n, 3))
    q = np.where(np.arange(n) < n // 2, 1.0, -1.0)
    return dict(name="plain-N%d" % n, params=base_params(theta=theta, p=p, C=C), q=q, xyz=xyz,
                n_mobile=n, n_fixed=0, step=1.0, seed=seed)


def root_for(rmax: float) -> tuple:
    side = 2.0 ** math.ceil(math.log2(2.0 * rmax * 1.2))
    return (-side / 2,) * 3, side


def colloid(n: int = 10000, seed: int = 2, R: float = 10.0, Z: float = -60.0,
            rmax: float = 50.0, theta: float = 0.5, p: int = 4, C: int = 8,
            Dmax: int = 20, fixed_direct: bool = True) -> dict:
    rng = np.random.default_rng(seed)
    nz = int(round(abs(Z)))
    if n < nz or (n - nz) % 2:
        raise ValueError("N - |Z| must be a non-negative even number")
    rmin = R + 0.5
    r = _radii(rng, n, rmin, rmax, R)
    xyz = r[:, None] * _unit_vectors(rng, n)
    sign = -1.0 if Z < 0 else 1.0
    npos_salt = (n - nz) // 2
    q = np.empty(n)
    q[:nz] = -sign  # counterions
    q[nz:nz + npos_salt] = 1.0
    q[nz + npos_salt:] = -1.0
    rng.shuffle(q)
    lo, side = root_for(rmax)
    params = base_params(theta=theta, p=p, C=C, Dmax=Dmax, root_lo=lo, root_side=side,
                         shell=(rmin, rmax), image=(R, -0.3), fixed_direct=fixed_direct)
    q_all = np.concatenate([q, [Z]])
    xyz_all = np.concatenate([xyz, np.zeros((1, 3))], axis=0)
    return dict(name="colloid-N%d" % n, params=params, q=q_all, xyz=xyz_all, n_mobile=n,
                n_fixed=1, step=1.0, seed=seed)


def batch_sizes(n_rep: int = 256, seed: int = 3, lo: int = 2000, hi: int = 50000,
                nz: int = 60) -> list:
    rng = np.random.default_rng(seed)
    ns = rng.integers(lo, hi + 1, n_rep)
    ns = ns - ((ns - nz) % 2)
    return [int(v) for v in ns]


def batch(n_rep: int = 256, seed: int = 3, theta: float = 0.5, p: int = 4, C: int = 8,
          sizes=None, fixed_direct: bool = True) -> list:
    sizes = sizes if sizes is not None else batch_sizes(n_rep, seed)
    return [colloid(n=sizes[r], seed=1000 + r, theta=theta, p=p, C=C, fixed_direct=fixed_direct)
            for r in range(len(sizes))]


def uniform(n: int = 100000, seed: int = 4, theta: float = 0.5, p: int = 4, C: int = 8) -> dict:
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-50.0, 50.0, (n, 3))
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    params = base_params(theta=theta, p=p, C=C, root_lo=(-64.0,) * 3, root_side=128.0)
    return dict(name="uniform-N%d" % n, params=params, q=q, xyz=xyz, n_mobile=n, n_fixed=0,
                step=1.0, seed=seed)


def large(n: int = 1000000, seed: int = 5, theta: float = 0.5, p: int = 6, fixed_direct: bool = True) -> dict:
    return colloid(n=n, seed=seed, R=40.0, Z=-2000.0, rmax=400.0, theta=theta, p=p, fixed_direct=fixed_direct)


def edl(n: int = 800, seed: int = 6, theta: float = 0.5, p: int = 2, C: int = 8,
        fixed_direct: bool = True) -> dict:
    """Snapshot shaped like the electric double layer of Sec. 4: n counterions of
    valence 2 around a fixed macroion of radius 30 and valence -2n, cell radius
    80, l_B = 7.14, radii drawn from exp(-(r - 30)/2) + 0.05 on [32, 78].  The
    ions' hard cores are not enforced (a snapshot for accuracy checks only)."""
    rng = np.random.default_rng(seed)
    a, rcell, tau = 30.0, 80.0, 4.0
    r = _radii(rng, n, a + tau / 2, rcell - tau / 2, a)
    xyz = r[:, None] * _unit_vectors(rng, n)
    lo, side = root_for(rcell)
    params = base_params(lB=7.14, theta=theta, p=p, C=C, root_lo=lo, root_side=side,
                         shell=(a + tau / 2, rcell - tau / 2), fixed_direct=fixed_direct)
    q = np.concatenate([np.full(n, 2.0), [-2.0 * n]])
    xyz = np.concatenate([xyz, np.zeros((1, 3))], axis=0)
    return dict(name="edl-N%d" % n, params=params, q=q, xyz=xyz, n_mobile=n, n_fixed=1,
                step=1.0, seed=seed)


def edl_hard(n: int = 800, seed: int = 8, theta: float = 0.5, p: int = 2, C: int = 8,
             Lmax: int = 0, fixed_direct: bool = True) -> dict:
    """The electric double layer of Sec. 4 with its hard cores (Eq. 2.1): n
    counterions of valence 2 and diameter 4 around a fixed macroion of radius
    30 and valence -2n in a cell of radius 80, l_B = 7.14.  Ion centres lie in
    [32, 78] (contact with the macroion and the cell wall), placed one by one
    uniformly in that shell, each redrawn until it is farther than 4 from all
    ions placed before (random sequential addition).  Lmax > 0 selects the
    fixed-level tree of Sec. 3.2 with leaves at depth Lmax (root cube of side
    256: Lmax = 6 gives leaves of side tau, which hold at most 4 ions)."""
    rng = np.random.default_rng(seed)
    a, rcell, tau = 30.0, 80.0, 4.0
    rmin, rmax = a + tau / 2, rcell - tau / 2
    xyz = np.zeros((n, 3))
    cells = {}  # cell list of side tau: a conflict can only lie in the 27 cells around
    for k in range(n):
        while True:
            r = (rng.uniform(rmin ** 3, rmax ** 3)) ** (1.0 / 3.0)
            x = r * _unit_vectors(rng, 1)[0]
            c = tuple(np.floor(x / tau).astype(int))
            near = [m for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)
                    for m in cells.get((c[0] + dx, c[1] + dy, c[2] + dz), ())]
            if not near or np.min(np.sum((xyz[near] - x) ** 2, axis=1)) > tau * tau * (1.0 + 1e-12):
                break
        xyz[k] = x
        cells.setdefault(c, []).append(k)
    lo, side = root_for(rcell)
    params = base_params(lB=7.14, theta=theta, p=p, C=C, root_lo=lo, root_side=side,
                         shell=(rmin, rmax), hard_core=tau, fixed_direct=fixed_direct)
    if Lmax > 0:
        params.update(Dmax=Lmax, fixed_depth=True)
    q = np.concatenate([np.full(n, 2.0), [-2.0 * n]])
    xyz = np.concatenate([xyz, np.zeros((1, 3))], axis=0)
    return dict(name="edl-hard-N%d%s" % (n, "-L%d" % Lmax if Lmax > 0 else ""), params=params, q=q, xyz=xyz, n_mobile=n, n_fixed=1,
                step=2.0, seed=seed)


def colloid_scaled(n: int = 100000, seed: int = 7, theta: float = 0.5, p: int = 4,
                   fixed_direct: bool = True) -> dict:
    """The colloid radial law scaled to n ions: lengths R and r_max times
    s = (n / 1e4)^(1/3), macroion charge Z times s^2 (nearest value with n - |Z|
    even), decay length 2 kept."""
    s = (n / 1e4) ** (1.0 / 3.0)
    nz = int(round(60 * s * s))
    if (n - nz) % 2:
        nz += 1
    return colloid(n=n, seed=seed, R=10.0 * s, Z=-float(nz), rmax=50.0 * s, theta=theta, p=p,
                   fixed_direct=fixed_direct)
