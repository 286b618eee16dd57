"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against something the paper or the mathematics
fixes: published Philox vectors, closed forms (Legendre expansion of 1/|R+y|,
two-charge and uniform-ball energies), the truncation bound of Eq. (3.4), the
theta -> 0 limit (treecode = direct sum), a brute-force tree built from the
split rule, rebuild-from-scratch after local adjustments, and the Boltzmann
distribution of a one-ion system sampled by the Metropolis chain.
"""
import math

import numpy as np
import pytest

from conftest import golden
from paper_1305_1825_gb300 import workloads as W


# ---------------------------------------------------------------- Philox
def test_philox_known_answers(oracle_mod):
    rows = [l.split() for l in open(golden("philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle_mod.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


# ---------------------------------------------------------------- Taylor coefficients
def _terms(p):
    for k in range(p + 1):
        for n1 in range(k, -1, -1):
            for n2 in range(k - n1, -1, -1):
                yield (n1, n2, k - n1 - n2)


def test_term_index_is_graded_bijection(oracle_mod):
    for p in range(11):
        idx = [oracle_mod.term_index(*n) for n in _terms(p)]
        assert idx == list(range(oracle_mod.nterms(p)))
        assert oracle_mod.nterms(p) == (p + 1) * (p + 2) * (p + 3) // 6


def test_taylor_legendre_closed_form(oracle_mod):
    """sum_{||n||=k} T_n(R) y^n = (-1)^k |y|^k P_k(R^.y^) / |R|^(k+1) for every k <= 10,
    at 80 generic y, which pins every individual coefficient of order <= 10."""
    rng = np.random.default_rng(7)
    p = 10
    for trial in range(4):
        R = rng.normal(size=3) * rng.uniform(0.5, 4.0)
        T = oracle_mod.taylor(p, R)
        Rn = np.linalg.norm(R)
        for _ in range(80):
            y = rng.normal(size=3)
            yn = np.linalg.norm(y)
            cosg = float(R @ y) / (Rn * yn)
            for k in range(p + 1):
                s = 0.0
                for n in _terms(p):
                    if sum(n) == k:
                        s += T[oracle_mod.term_index(*n)] * y[0] ** n[0] * y[1] ** n[1] * y[2] ** n[2]
                Pk = np.polynomial.legendre.legval(cosg, [0] * k + [1])
                want = (-1) ** k * yn ** k * Pk / Rn ** (k + 1)
                scale = yn ** k / Rn ** (k + 1)
                assert abs(s - want) <= 1e-11 * scale, (k, s, want)


def test_taylor_low_orders_and_finite_differences(oracle_mod):
    R = np.array([0.7, -1.3, 0.45])
    x, y, z = R
    r = np.linalg.norm(R)
    T = oracle_mod.taylor(3, R)
    ti = oracle_mod.term_index
    assert T[ti(0, 0, 0)] == pytest.approx(1 / r, rel=1e-15)
    assert T[ti(1, 0, 0)] == pytest.approx(-x / r ** 3, rel=1e-14)
    assert T[ti(0, 0, 1)] == pytest.approx(-z / r ** 3, rel=1e-14)
    assert T[ti(2, 0, 0)] == pytest.approx((3 * x * x - r * r) / (2 * r ** 5), rel=1e-13)
    assert T[ti(1, 1, 0)] == pytest.approx(3 * x * y / r ** 5, rel=1e-13)
    assert T[ti(3, 0, 0)] == pytest.approx((3 * x * r * r - 5 * x ** 3) / (2 * r ** 7), rel=1e-13)
    # second derivatives by FP64 central differences of 1/r
    f = lambda v: 1.0 / np.linalg.norm(v)
    h = 1e-4
    e = np.eye(3)
    d2 = (f(R + h * e[1] + h * e[2]) - f(R + h * e[1] - h * e[2]) - f(R - h * e[1] + h * e[2])
          + f(R - h * e[1] - h * e[2])) / (4 * h * h)
    assert T[ti(0, 1, 1)] == pytest.approx(d2, rel=1e-6)


# ---------------------------------------------------------------- closed-form energies
def test_two_charge_energy_and_move(oracle_mod):
    params = W.base_params(lB=0.7)
    q = np.array([2.0, -1.5])
    xyz = np.array([[0.1, 0.2, -0.3], [1.1, -0.4, 0.5]])
    s = oracle_mod.System(params, q, xyz, n_mobile=2)
    r = np.linalg.norm(xyz[0] - xyz[1])
    assert s.energy_direct() == pytest.approx(0.7 * 2.0 * -1.5 / r, rel=1e-15)
    assert s.energy_tree() == pytest.approx(0.7 * 2.0 * -1.5 / r, rel=1e-15)
    b = np.array([-0.9, 0.6, 0.2])
    rb = np.linalg.norm(b - xyz[1])
    want = 0.7 * 2.0 * -1.5 * (1 / rb - 1 / r)
    assert s.delta_energy(0, b).dE == pytest.approx(want, rel=1e-14)
    assert s.delta_energy_direct(0, b)[1] == pytest.approx(want, rel=1e-14)


def _ball(rng, n, a):
    out = np.empty((0, 3))
    while len(out) < n:
        v = rng.uniform(-a, a, (2 * n, 3))
        out = np.concatenate([out, v[np.linalg.norm(v, axis=1) < a]])
    return out[:n]


def test_uniform_ball_energy_expectation(oracle_mod):
    """N iid uniform charges Q/N in a ball of radius a: E[E] = (N-1)/N (3/5) l_B Q^2 / a."""
    rng = np.random.default_rng(11)
    N, a, Q, lB = 60, 5.0, 6.0, 1.3
    q = np.full(N, Q / N)
    es = np.array([oracle_mod.direct_energy_raw(q, _ball(rng, N, a), lB) for _ in range(400)])
    want = (N - 1) / N * 0.6 * lB * Q * Q / a
    z = (es.mean() - want) / (es.std(ddof=1) / math.sqrt(len(es)))
    assert abs(z) < 4.5, (es.mean(), want, z)


# ---------------------------------------------------------------- treecode vs direct
def _systems(oracle_mod, theta, p):
    wl = W.plain(n=600, seed=5, theta=theta, p=p)
    yield wl, oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"])
    wl = W.colloid(n=400, seed=6, theta=theta, p=p)
    yield wl, oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])


def test_theta_zero_is_direct_sum(oracle_mod):
    for wl, s in _systems(oracle_mod, 0.0, 4):
        q, x = s.charges()
        for j in range(0, s.n_charges, 37):
            e = s.phi(x[j], excl=[j])
            assert e.accepted == 0
            assert abs(e.phi - s.phi_direct(x[j], excl=[j])) <= 1e-13 * e.abs_sum


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
@pytest.mark.parametrize("p", [0, 1, 2, 4, 6, 10])
def test_truncation_bound(oracle_mod, theta, p):
    """|phi_tree - phi_direct| <= sum over accepted clusters of sum_j |q_j| gamma^(p+1)/(R(1-gamma))."""
    rng = np.random.default_rng(100 * p + int(10 * theta))
    for wl, s in _systems(oracle_mod, theta, p):
        s.set_bound(True)
        q, x = s.charges()
        for t in range(25):
            j = int(rng.integers(0, s.n_mobile))
            excl = [j]
            if wl["params"]["image"]:
                excl.append(s.n_mobile + s.n_fixed + j)
            pt = x[j] + rng.uniform(-0.5, 0.5, 3) if t % 2 else x[j]
            e = s.phi(pt, excl=excl)
            d = s.phi_direct(pt, excl=excl)
            assert abs(e.phi - d) <= e.bound + 1e-12 * e.abs_sum, (t, e.phi, d, e.bound)
            assert e.accepted > 0



def test_cluster_holding_the_point_is_never_approximated(oracle_mod):
    """A cluster that contains the evaluation point has |r_A - x| <= rho_A, so it
    fails the MAC for every theta < 1 (Sec. 3.2).  At theta = 0.99 every accepted
    cluster must still have gamma = rho_A/|r_A - x| < 1: the truncation bound of
    Eq. (3.4) stays finite and holds at the charges' own positions."""
    for wl, s in _systems(oracle_mod, 0.99, 6):
        s.set_bound(True)
        q, x = s.charges()
        for j in range(0, s.n_mobile, 29):
            excl = [j]
            if wl["params"]["image"]:
                excl.append(s.n_mobile + s.n_fixed + j)
            e = s.phi(x[j], excl=excl)
            assert e.accepted > 0 and math.isfinite(e.bound) and e.bound >= 0.0
            assert abs(e.phi - s.phi_direct(x[j], excl=excl)) <= e.bound + 1e-12 * e.abs_sum

def test_high_order_converges_to_direct(oracle_mod):
    for wl, s in _systems(oracle_mod, 0.3, 10):
        q, x = s.charges()
        for j in range(0, s.n_mobile, 53):
            e = s.phi(x[j], excl=[j])
            assert abs(e.phi - s.phi_direct(x[j], excl=[j])) <= 1e-7 * e.abs_sum


def test_delta_energy_within_bound_of_direct(oracle_mod):
    for wl, s in _systems(oracle_mod, 0.5, 4):
        s.set_bound(True)
        rng = np.random.default_rng(3)
        q, x = s.charges()
        n = 0
        for t in range(40):
            i = int(rng.integers(0, s.n_mobile))
            b = x[i] + rng.uniform(-0.5, 0.5, 3)
            e = s.delta_energy(i, b)
            st, d = s.delta_energy_direct(i, b)
            assert st == e.status
            if st:
                continue
            n += 1
            assert abs(e.dE - d) <= e.bound + 1e-12 * e.abs_sum
        assert n > 20


# ---------------------------------------------------------------- tree structure
def brute_tree(xyz, lo, side, C, Dmax):
    """The canonical tree written out from its definition: a cube splits into its
    eight octants (upper half-open on ties) while it holds more than C points
    and is above depth Dmax."""
    out = {}

    def rec(idx, depth, key, c, h):
        leaf = not (len(idx) > C and depth < Dmax)
        out[(depth, key)] = (leaf, len(idx), tuple(sorted(int(v) for v in idx)) if leaf else None)
        if leaf:
            return
        pts = xyz[idx]
        o = (pts[:, 0] >= c[0]) * 1 + (pts[:, 1] >= c[1]) * 2 + (pts[:, 2] >= c[2]) * 4
        for k in range(8):
            cc = [c[a] + (h / 2 if (k >> a) & 1 else -h / 2) for a in range(3)]
            rec(idx[o == k], depth + 1, (key << 3) | k, cc, h / 2)

    h = side / 2
    rec(np.arange(len(xyz)), 0, 1, [lo[a] + h for a in range(3)], h)
    return out



def test_moved_set_exclusion_equals_zeroed_charge(oracle_mod):
    """The potential at a trial point with ion i excluded (moments corrected by
    q_i (r_i - r_A)^n on i's ancestors, i skipped in leaf sums) equals the
    treecode potential of the same tree with q_i set to zero: the tree's shape
    depends on positions only, and with N0 = 0 a cluster left empty by the
    exclusion contributes nothing either way.  Also with two excluded charges."""
    rng = np.random.default_rng(2)
    for wl in (W.plain(n=500, seed=17, C=3), W.colloid(n=400, seed=17, C=3)):
        wl["params"]["Dmax"] = 12
        q, x = wl["q"], wl["xyz"]
        nm, nf = wl["n_mobile"], wl["n_fixed"]
        s = oracle_mod.System(wl["params"], q, x, nm, nf)
        images = bool(wl["params"]["image"])
        for _ in range(12):
            i, j = (int(v) for v in rng.choice(nm, 2, replace=False))
            # an ion's image charge follows the ion's: zeroing q_i zeroes both
            sets = ([i], [i, j]) if not images else ([i], [j])
            for ions in sets:
                excl = ions + ([nm + nf + k for k in ions] if images else [])
                b = x[ions[0]] + rng.uniform(-0.6, 0.6, 3)
                q0 = q.copy()
                q0[ions] = 0.0
                z = oracle_mod.System(wl["params"], q0, x, nm, nf)
                assert z.export_tree() == s.export_tree()
                e, e0 = s.phi(b, excl=excl), z.phi(b)
                assert abs(e.phi - e0.phi) <= 1e-12 * e0.abs_sum, (excl, e.phi, e0.phi)

def test_tree_matches_brute_force_including_ties(oracle_mod):
    rng = np.random.default_rng(21)
    for C, Dmax in [(2, 6), (3, 8), (8, 20)]:
        # points on a coarse lattice put many coordinates exactly on cluster mid-planes
        xyz = np.round(rng.uniform(-8, 8, (300, 3)) * 2) / 2
        xyz = np.unique(xyz, axis=0)[:250]
        q = rng.choice([-1.0, 1.0], len(xyz))
        params = W.base_params(C=C, Dmax=Dmax)
        s = oracle_mod.System(params, q, xyz, n_mobile=len(xyz))
        assert s.check() == 0
        assert s.export_tree() == brute_tree(xyz, params["root_lo"], params["root_side"], C, Dmax)


def test_fixed_depth_tree_matches_brute_force(oracle_mod):
    """The Sec. 3.2 tree of fixed level L_max: every non-empty cluster above L_max
    is bisected, so every charge sits in a leaf at depth L_max (the brute-force
    tree with split threshold 0), and the leaf counts reproduce a histogram of
    the points over the 8^L_max cells."""
    rng = np.random.default_rng(23)
    for Lmax in (3, 4, 5):
        xyz = np.round(rng.uniform(-8, 8, (300, 3)) * 2) / 2
        xyz = np.unique(xyz, axis=0)[:250]
        params = W.base_params(C=32, Dmax=Lmax)
        params["fixed_depth"] = True
        s = oracle_mod.System(params, np.ones(len(xyz)), xyz, n_mobile=len(xyz))
        assert s.check() == 0
        tree = s.export_tree()
        assert tree == brute_tree(xyz, params["root_lo"], params["root_side"], 0, Lmax)
        lo, side = np.array(params["root_lo"]), params["root_side"]
        cell = np.floor((xyz - lo) / (side / 2 ** Lmax)).astype(int)
        _, hist = np.unique(cell, axis=0, return_counts=True)
        leaves = sorted(c for (d, k), (leaf, c, _) in tree.items() if leaf and c > 0)
        assert all(d == Lmax for (d, k), (leaf, c, _) in tree.items() if leaf and c > 0)
        assert leaves == sorted(hist.tolist())


def test_capacity_rule_at_dmax(oracle_mod):
    params = W.base_params(C=2, Dmax=3)
    xyz = np.array([[0.1, 0.1, 0.1], [0.2, 0.2, 0.2], [0.3, 0.1, 0.2], [5.0, 5.0, 5.0]])
    with pytest.raises(ValueError):
        oracle_mod.System(params, np.ones(4), xyz, n_mobile=4)
    s = oracle_mod.System(params, np.ones(3), xyz[1:], n_mobile=3)
    assert s.capacity_violation(2, np.array([0.15, 0.15, 0.15]))
    assert s.commit_move(2, np.array([0.15, 0.15, 0.15])) == oracle_mod.ECAPACITY
    assert not s.capacity_violation(2, np.array([-5.0, 0.15, 0.15]))


def _rebuilt(oracle_mod, s, wl):
    q, x = s.charges()
    n = s.n_mobile + s.n_fixed
    return oracle_mod.System(wl["params"], q[:n], x[:n], s.n_mobile, s.n_fixed)


@pytest.mark.parametrize("kind", ["plain", "colloid", "fixed-depth"])
def test_commit_equals_rebuild(oracle_mod, kind):
    """After every local adjustment (with splits and merges) the tree equals the
    tree built from scratch from the new particle set, and the running moments
    equal freshly summed moments up to accumulated rounding."""
    rng = np.random.default_rng(31)
    if kind == "plain":
        wl = W.plain(n=300, seed=8, C=2)
        wl["params"]["Dmax"] = 9
    elif kind == "colloid":
        wl = W.colloid(n=200, seed=9, C=3)
        wl["params"]["Dmax"] = 10
    else:  # the fixed-level tree of Sec. 3.2: merges and splits reach down to Dmax
        wl = W.plain(n=300, seed=8, C=4)
        wl["params"].update(Dmax=5, fixed_depth=True)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    done = 0
    for t in range(400):
        q, x = s.charges()
        i = int(rng.integers(0, s.n_mobile))
        b = x[i] + rng.uniform(-1.5, 1.5, 3)
        st = s.commit_move(i, b)
        if st != 0:
            assert st in (oracle_mod.EDOMAIN, oracle_mod.EOVERLAP, oracle_mod.ECAPACITY)
            continue
        done += 1
        assert s.check() == 0
        if t % 20 == 0:
            r = _rebuilt(oracle_mod, s, wl)
            tree = s.export_tree()
            assert tree == r.export_tree()
            for (d, k), (leaf, cnt, _) in list(tree.items())[::7]:
                _, M1 = s.node_moments(d, k)
                _, M2 = r.node_moments(d, k)
                assert np.allclose(M1, M2, rtol=1e-9, atol=1e-9 * (np.abs(M2).max() + 1))
    assert done > 200


def test_delta_energy_is_energy_difference(oracle_mod):
    wl = W.colloid(n=150, seed=12)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    rng = np.random.default_rng(5)
    for _ in range(10):
        q, x = s.charges()
        i = int(rng.integers(0, s.n_mobile))
        b = x[i] + rng.uniform(-0.5, 0.5, 3)
        st, d = s.delta_energy_direct(i, b)
        if st:
            continue
        e0 = s.energy_direct()
        assert s.commit_move(i, b) == 0
        e1 = s.energy_direct()
        assert (e1 - e0) == pytest.approx(d, abs=1e-10 * abs(e0) + 1e-12)


# ---------------------------------------------------------------- Metropolis chain
def test_metropolis_samples_boltzmann_one_ion(oracle_mod):
    """One ion (q=+1) around a fixed charge Z=-4 in the shell 1 <= r <= 4, with its
    image (R=0.8, alpha=-0.3): the radial density is r^2 exp(-beta E(r)),
    E(r) = l_B [q Z/r + alpha q^2 R/(r^2 - R^2)] + const."""
    lB, beta, Z, R, alpha = 1.0, 1.0, -4.0, 0.8, -0.3
    params = W.base_params(lB=lB, beta=beta, shell=(1.0, 4.0), image=(R, alpha))
    s = oracle_mod.System(params, np.array([1.0, Z]), np.array([[2.0, 0.3, -0.4], [0, 0, 0]]),
                          n_mobile=1, n_fixed=1)
    recs = s.mc_run(seed=77, n_moves=300000, step=1.6)
    r = np.empty(len(recs))
    cur = np.linalg.norm([2.0, 0.3, -0.4])
    for t, rec in enumerate(recs):
        if rec["outcome"] == 0:
            cur = np.linalg.norm(rec["r_new"])
        r[t] = cur
    grid = np.linspace(1.0, 4.0, 200001)
    E = lB * (Z / grid + alpha * R / (grid ** 2 - R ** 2))
    w = grid ** 2 * np.exp(-beta * E)
    for f in (lambda v: v, lambda v: 1 / v, lambda v: v * v):
        want = np.trapezoid(f(grid) * w, grid) / np.trapezoid(w, grid)
        batches = f(r).reshape(100, -1).mean(axis=1)
        z = (batches.mean() - want) / (batches.std(ddof=1) / 10)
        assert abs(z) < 5, (want, batches.mean(), z)


def test_mc_chain_keeps_tree_canonical(oracle_mod):
    wl = W.colloid(n=300, seed=13, C=4)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    recs = s.mc_run(seed=2, n_moves=2000)
    assert s.check() == 0
    assert s.export_tree() == _rebuilt(oracle_mod, s, wl).export_tree()
    out = np.bincount(recs["outcome"], minlength=5)
    assert out[0] > 500 and out[3] > 0


def test_mc_chain_keeps_fixed_level_tree(oracle_mod):
    """A Metropolis chain on the fixed-level tree of Sec. 3.2 (hard-core double
    layer, L_max = 6): after 3000 moves every charge still sits in a depth-L_max
    leaf, the tree equals the one rebuilt from the particle set, and no pair of
    ions is closer than the hard-core diameter (Eq. 2.1)."""
    wl = W.edl_hard(n=300, seed=19, Lmax=6)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    recs = s.mc_run(seed=5, n_moves=3000, step=wl["step"])
    assert s.check() == 0
    tree = s.export_tree()
    assert tree == _rebuilt(oracle_mod, s, wl).export_tree()
    assert all(d == 6 for (d, k), (leaf, c, _) in tree.items() if leaf and c > 0)
    x = s.charges()[1][:300]
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1) + np.eye(300) * 1e9
    assert d2.min() > 16.0
    out = np.bincount(recs["outcome"], minlength=5)
    assert out[0] > 300 and out[3] > 0


def _eq41(vt, vd, n):
    """Eq. (4.1): E = (sum_i |V_i - Vt_i|^2 / sum_i |V_i|^2)^(1/2) over the N
    counterions i = 1..N (the first n charges), V exact, Vt the treecode."""
    return math.sqrt(((vt[:n] - vd[:n]) ** 2).sum() / (vd[:n] ** 2).sum())


def test_relative_error_decreases_with_order(oracle_mod):
    """Eq. (4.1) over the N = 800 counterions of a snapshot shaped like the Sec. 4
    double layer (valence 2 around a fixed macroion, l_B = 7.14), the macroion's
    interactions exact: E falls with p and with theta, and at p = 2 it is below
    1 % for theta = 0.5 and below 0.1 % for theta = 0.3, the accuracy the paper
    reports for its own snapshots."""
    errs = {}
    for theta in (0.3, 0.5):
        for p in (0, 2, 4):
            wl = W.edl(n=800, seed=14, theta=theta, p=p)
            assert wl["params"]["fixed_direct"]
            s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
            vt, vd = s.potentials()
            errs[(theta, p)] = _eq41(vt, vd, 800)
    for theta in (0.3, 0.5):
        assert errs[(theta, 0)] > errs[(theta, 2)] > errs[(theta, 4)]
    for p in (0, 2, 4):
        assert errs[(0.3, p)] < errs[(0.5, p)]
    assert errs[(0.5, 2)] < 0.01 and errs[(0.3, 2)] < 0.001


def test_relative_error_roughly_independent_of_n(oracle_mod):
    """Sec. 4: the Eq. (4.1) error over the N counterions at p = 2 stays of the
    same size for N from 100 up (double-layer snapshots of 100 to 3200 ions):
    below 1 % / 0.1 % at theta = 0.5 / 0.3 for every N, within a factor of
    five across N."""
    for theta, cap in ((0.5, 0.01), (0.3, 0.001)):
        errs = []
        for n in (100, 400, 1600, 3200):
            wl = W.edl(n=n, seed=14, theta=theta, p=2)
            s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
            vt, vd = s.potentials()
            errs.append(_eq41(vt, vd, n))
        assert max(errs) < cap and max(errs) / min(errs) < 5.0, errs


def test_relative_error_on_equilibrated_hard_core_layer(oracle_mod):
    """Eq. (4.1) over the 800 counterions on a snapshot of an equilibrated chain
    of the Sec. 4 double layer with hard cores (Eq. 2.1), the macroion fixed at
    the centre with exact interactions: below 1 % at theta = 0.5 and 0.1 % at
    theta = 0.3 for p = 2, falling with p."""
    wl = W.edl_hard(n=800, seed=8)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    s.mc_run(3, 200000, step=wl["step"])
    snap = s.charges()[1][:801].copy()
    assert np.median(np.linalg.norm(snap[:800], axis=1)) < 40.0  # condensed at the surface
    errs = {}
    for theta in (0.3, 0.5):
        for p in (1, 2, 3):
            w = W.edl_hard(n=800, seed=8, theta=theta, p=p)
            t = oracle_mod.System(w["params"], w["q"], snap, w["n_mobile"], w["n_fixed"])
            vt, vd = t.potentials()
            errs[(theta, p)] = _eq41(vt, vd, 800)
    for theta in (0.3, 0.5):
        assert errs[(theta, 1)] > errs[(theta, 2)] > errs[(theta, 3)]
    assert errs[(0.5, 2)] < 0.01 and errs[(0.3, 2)] < 0.001


def test_macroion_in_the_tree_misses_the_papers_accuracy(oracle_mod):
    """Why the macroion's interactions are exact: with the -1600 macroion as an
    ordinary tree charge at the origin, the origin is a corner of every cluster
    below the root that holds it (ties go to the upper child), the macroion sits
    at the largest offset its cluster's expansion allows, and E over the
    counterions at p = 2, theta = 0.5 is ~13 %, far above the paper's < 1 %.
    Moving the root cube by side/16, so that the origin becomes the centre of
    the level-3 cluster holding only the macroion (its expansion then exact),
    brings it back under 1 %."""
    wl = W.edl(n=800, seed=14, theta=0.5, p=2, fixed_direct=False)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    vt, vd = s.potentials()
    assert _eq41(vt, vd, 800) > 0.05
    side = wl["params"]["root_side"]
    wl["params"]["root_lo"] = tuple(x - side / 16 for x in wl["params"]["root_lo"])
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    vt, vd = s.potentials()
    assert _eq41(vt, vd, 800) < 0.01


def test_fixed_direct_equals_tree_without_fixed_plus_exact_terms(oracle_mod):
    """fixed_direct: the potential at any point is the treecode over the tree of
    the other charges (the same tree as a system with the fixed charges removed)
    plus the exact q_f / |r_f - x| of every fixed charge; the potential at a
    fixed charge is the exact sum; the tree holds no fixed charge."""
    wl = W.colloid(n=400, seed=5, p=3)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    assert s.check() == 0
    members = sorted(m for (leaf, cnt, mem) in s.export_tree().values() if leaf for m in mem)
    n, nf = wl["n_mobile"], wl["n_fixed"]
    assert members == list(range(n)) + list(range(n + nf, n + nf + n))
    # the same tree without the macroion: remove it and renumber the images
    w0 = W.colloid(n=400, seed=5, p=3, fixed_direct=False)
    t = oracle_mod.System(w0["params"], w0["q"][:n], w0["xyz"][:n], n, 0)
    rng = np.random.default_rng(3)
    qf, rf = wl["q"][n], wl["xyz"][n]
    for _ in range(20):
        x = rng.uniform(-40.0, 40.0, 3)
        want = t.phi(x).phi + qf / np.linalg.norm(rf - x)
        assert s.phi(x).phi == pytest.approx(want, rel=1e-13, abs=1e-13)
    vt, vd = s.potentials()
    assert vt[n] == vd[n]


def test_fixed_direct_theta_zero_equals_direct(oracle_mod):
    """theta = 0 with fixed_direct: every tree pair direct, every fixed pair exact,
    so the treecode energy, potentials and the move's dE equal the direct sums."""
    wl = W.colloid(n=300, seed=6, theta=0.0, p=2)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    assert s.energy_tree() == pytest.approx(s.energy_direct(), rel=1e-12)
    vt, vd = s.potentials()
    np.testing.assert_allclose(vt, vd, rtol=1e-11, atol=1e-11)
    rng = np.random.default_rng(8)
    for _ in range(10):
        i = int(rng.integers(0, 300))
        b = wl["xyz"][i] + rng.uniform(-0.5, 0.5, 3)
        e = s.delta_energy(i, b)
        if e.status:
            continue
        st, d = s.delta_energy_direct(i, b)
        assert e.dE == pytest.approx(d, rel=1e-10, abs=1e-12)


# ---------------------------------------------------------------- adjoint (forces)
def test_forces_euler_identity_and_finite_differences(oracle_mod):
    """E_tree is a quadratic form in the charges: sum_k q_k dE/dq_k = 2E exactly;
    dE/dr and dE/dq agree with FP64 central differences of the rebuilt treecode
    energy (h = 1e-6, where no MAC decision of these targets flips)."""
    wl = W.plain(n=300, seed=3)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"])
    g, dq = s.forces()
    assert float(wl["q"] @ dq) == pytest.approx(2.0 * s.energy_tree(), rel=1e-12)

    def et(xyz, q):
        return oracle_mod.System(wl["params"], q, xyz, len(q)).energy_tree()
    h = 1e-6
    for k in (0, 5, 77, 210):
        for c in range(3):
            xp, xm = wl["xyz"].copy(), wl["xyz"].copy()
            xp[k, c] += h
            xm[k, c] -= h
            assert g[k, c] == pytest.approx((et(xp, wl["q"]) - et(xm, wl["q"])) / (2 * h), abs=1e-6)
        qp, qm = wl["q"].copy(), wl["q"].copy()
        qp[k] += h
        qm[k] -= h
        assert dq[k] == pytest.approx((et(wl["xyz"], qp) - et(wl["xyz"], qm)) / (2 * h), abs=1e-6)


def test_forces_fixed_direct_finite_differences(oracle_mod):
    """Adjoint with the macroion held outside the tree (its pairs exact): dE/dr
    and dE/dq of an ion, an image and the macroion itself agree with FP64
    central differences of the rebuilt treecode energy at theta = 0.5, and
    sum_k q_k dE/dq_k = 2E."""
    wl = W.colloid(n=200, seed=9, p=3, C=4)
    n, nf = wl["n_mobile"], wl["n_fixed"]
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], n, nf)
    g, dq = s.forces()
    q_all, x_all = s.charges()
    assert float(q_all @ dq) == pytest.approx(2.0 * s.energy_tree(), rel=1e-12)
    # images follow their ions in the system, so the energy is rebuilt with the
    # images as independent fixed-position charges: ions, then the images as
    # plain mobile charges (no shell: it does not enter the energy), then the
    # macroion (fixed_direct applies to it)
    params = dict(wl["params"], image=None, shell=None)

    def et(x, q):
        order = list(range(n)) + list(range(n + nf, n + nf + n)) + [n]
        return oracle_mod.System(params, q[order], x[order], 2 * n, nf).energy_tree()
    h = 1e-6
    for k in (7, n, n + nf + 33):  # an ion, the macroion, an image
        for c in range(3):
            xp, xm = x_all.copy(), x_all.copy()
            xp[k, c] += h
            xm[k, c] -= h
            assert g[k, c] == pytest.approx((et(xp, q_all) - et(xm, q_all)) / (2 * h), rel=1e-6, abs=1e-6)
        qp, qm = q_all.copy(), q_all.copy()
        qp[k] += h
        qm[k] -= h
        assert dq[k] == pytest.approx((et(x_all, qp) - et(x_all, qm)) / (2 * h), rel=1e-6, abs=1e-6)


def test_forces_theta_zero_equal_direct_sum(oracle_mod):
    """theta = 0 (all pairs direct): dE/dr_k = -l_B q_k sum_j q_j (r_k - r_j)/r^3 and
    dE/dq_k = l_B sum_j q_j / r_kj, written out from Eq. (1.1)."""
    wl = W.colloid(n=120, seed=4, theta=0.0)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    g, dq = s.forces()
    q, x = s.charges()
    d = x[:, None, :] - x[None, :, :]
    r = np.linalg.norm(d, axis=2)
    np.fill_diagonal(r, np.inf)
    want_r = -(q[:, None, None] * q[None, :, None] * d / r[:, :, None] ** 3).sum(axis=1)
    want_q = (q[None, :] / r).sum(axis=1)
    assert np.allclose(g, want_r, rtol=1e-10, atol=1e-12)
    assert np.allclose(dq, want_q, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- Langevin proposals
def test_ion_energy_gradient_matches_delta_energy(oracle_mod):
    """grad U (ion and its image, with the image chain rule) against central
    differences of the oracle's own dE(i, x) = U(x) - U(a)."""
    wl = W.colloid(n=400, seed=3)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    q, x = s.charges()
    h = 1e-6
    for i in (3, 50, 311):
        pt = x[i] * 1.02
        U, g = s.ion_energy_grad(i, pt)
        assert U - s.ion_energy_grad(i, x[i])[0] == pytest.approx(s.delta_energy(i, pt).dE, abs=1e-12)
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            fd = (s.delta_energy(i, pt + e).dE - s.delta_energy(i, pt - e).dE) / (2 * h)
            assert g[c] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_mala_samples_boltzmann_one_ion(oracle_mod):
    """The Langevin chain samples the same radial density r^2 exp(-beta E(r)) as
    the plain Metropolis chain (one ion and its image around a fixed charge)."""
    lB, beta, Z, R, alpha = 1.0, 1.0, -4.0, 0.8, -0.3
    params = W.base_params(lB=lB, beta=beta, shell=(1.0, 4.0), image=(R, alpha))
    s = oracle_mod.System(params, np.array([1.0, Z]), np.array([[2.0, 0.3, -0.4], [0, 0, 0]]),
                          n_mobile=1, n_fixed=1)
    recs = s.mala_run(seed=78, n_moves=300000, tau=0.2)
    r = np.empty(len(recs))
    cur = np.linalg.norm([2.0, 0.3, -0.4])
    for t, rec in enumerate(recs):
        if rec["outcome"] == 0:
            cur = np.linalg.norm(rec["r_new"])
        r[t] = cur
    grid = np.linspace(1.0, 4.0, 200001)
    E = lB * (Z / grid + alpha * R / (grid ** 2 - R ** 2))
    w = grid ** 2 * np.exp(-beta * E)
    for f in (lambda v: v, lambda v: 1 / v, lambda v: v * v):
        want = np.trapezoid(f(grid) * w, grid) / np.trapezoid(w, grid)
        batches = f(r).reshape(100, -1).mean(axis=1)
        z = (batches.mean() - want) / (batches.std(ddof=1) / 10)
        assert abs(z) < 5, (want, batches.mean(), z)


# ---------------------------------------------------------------- hard cores (Eq. 2.1)
def test_hard_core_contact_rule(oracle_mod):
    """A trial position at distance exactly tau from another mobile ion is
    rejected (the pair potential is infinite for r <= tau); just beyond is not."""
    tau = 1.5
    params = W.base_params(hard_core=tau, root_lo=(-8.0,) * 3, root_side=16.0)
    xyz = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0], [-3.0, 1.0, 0.0]])
    s = oracle_mod.System(params, np.array([1.0, -1.0, 1.0]), xyz, 3, 0)
    assert s.delta_energy(0, [3.0 - tau, 0.0, 0.0]).status == oracle_mod.EOVERLAP
    assert s.delta_energy(0, [3.0 - tau - 1e-9, 0.0, 0.0]).status == 0
    assert s.delta_energy(0, [0.5, 0.5, 0.5]).status == 0
    # the moved ion itself never blocks its own move
    assert s.delta_energy(1, [3.0 + 0.1, 0.0, 0.0]).status == 0
    with pytest.raises(Exception):  # an initial overlap is refused
        oracle_mod.System(params, np.array([1.0, 1.0]), np.array([[0.0, 0, 0], [1.0, 0, 0]]), 2, 0)


def test_hard_core_chain_samples_excluded_volume(oracle_mod):
    """Two neutral hard spheres of diameter tau in a ball of radius R: the chain
    samples the uniform measure on non-overlapping pairs, so the pair distance
    has density f(r) = 3r^2/R^3 - 9r^3/(4R^4) + 3r^5/(16R^6) (two uniform
    points in a ball) restricted to r > tau."""
    R, tau = 2.0, 1.0
    params = W.base_params(hard_core=tau, shell=(0.0, R), root_lo=(-4.0,) * 3, root_side=8.0)
    xyz = np.array([[1.0, 0.0, 0.0], [-1.0, 0.0, 0.0]])
    s = oracle_mod.System(params, np.zeros(2), xyz, 2, 0)
    recs = s.mc_run(seed=91, n_moves=400000, step=1.5)
    assert not np.any(recs["outcome"] == 1)  # neutral: no energy rejections
    pos = xyz.copy()
    d = np.empty(len(recs))
    for t, rec in enumerate(recs):
        if rec["outcome"] == 0:
            pos[rec["i"]] = rec["r_new"]
        d[t] = np.linalg.norm(pos[0] - pos[1])
    assert d.min() > tau
    grid = np.linspace(tau, 2 * R, 200001)
    f = 3 * grid ** 2 / R ** 3 - 9 * grid ** 3 / (4 * R ** 4) + 3 * grid ** 5 / (16 * R ** 6)
    for g in (lambda v: v, lambda v: v * v):
        want = np.trapezoid(g(grid) * f, grid) / np.trapezoid(f, grid)
        batches = g(d).reshape(100, -1).mean(axis=1)
        z = (batches.mean() - want) / (batches.std(ddof=1) / 10)
        assert abs(z) < 5, (want, batches.mean(), z)


def test_edl_hard_initial_configuration(oracle_mod):
    wl = W.edl_hard(n=300, seed=2)
    s = oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])
    q, x = s.charges()
    d2 = np.sum((x[:300, None, :] - x[None, :300, :]) ** 2, axis=2) + np.eye(300) * 1e9
    assert d2.min() > 16.0
