"""GPU adjoint (forces -dE/dr and dE/dq through the traversal) against the
oracle's adjoint, FP64 central differences and direct-sum forces; the
torch.autograd.Function wrapper.

Element-wise bar: |g_gpu - g_oracle| <= 1e-5 |g_oracle| + c A, per component,
A the oracle's conditioning sum of the adjoint (every term replaced by its
magnitude).  FP32 traversal: c = C32; the FP32 terms (Taylor coefficients to
order p + 1 by the recurrence, products with the FP32 moment mirror, the
cluster adjoints q_i T_n summed over a warp in FP32) carry relative errors of
a few 2^-24 each; measured on the 1500- and 2000-charge systems below, the
largest |error| / A is 2.5e-7 (99th percentile 9e-8), so C32 = 5e-7.  FP64:
measured 3.4e-15, C64 = 1e-13.
"""
import numpy as np
import pytest

from paper_1305_1825_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C32, C64 = 5e-7, 1e-13


@pytest.fixture(scope="module")
def bh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1825_gb300 import bhmc
    return bhmc


def _oracle(oracle_mod, wl):
    return oracle_mod.System(wl["params"], wl["q"], wl["xyz"], wl["n_mobile"], wl["n_fixed"])


def _rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def _elementwise(g, g0, A, c):
    """Max over components of the excess over 1e-5 |g0|, in units of A (<= c passes)."""
    return float(np.max((np.abs(g - g0) - 1e-5 * np.abs(g0)) / A))


@pytest.mark.parametrize("kind", ["plain", "colloid", "colloid-macroion-in-tree"])
def test_forces_match_oracle_adjoint(bh, oracle_mod, kind):
    if kind == "plain":
        wl = W.plain(n=2000)
    else:
        wl = W.colloid(n=1500, seed=4, fixed_direct=(kind == "colloid"))
    ref = _oracle(oracle_mod, wl)
    g0, q0 = ref.forces()
    Ar, Aq = ref.forces_abs()
    for prec, c in ((bh.PREC_F32, C32), (bh.PREC_F64, C64)):
        ctx = bh.Context(wl, precision=prec, warps=8, layout=1)
        g, dq = ctx.forces()
        er, eq = _elementwise(g, g0, Ar, c), _elementwise(dq, q0, Aq, c)
        assert er <= c and eq <= c, (prec, er, eq)
        q, x = ctx.charges()
        assert float(q @ dq) == pytest.approx(2 * ctx.energy(), rel=1e-6 if prec == 0 else 1e-11)


def _direct_forces(q, x, idx, lB):
    out = np.zeros((len(idx), 3))
    for a, k in enumerate(idx):
        d = x[k] - x
        r = np.linalg.norm(d, axis=1)
        r[k] = np.inf
        out[a] = -lB * q[k] * (q[:, None] * d / r[:, None] ** 3).sum(axis=0)
    return out


@pytest.mark.parametrize("n", [100000, pytest.param(1000000, marks=pytest.mark.slow)])
def test_uniform_cube_forces_fd_and_direct(bh, oracle_mod, n):
    """Uniform cube of side 100, alternating charges: FP64 central differences
    (h = 1e-4) of the treecode energy on sampled particles, against the FP64
    and, element-wise with the FP32 bar, the FP32 gradient; samples whose MAC
    decisions change within +-h (interaction counters differ) are flagged.  At
    N = 1e5 the FP32 gradient of every charge is also held to the element-wise
    bar against the FP64 one."""
    wl = W.uniform(n=n, seed=4)
    c64 = bh.Context(wl, precision=bh.PREC_F64, warps=8)
    g64, dq64 = c64.forces()
    c32 = bh.Context(wl, warps=8, layout=1)
    g32, dq32 = c32.forces()
    assert _rel_rms(g32, g64) < 2e-5 and _rel_rms(dq32, dq64) < 2e-5
    Ar = None
    if n <= 100000:  # the oracle's conditioning sums (about a minute of CPU at 1e5)
        Ar, Aq = _oracle(oracle_mod, wl).forces_abs()
        er, eq = _elementwise(g32, g64, Ar, C32), _elementwise(dq32, dq64, Aq, C32)
        assert er <= C32 and eq <= C32, (er, eq)
    rng = np.random.default_rng(11)
    idx = rng.choice(n, 64 if n <= 100000 else 8, replace=False)
    h = 1e-4
    flagged = checked = 0
    for k in idx:
        x0 = wl["xyz"][k].copy()
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            cp = c64.delta_energy(int(k), x0 + e)[2]
            cm = c64.delta_energy(int(k), x0 - e)[2]
            if (cp.visited, cp.accepted, cp.pairs) != (cm.visited, cm.accepted, cm.pairs):
                flagged += 1
                continue
            assert c64.commit_move(int(k), x0 + e) == 0
            ep = c64.energy()
            assert c64.commit_move(int(k), x0 - e) == 0
            em = c64.energy()
            assert c64.commit_move(int(k), x0) == 0
            fd = (ep - em) / (2 * h)
            checked += 1
            assert abs(fd - g64[k, c]) <= 1e-6 * abs(g64[k, c]) + 1e-6, (k, c, fd, g64[k, c])
            if Ar is not None:  # FP32: the same difference quotient, plus the FP32 bar
                assert abs(fd - g32[k, c]) <= 1e-5 * abs(fd) + 1e-6 + C32 * Ar[k, c], (k, c, fd, g32[k, c])
    assert checked >= 0.75 * 3 * len(idx), flagged
    # direct-sum forces on the sampled particles: within the truncation error
    q, x = c64.charges()
    d = _direct_forces(q, x, idx, 1.0)
    assert _rel_rms(g64[idx], d) < 1e-2


def test_scaled_colloid_forces_vs_direct(bh):
    """The colloid radial law scaled to N = 1e5 (with images): sampled forces
    against the direct sum over all charges."""
    wl = W.colloid_scaled(n=100000)
    ctx = bh.Context(wl, warps=8, layout=1)
    g, dq = ctx.forces()
    q, x = ctx.charges()
    idx = np.random.default_rng(12).choice(len(q), 64, replace=False)
    assert _rel_rms(g[idx], _direct_forces(q, x, idx, 1.0)) < 1e-2
    phi_d = np.array([(np.delete(q, k) / np.linalg.norm(np.delete(x, k, 0) - x[k], axis=1)).sum() for k in idx])
    # dE/dq_k = l_B phi_k exactly for the direct sum; the treecode within its truncation error
    assert _rel_rms(dq[idx], phi_d) < 1e-2


def test_autograd_function(bh, oracle_mod):
    import torch
    from paper_1305_1825_gb300.autograd import treecode_energy
    wl = W.plain(n=1500, seed=9)
    q = torch.tensor(wl["q"], device="cuda", requires_grad=True)
    xyz = torch.tensor(wl["xyz"], device="cuda", requires_grad=True)
    E = treecode_energy(q, xyz, wl["params"], precision=bh.PREC_F64)
    E.backward()
    ref = _oracle(oracle_mod, wl)
    g0, q0 = ref.forces()
    assert E.item() == pytest.approx(ref.energy_tree(), rel=1e-11)
    assert _rel_rms(xyz.grad.cpu().numpy(), g0) < 1e-11
    assert _rel_rms(q.grad.cpu().numpy(), q0) < 1e-11
