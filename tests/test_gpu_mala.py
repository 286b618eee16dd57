"""GPU Metropolis-adjusted Langevin single-ion moves against the oracle's chain.

The proposal b = a - tau beta grad U(a) + sqrt(2 tau) xi needs the gradient of
the single-ion energy (ion and image, with the image chain rule), so the chain
checks the gradient traversal too:
  * FP64 traversal: proposals within 1e-9 (the gradients agree to rounding),
    dE within 1e-9 |dE| + 1e-10, outcomes identical except flagged decisions
    (|ln acceptance - ln alpha| < 1e-6);
  * FP32 traversal: proposals within 1e-4 (relative gradient error ~1e-6,
    scaled by tau beta), outcomes identical except flagged decisions;
  * one ion and its image around a fixed charge: the chain samples the radial
    Boltzmann density r^2 exp(-beta E(r)).
"""
import numpy as np
import pytest

from paper_1305_1825_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def _compare(rec, orec, r_tol, dE_tol):
    """Number of moves that agree before the first (flagged) outcome difference."""
    for t in range(len(orec)):
        assert rec["i"][t] == orec["i"][t], t
        assert np.abs(rec["r_new"][t] - orec["r_new"][t]).max() <= r_tol, (t, rec["r_new"][t], orec["r_new"][t])
        if rec["outcome"][t] != orec["outcome"][t]:
            assert orec["flagged"][t] or rec["flagged"][t], t
            return t
        if dE_tol is not None and orec["outcome"][t] in (0, 1):
            assert abs(rec["dE"][t] - orec["dE"][t]) <= dE_tol * (abs(orec["dE"][t]) + 0.1), t
    return len(orec)


@pytest.mark.parametrize("kind", ["colloid", "plain"])
def test_mala_chain_f64(bh, oracle_mod, kind):
    wl = W.colloid(n=1200, seed=5) if kind == "colloid" else W.plain(n=1500)
    ctx = bh.Context(wl, precision=bh.PREC_F64, warps=4)
    ref = _oracle(oracle_mod, wl)
    tau = 0.5
    st1, rec1 = ctx.step_mala(200, tau, seed=21, records=True)
    st2, rec2 = ctx.step_mala(100, tau, seed=21, move0=200, records=True)
    rec = np.concatenate([rec1, rec2])
    orec = ref.mala_run(21, 300, tau)
    assert _compare(rec, orec, 1e-9, 1e-9) == 300
    acc = int((orec["outcome"] == 0).sum())
    assert st1.moves + st2.moves == 300 and st1.accepted + st2.accepted == acc
    assert 30 < acc < 300  # the step is neither frozen nor unconditionally accepted
    q, x = ctx.charges()
    assert np.allclose(x, ref.charges()[1], rtol=0, atol=1e-9)
    assert ctx.export_tree() == ref.export_tree()
    assert st2.energy == pytest.approx(orec["dE"][orec["outcome"] == 0].sum(), abs=1e-8)


@pytest.mark.parametrize("warps,layout", [(8, 1), (2, 0)])
def test_mala_chain_f32(bh, oracle_mod, warps, layout):
    wl = W.colloid(n=2000, seed=6)
    ctx = bh.Context(wl, warps=warps, layout=layout)
    ref = _oracle(oracle_mod, wl)
    st, rec = ctx.step_mala(300, 0.3, seed=33, records=True)
    orec = ref.mala_run(33, 300, 0.3)
    upto = _compare(rec, orec, 1e-4, 1e-4)
    assert upto == 300 or orec["flagged"][upto] or rec["flagged"][upto]


def test_mala_samples_boltzmann_one_ion(bh):
    lB, beta, Z, R, alpha = 1.0, 1.0, -4.0, 0.8, -0.3
    params = W.base_params(lB=lB, beta=beta, shell=(1.0, 4.0), image=(R, alpha))
    wl = dict(params=params, q=np.array([1.0, Z]), xyz=np.array([[2.0, 0.3, -0.4], [0, 0, 0]]),
              n_mobile=1, n_fixed=1)
    ctx = bh.Context(wl, warps=1)
    n = 200000
    st, recs = ctx.step_mala(n, 0.2, seed=79, records=True)
    r = np.empty(n)
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


def test_mala_invalid_arguments(bh):
    wl = W.plain(n=200)
    ctx = bh.Context(wl)
    for tau in (0.0, -1.0, float("nan")):
        with pytest.raises(bh.BhmcError):
            ctx.step_mala(10, tau, seed=1)
    st, _ = ctx.step_mala(0, 0.1, seed=1)
    assert st.moves == 0
