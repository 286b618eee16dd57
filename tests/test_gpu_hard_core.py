"""Hard cores of Eq. (2.1) on the GPU against the oracle: the electric double
layer of Sec. 4 (valence-2 counterions of diameter 4 around a macroion of
radius 30 in a cell of radius 80, l_B = 7.14).  A trial position within the
diameter of another mobile ion is rejected before evaluation (outcome 3,
dE = 0); the chains must agree move by move, rejections included."""
import numpy as np
import pytest

from paper_1305_1825_gb300 import workloads as W

pytestmark = pytest.mark.gpu

from tolerances import FLOOR32, REL


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


def _compare_chain(rec, orec, dE_floor):
    for t in range(len(orec)):
        assert rec["i"][t] == orec["i"][t] and np.array_equal(rec["r_new"][t], orec["r_new"][t]), t
        if rec["outcome"][t] != orec["outcome"][t]:
            assert orec["flagged"][t] or rec["flagged"][t], (t, rec["outcome"][t], orec["outcome"][t])
            return t
        if orec["outcome"][t] in (0, 1):
            assert abs(rec["dE"][t] - orec["dE"][t]) <= REL * abs(orec["dE"][t]) + dE_floor * orec["abs_sum"][t]
        else:
            assert rec["dE"][t] == 0.0
    return len(orec)


@pytest.mark.parametrize("precision", [0, 1])
def test_edl_hard_core_chain(bh, oracle_mod, precision):
    wl = W.edl_hard(n=800, seed=8)
    ctx = bh.Context(wl, precision=precision, warps=4)
    ref = _oracle(oracle_mod, wl)
    st, rec = ctx.step_mc(2000, wl["step"], seed=17, records=True)
    orec = ref.mc_run(17, 2000, step=wl["step"])
    n_hc = int((orec["outcome"] == 3).sum())
    assert n_hc > 20  # the step makes hard-core rejections common
    assert _compare_chain(rec, orec, 1e-12 if precision else FLOOR32) == 2000
    q, x = ctx.charges()
    assert np.array_equal(x, ref.charges()[1])
    assert ctx.export_tree() == ref.export_tree()


def test_delta_energy_at_contact(bh, oracle_mod):
    wl = W.edl_hard(n=200, seed=3)
    ctx = bh.Context(wl, warps=2)
    ref = _oracle(oracle_mod, wl)
    x = wl["xyz"]
    rng = np.random.default_rng(1)
    for _ in range(40):
        i, j = rng.choice(200, 2, replace=False)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        for dist in (4.0, 4.0 * (1 - 1e-12), 4.0 * (1 + 1e-9), 3.0, 5.0):
            b = x[j] + dist * u
            rc, dE, cnt = ctx.delta_energy(int(i), b)
            e = ref.delta_energy(int(i), b)
            assert rc == e.status, (dist, rc, e.status)


def test_initial_overlap_rejected(bh):
    wl = W.edl_hard(n=100, seed=4)
    xyz = wl["xyz"].copy()
    u = xyz[1] / np.linalg.norm(xyz[1])
    xyz[0] = xyz[1] + 3.9 * np.cross(u, [0.0, 0.0, 1.0]) / np.linalg.norm(np.cross(u, [0.0, 0.0, 1.0]))
    bad = dict(wl, xyz=xyz)
    with pytest.raises(bh.BhmcError):
        bh.Context(bad)


def test_batch_hard_core(bh, oracle_mod):
    systems = [W.edl_hard(n=n, seed=50 + k) for k, n in enumerate((300, 800, 500, 650))]
    batch = bh.Batch(systems, warps=8)
    seeds = [700 + r for r in range(len(systems))]
    stats = batch.step_mc(400, 2.0, seeds)
    for r, wl in enumerate(systems):
        ref = _oracle(oracle_mod, wl)
        orec = ref.mc_run(seeds[r], 400, step=2.0, replica=r)
        flagged = int(orec["flagged"].sum())
        assert abs(stats[r]["accepted"] - int((orec["outcome"] == 0).sum())) <= flagged
        assert stats[r]["rej_overlap"] == int((orec["outcome"] == 3).sum()) or flagged
        if flagged == 0:
            assert np.array_equal(batch.replica(r).charges()[1], ref.charges()[1])


def test_mala_hard_core_f64(bh, oracle_mod):
    wl = W.edl_hard(n=400, seed=9)
    ctx = bh.Context(wl, precision=bh.PREC_F64, warps=4)
    ref = _oracle(oracle_mod, wl)
    st, rec = ctx.step_mala(300, 2.0, seed=4, records=True)
    orec = ref.mala_run(4, 300, 2.0)
    assert int((orec["outcome"] == 3).sum()) > 0
    for t in range(300):
        assert rec["i"][t] == orec["i"][t]
        assert np.abs(rec["r_new"][t] - orec["r_new"][t]).max() <= 1e-9
        assert rec["outcome"][t] == orec["outcome"][t] or orec["flagged"][t]
