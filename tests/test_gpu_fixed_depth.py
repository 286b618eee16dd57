"""The fixed-level tree of Sec. 3.2 on the GPU against the oracle: every
non-empty cluster is bisected down to L_max, so every ion sits in a leaf at
depth L_max and a move may split a chain of empty clusters down to L_max or
merge one back.  Workload: the hard-core double layer of Sec. 4 (valence-2
counterions of diameter 4, macroion radius 30, cell radius 80, l_B = 7.14)."""
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


@pytest.mark.parametrize("Lmax,C,precision", [(6, 8, 0), (5, 32, 0), (6, 8, 1)])
def test_fixed_depth_chain(bh, oracle_mod, Lmax, C, precision):
    wl = W.edl_hard(n=800, seed=8, Lmax=Lmax, C=C)
    ctx = bh.Context(wl, precision=precision, warps=4)
    ref = _oracle(oracle_mod, wl)
    tree = ctx.export_tree()
    assert tree == ref.export_tree()
    assert all(d == Lmax for (d, k), (leaf, c, _) in tree.items() if leaf and c > 0)
    st, rec = ctx.step_mc(2000, wl["step"], seed=17, records=True)
    orec = ref.mc_run(17, 2000, step=wl["step"])
    floor = 1e-12 if precision else FLOOR32
    for t in range(2000):
        assert rec["i"][t] == orec["i"][t] and np.array_equal(rec["r_new"][t], orec["r_new"][t]), t
        assert rec["outcome"][t] == orec["outcome"][t] or orec["flagged"][t] or rec["flagged"][t], t
        if rec["outcome"][t] != orec["outcome"][t]:
            pytest.skip("a flagged decision split the chains at move %d" % t)
        if orec["outcome"][t] in (0, 1):
            assert abs(rec["dE"][t] - orec["dE"][t]) <= REL * abs(orec["dE"][t]) + floor * orec["abs_sum"][t]
    assert np.array_equal(ctx.charges()[1], ref.charges()[1])
    assert ctx.export_tree() == ref.export_tree()
    e, e_ref = ctx.energy(), ref.energy_tree()
    tol = 1e-12 if precision else 2e-6
    assert abs(e - e_ref) <= tol * abs(e_ref) + tol * float(np.abs(wl["q"]).sum())


def test_fixed_depth_batch(bh, oracle_mod):
    systems = [W.edl_hard(n=n, seed=60 + k, Lmax=6) for k, n in enumerate((300, 800, 500))]
    batch = bh.Batch(systems, warps=8)
    seeds = [900 + r for r in range(len(systems))]
    stats = batch.step_mc(500, 2.0, seeds)
    for r, wl in enumerate(systems):
        ref = _oracle(oracle_mod, wl)
        orec = ref.mc_run(seeds[r], 500, step=2.0, replica=r)
        if int(orec["flagged"].sum()) == 0:
            assert stats[r]["accepted"] == int((orec["outcome"] == 0).sum())
            assert np.array_equal(batch.replica(r).charges()[1], ref.charges()[1])
            assert batch.replica(r).export_tree() == ref.export_tree()
