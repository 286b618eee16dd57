"""GPU parity: the CUDA path (through the C-ABI) against the FP64 CPU oracle.

Bars:
  * tree structure, leaf membership, interaction-list counters, proposals and
    accept/reject sequences: exact (decisions with |beta dE + ln alpha| < 1e-6
    are flagged and may differ);
  * dE, FP32 traversal: |dE_gpu - dE_oracle| <= 1e-5 |dE_oracle| + 1e-7 * A,
    A = l_B sum over the interaction lists of |term| (derivation in
    tests/tolerances.py);
  * dE, FP64 mode: |dE_gpu - dE_oracle| <= 1e-12 * A.
"""
import numpy as np
import pytest

from paper_1305_1825_gb300 import workloads as W

pytestmark = pytest.mark.gpu

from tolerances import FLOOR32, FLOOR64, REL


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


def _off_tree(wl, j):
    """Charge j is a fixed charge held outside the tree (exact interactions)."""
    return bool(wl["params"].get("fixed_direct")) and wl["n_mobile"] <= j < wl["n_mobile"] + wl["n_fixed"]


def _moves(wl, n, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        i = int(rng.integers(0, wl["n_mobile"]))
        yield i, wl["xyz"][i] + rng.uniform(-scale, scale, 3)


@pytest.mark.parametrize("kind", ["plain", "colloid", "colloid-macroion-in-tree"])
def test_build_matches_oracle(bh, oracle_mod, kind):
    wl = W.plain(n=2000) if kind == "plain" else W.colloid(n=2000, seed=4, fixed_direct=(kind == "colloid"))
    ctx = bh.Context(wl)
    ref = _oracle(oracle_mod, wl)
    tree, moms = ctx.export_tree(moments=True)
    assert tree == ref.export_tree()
    for (d, k) in list(tree)[::5]:
        _, M = ref.node_moments(d, k)
        assert np.allclose(moms[(d, k)], M, rtol=1e-11, atol=1e-11 * (np.abs(M).max() + 1.0))
    q, x = ctx.charges()
    q0, x0 = ref.charges()
    assert np.array_equal(q, q0) and np.array_equal(x, x0)


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_delta_energy_matches_oracle(bh, oracle_mod, theta, p):
    wl = W.colloid(n=2000, seed=5, theta=theta, p=p)
    ref = _oracle(oracle_mod, wl)
    for warps, layout in [(1, 0), (2, 1), (4, 0)]:
        ctx = bh.Context(wl, warps=warps, layout=layout)
        n = 0
        for i, b in _moves(wl, 40, seed=p * 10 + int(theta * 10)):
            rc, dE, cnt = ctx.delta_energy(i, b)
            e = ref.delta_energy(i, b)
            assert rc == e.status
            if rc:
                continue
            n += 1
            assert (cnt.visited, cnt.accepted, cnt.pairs) == (e.visited, e.accepted, e.pairs)
            assert abs(dE - e.dE) <= REL * abs(e.dE) + FLOOR32 * e.abs_sum, (dE, e.dE, e.abs_sum)
        assert n > 20
        ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("p", [2, 4])
def test_delta_energy_macroion_in_tree(bh, oracle_mod, p, precision):
    """The reading with the macroion as an ordinary tree charge (fixed_direct
    off) stays available and matches the oracle under the same reading."""
    wl = W.colloid(n=2000, seed=5, p=p, fixed_direct=False)
    ref = _oracle(oracle_mod, wl)
    ctx = bh.Context(wl, precision=precision, warps=4)
    n = 0
    for i, b in _moves(wl, 40, seed=90 + p):
        rc, dE, cnt = ctx.delta_energy(i, b)
        e = ref.delta_energy(i, b)
        assert rc == e.status
        if rc:
            continue
        n += 1
        assert (cnt.visited, cnt.accepted, cnt.pairs) == (e.visited, e.accepted, e.pairs)
        bar = FLOOR64 * e.abs_sum if precision else REL * abs(e.dE) + FLOOR32 * e.abs_sum
        assert abs(dE - e.dE) <= bar, (dE, e.dE, e.abs_sum)
    assert n > 20


@pytest.mark.parametrize("p", [8, 10])
def test_delta_energy_high_order_f64(bh, oracle_mod, p):
    """All-FP64 traversal at the highest orders against the oracle."""
    wl = W.colloid(n=1500, seed=15, p=p)
    ref = _oracle(oracle_mod, wl)
    ctx = bh.Context(wl, precision=bh.PREC_F64, warps=4)
    n = 0
    for i, b in _moves(wl, 40, seed=70 + p):
        rc, dE, cnt = ctx.delta_energy(i, b)
        e = ref.delta_energy(i, b)
        assert rc == e.status
        if rc:
            continue
        n += 1
        assert (cnt.visited, cnt.accepted, cnt.pairs) == (e.visited, e.accepted, e.pairs)
        assert abs(dE - e.dE) <= FLOOR64 * e.abs_sum
    assert n > 20


def test_delta_energy_plain_config_every_move(bh, oracle_mod):
    """The 2000-charge plain system: dE against the oracle treecode and within the
    truncation bound of the direct sum, FP32 and FP64 modes."""
    wl = W.plain(n=2000)
    ref = _oracle(oracle_mod, wl)
    ref.set_bound(True)
    c32 = bh.Context(wl, precision=bh.PREC_F32)
    c64 = bh.Context(wl, precision=bh.PREC_F64)
    for i, b in _moves(wl, 200, seed=11):
        e = ref.delta_energy(i, b)
        st, d = ref.delta_energy_direct(i, b)
        rc, g32, cnt = c32.delta_energy(i, b)
        rc2, g64, cnt2 = c64.delta_energy(i, b)
        assert rc == rc2 == e.status == st == 0
        assert abs(g32 - e.dE) <= REL * abs(e.dE) + FLOOR32 * e.abs_sum
        assert abs(g64 - e.dE) <= FLOOR64 * e.abs_sum
        assert abs(g32 - d) <= e.bound + FLOOR32 * e.abs_sum
        assert (cnt.visited, cnt.accepted, cnt.pairs) == (cnt2.visited, cnt2.accepted, cnt2.pairs)


def test_rejections_match(bh, oracle_mod):
    wl = W.colloid(n=800, seed=6)
    ctx = bh.Context(wl)
    ref = _oracle(oracle_mod, wl)
    q, x = ref.charges()
    cases = [(0, np.array([0.0, 0.0, 1.0])), (1, np.array([60.0, 0.0, 0.0])), (2, np.array([70.0, 0, 0]))]
    for i, b in cases:
        rc, dE, _ = ctx.delta_energy(i, b)
        assert rc == ref.delta_energy(i, b).status != 0
        assert ctx.commit_move(i, b) == rc


@pytest.mark.parametrize("kind", ["plain", "colloid"])
def test_commit_matches_oracle(bh, oracle_mod, kind):
    """Forced commits with splits and merges: tree and moments follow the oracle."""
    if kind == "plain":
        wl = W.plain(n=600, seed=8, C=2)
        wl["params"]["Dmax"] = 9
    else:
        wl = W.colloid(n=400, seed=9, C=3)
        wl["params"]["Dmax"] = 10
    ctx = bh.Context(wl)
    ref = _oracle(oracle_mod, wl)
    rng = np.random.default_rng(1)
    done = 0
    for t in range(300):
        q, x = ref.charges()
        i = int(rng.integers(0, wl["n_mobile"]))
        b = x[i] + rng.uniform(-1.5, 1.5, 3)
        st = ref.commit_move(i, b)
        assert ctx.commit_move(i, b) == st
        done += st == 0
        if t % 25 == 0:
            tree, moms = ctx.export_tree(moments=True)
            assert tree == ref.export_tree()
            for key in list(tree)[::9]:
                _, M = ref.node_moments(*key)
                assert np.allclose(moms[key], M, rtol=1e-9, atol=1e-9 * (np.abs(M).max() + 1.0))
    assert done > 150
    assert ctx.export_tree() == ref.export_tree()
    q, x = ctx.charges()
    q0, x0 = ref.charges()
    assert np.array_equal(x, x0) and np.array_equal(q, q0)


def _compare_chain(rec, orec):
    """Exact proposals and outcomes up to the first flagged disagreement."""
    n = len(orec)
    for t in range(n):
        assert rec["i"][t] == orec["i"][t]
        assert np.array_equal(rec["r_new"][t], orec["r_new"][t])
        if rec["outcome"][t] != orec["outcome"][t]:
            assert orec["flagged"][t] or rec["flagged"][t], t
            return t
        if orec["outcome"][t] in (0, 1):
            assert abs(rec["dE"][t] - orec["dE"][t]) <= REL * abs(orec["dE"][t]) + FLOOR32 * orec["abs_sum"][t]
    return n


@pytest.mark.parametrize("precision", [0, 1])
def test_mc_chain_plain_config(bh, oracle_mod, precision):
    """The 1000-move Metropolis chain of the plain 2000-charge system (seed 1)."""
    wl = W.plain(n=2000)
    ctx = bh.Context(wl, precision=precision)
    ref = _oracle(oracle_mod, wl)
    st, rec = ctx.step_mc(1000, 1.0, seed=1, records=True)
    orec = ref.mc_run(1, 1000)
    upto = _compare_chain(rec, orec)
    assert upto == 1000
    assert st.moves == 1000 and st.accepted == int((orec["outcome"] == 0).sum())
    assert ctx.export_tree() == ref.export_tree()
    assert st.energy == pytest.approx(orec["dE"][orec["outcome"] == 0].sum(), abs=1e-6 * orec["abs_sum"].max())


@pytest.mark.parametrize("warps", [1, 4])
@pytest.mark.parametrize("fixed_direct", [True, False])
def test_mc_chain_colloid(bh, oracle_mod, fixed_direct, warps):
    """The colloid chain (ion and image moved together) move by move against
    the oracle's; one warp runs decision and commit alone (merge and split
    tests of both moved charges in turn), four split them."""
    wl = W.colloid(n=2000, seed=10, fixed_direct=fixed_direct)
    ctx = bh.Context(wl, warps=warps)
    ref = _oracle(oracle_mod, wl)
    st, rec = ctx.step_mc(600, 1.0, seed=2, records=True)
    orec = ref.mc_run(2, 600)
    assert _compare_chain(rec, orec) == 600
    assert ctx.export_tree() == ref.export_tree()


@pytest.mark.parametrize("warps", [1, 2, 8])
def test_batch_replicas_match_oracle_chains(bh, oracle_mod, warps):
    """Persistent batched chains against the oracle's; with 8 warps the next
    move's setup is computed while the current move is decided."""
    sizes = [660, 1000, 760, 900]
    systems = W.batch(sizes=sizes)
    batch = bh.Batch(systems, warps=warps)
    seeds = [1000 + r for r in range(len(sizes))]
    stats = batch.step_mc(150, 1.0, seeds)
    stats2 = batch.step_mc(100, 1.0, seeds, move0=150)
    for r, wl in enumerate(systems):
        ref = _oracle(oracle_mod, wl)
        orec = ref.mc_run(seeds[r], 250, replica=r)
        acc = int((orec["outcome"] == 0).sum())
        flagged = int(orec["flagged"].sum())
        assert abs(stats[r]["accepted"] + stats2[r]["accepted"] - acc) <= flagged
        if flagged == 0:
            assert batch.replica(r).export_tree() == ref.export_tree()
            q, x = batch.replica(r).charges()
            assert np.array_equal(x, ref.charges()[1])


def test_full_energy(bh, oracle_mod):
    for wl in (W.plain(n=1500), W.colloid(n=1200, seed=12), W.colloid(n=1200, seed=12, fixed_direct=False)):
        ref = _oracle(oracle_mod, wl)
        for prec, tol in ((0, 2e-6), (1, 1e-12)):
            ctx = bh.Context(wl, precision=prec)
            e_tree = ctx.energy()
            e_ref = ref.energy_tree()
            scale = float(np.abs(wl["q"]).sum())
            assert abs(e_tree - e_ref) <= tol * abs(e_ref) + tol * scale
            # FP64 sums of N^2/2 mixed-sign pairs in different orders
            assert ctx.energy_direct() == pytest.approx(ref.energy_direct(), rel=1e-9)


@pytest.mark.parametrize("fixed_direct", [True, False])
@pytest.mark.parametrize("precision", [0, 1])
def test_energy_counters_match_oracle(bh, oracle_mod, precision, fixed_direct):
    """The full-energy pass's interaction lists, summed over all targets, equal
    the oracle's per-target traversals (target j excluded)."""
    wl = W.colloid(n=600, seed=12, fixed_direct=fixed_direct)
    ctx = bh.Context(wl, precision=precision, warps=2)
    ref = _oracle(oracle_mod, wl)
    E, cnt = ctx.energy_counters()
    assert E == ctx.energy()
    q, x = ref.charges()
    want = np.zeros(3, dtype=np.int64)
    for j in range(len(q)):
        if _off_tree(wl, j):  # the macroion's potential is an exact sum, not a traversal
            continue
        e = ref.phi(x[j], excl=[j])
        want += (e.visited, e.accepted, e.pairs)
    assert (cnt.visited, cnt.accepted, cnt.pairs) == tuple(int(v) for v in want)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("p", [4, 6, 10])
def test_energy_after_chain(bh, oracle_mod, layout, p):
    """The full-energy pass after a chain of accepted moves (at p = 6 it
    evaluates coefficients refreshed from the running moments) against the
    oracle's treecode energy of the same final configuration."""
    wl = W.colloid(n=1200, seed=13, p=p)
    ctx = bh.Context(wl, warps=8, layout=layout)
    ref = _oracle(oracle_mod, wl)
    st, rec = ctx.step_mc(400, 1.0, seed=5, records=True)
    orec = ref.mc_run(5, 400)
    assert _compare_chain(rec, orec) == 400
    assert st.accepted > 200
    e_tree = ctx.energy()
    e_ref = ref.energy_tree()
    scale = float(np.abs(wl["q"]).sum())
    assert abs(e_tree - e_ref) <= 2e-6 * abs(e_ref) + 2e-6 * scale


@pytest.mark.parametrize("p", [2, 6, 10])
def test_potentials_sampled(bh, oracle_mod, p):
    """Per-charge treecode potentials of the full-energy pass (recurrence at
    p = 2, evaluation coefficients at p = 6 and 10) against the oracle, sampled."""
    wl = W.colloid(n=2000, seed=14, p=p)
    ctx = bh.Context(wl, warps=4, layout=1)
    ref = _oracle(oracle_mod, wl)
    phi = ctx.potentials()
    q, x = ref.charges()
    rng = np.random.default_rng(p)
    for j in list(rng.choice(len(q), 150, replace=False)) + [wl["n_mobile"]]:
        if _off_tree(wl, j):  # the macroion: the exact sum over all other charges
            assert phi[j] == pytest.approx(ref.phi_direct(x[j], excl=[int(j)]), rel=1e-12)
            continue
        e = ref.phi(x[j], excl=[int(j)])
        assert abs(phi[j] - e.phi) <= REL * abs(e.phi) + FLOOR32 * e.abs_sum, (j, phi[j], e.phi)


@pytest.mark.parametrize("p", [0, 1, 3, 5, 7, 8, 9, 10])
def test_chain_and_energy_every_order(bh, oracle_mod, p):
    """Orders beyond the benchmark's: a batched chain (8 warps) and the full
    energy against the oracle."""
    wl = W.colloid(n=1500, seed=20 + p, p=p)
    ref = _oracle(oracle_mod, wl)
    batch = bh.Batch([wl], warps=8)
    st = batch.step_mc(300, 1.0, [31])
    orec = ref.mc_run(31, 300, replica=0)
    flagged = int(orec["flagged"].sum())
    assert abs(st[0]["accepted"] - int((orec["outcome"] == 0).sum())) <= flagged
    if flagged == 0:
        assert batch.replica(0).export_tree() == ref.export_tree()
    ctx = bh.Context(wl, warps=4, layout=1)
    ref0 = _oracle(oracle_mod, wl)
    scale = float(np.abs(wl["q"]).sum())
    assert abs(ctx.energy() - ref0.energy_tree()) <= 2e-6 * abs(ref0.energy_tree()) + 2e-6 * scale
