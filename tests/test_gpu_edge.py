"""Edge cases and failure paths of the CUDA library (none of them faults a GPU:
every failure is a status returned by the C-ABI)."""
import numpy as np
import pytest
from tolerances import FLOOR32, REL

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


def _wl(q, xyz, n_mobile, n_fixed=0, **kw):
    return dict(params=W.base_params(**kw), q=np.asarray(q, float), xyz=np.asarray(xyz, float),
                n_mobile=n_mobile, n_fixed=n_fixed)


def test_single_charge_and_pair(bh, oracle_mod):
    one = _wl([1.0], [[0.5, -0.25, 3.0]], 1)
    ctx = bh.Context(one)
    rc, dE, cnt = ctx.delta_energy(0, [1.0, 1.0, 1.0])
    assert rc == 0 and dE == 0.0 and cnt.pairs == 0
    st, _ = ctx.step_mc(20, 1.0, seed=3)
    assert st.accepted == 20
    pair = _wl([2.0, -1.5], [[0.1, 0.2, -0.3], [1.1, -0.4, 0.5]], 2, lB=0.7)
    ctx = bh.Context(pair, precision=bh.PREC_F64)
    b = np.array([-0.9, 0.6, 0.2])
    r0, rb = np.linalg.norm(pair["xyz"][0] - pair["xyz"][1]), np.linalg.norm(b - pair["xyz"][1])
    rc, dE, _ = ctx.delta_energy(0, b)
    assert dE == pytest.approx(0.7 * 2.0 * -1.5 * (1 / rb - 1 / r0), rel=1e-14)


def test_root_leaf_and_theta_zero(bh, oracle_mod):
    wl = W.plain(n=6, seed=4)  # n <= C: the root is a leaf, all terms direct
    ctx, ref = bh.Context(wl), _oracle(oracle_mod, wl)
    assert ctx.export_tree() == ref.export_tree()
    wl = W.plain(n=500, seed=5, theta=0.0)  # theta = 0: no multipole anywhere
    ctx, ref = bh.Context(wl, warps=8, layout=1), _oracle(oracle_mod, wl)
    rng = np.random.default_rng(0)
    for _ in range(10):
        i = int(rng.integers(0, 500))
        b = wl["xyz"][i] + rng.uniform(-0.5, 0.5, 3)
        rc, dE, cnt = ctx.delta_energy(i, b)
        st, d = ref.delta_energy_direct(i, b)
        assert cnt.accepted == 0 and abs(dE - d) <= REL * abs(d) + FLOOR32 * ref.delta_energy(i, b).abs_sum


def test_midplane_ties_tree(bh, oracle_mod):
    rng = np.random.default_rng(21)
    xyz = np.unique(np.round(rng.uniform(-8, 8, (400, 3)) * 2) / 2, axis=0)[:300]
    wl = _wl(rng.choice([-1.0, 1.0], len(xyz)), xyz, len(xyz), C=2, Dmax=6)
    ctx, ref = bh.Context(wl), _oracle(oracle_mod, wl)
    assert ctx.export_tree() == ref.export_tree()
    for t in range(60):  # moves landing exactly on mid-planes
        i = int(rng.integers(0, len(xyz)))
        b = np.round(xyz[i] + rng.uniform(-1, 1, 3))
        assert ctx.commit_move(i, b) == ref.commit_move(i, b)
    assert ctx.export_tree() == ref.export_tree()


def test_capacity_rule(bh, oracle_mod):
    xyz = [[0.1, 0.1, 0.1], [0.2, 0.2, 0.2], [0.3, 0.1, 0.2], [5.0, 5.0, 5.0]]
    with pytest.raises(bh.BhmcError) as e:
        bh.Context(_wl(np.ones(4), xyz, 4, C=2, Dmax=3))
    assert e.value.status == bh.ECAPACITY
    wl = _wl(np.ones(3), xyz[1:], 3, C=2, Dmax=3)
    ctx, ref = bh.Context(wl), _oracle(oracle_mod, wl)
    b = [0.15, 0.15, 0.15]
    assert ctx.commit_move(2, b) == ref.commit_move(2, b) == bh.ECAPACITY
    assert ctx.export_tree() == ref.export_tree()


def test_invalid_inputs(bh):
    wl = W.plain(n=50, seed=6)
    ctx = bh.Context(wl)
    assert ctx.delta_energy(50, [0, 0, 0])[0] == bh.EINVAL
    assert ctx.delta_energy(-1, [0, 0, 0])[0] == bh.EINVAL
    assert ctx.delta_energy(0, [np.nan, 0, 0])[0] == bh.EDOMAIN
    assert ctx.delta_energy(0, [np.inf, 0, 0])[0] == bh.EDOMAIN
    assert ctx.delta_energy(0, [16.0, 0, 0])[0] == bh.EDOMAIN  # upper root face is outside
    assert ctx.commit_move(0, [0, -np.inf, 0]) == bh.EDOMAIN
    bad = dict(wl, xyz=wl["xyz"].copy())
    bad["xyz"][3, 1] = np.nan
    with pytest.raises(bh.BhmcError) as e:
        bh.Context(bad)
    assert e.value.status == bh.EDOMAIN
    fixed_only = _wl([1.0, -1.0], [[0, 0, 0], [1, 1, 1]], 0, 2)
    ctx = bh.Context(fixed_only)
    with pytest.raises(bh.BhmcError) as e:
        ctx.step_mc(5, 1.0, seed=1)
    assert e.value.status == bh.EINVAL


def test_node_pool_exhaustion_is_reported(bh):
    """A pool too small for the next split: the commit returns ENOMEM_POOL and the
    context refuses further work with ESTATE (no fault, no hang)."""
    wl = W.plain(n=300, seed=8, C=2)
    wl["params"]["Dmax"] = 9
    f = 0.05
    while True:  # smallest pool the build fits in
        try:
            ctx = bh.Context(wl, node_factor=f)
            break
        except bh.BhmcError as e:
            assert e.status == bh.ENOMEM_POOL
            f *= 1.25
    rng = np.random.default_rng(2)
    seen = None
    for _ in range(2000):
        i = int(rng.integers(0, 300))
        rc = ctx.commit_move(i, rng.uniform(-9.9, 9.9, 3))
        if rc not in (bh.OK, bh.ECAPACITY):
            seen = rc
            break
    assert seen == bh.ENOMEM_POOL
    assert ctx.delta_energy(0, [0.0, 0.0, 0.0])[0] == bh.ESTATE


def test_batch_pool_exhaustion_stops_the_chain(bh):
    """Batched persistent chains whose node pool runs out: the launch stops a
    chain at its first device error (no move runs on the tree the failed split
    left), the call reports ENOMEM_POOL, the replica's context latches it
    (ESTATE) and nothing faults or waits."""
    systems = []
    for seed in (8, 9):
        wl = W.plain(n=300, seed=seed, C=2)
        wl["params"]["Dmax"] = 9
        systems.append(wl)
    f = 0.05
    while True:  # smallest pool both builds fit in
        try:
            batch = bh.Batch(systems, warps=8, layout=1, node_factor=f)
            break
        except bh.BhmcError as e:
            assert e.status == bh.ENOMEM_POOL
            f *= 1.25
    seen = None
    for call in range(20):
        try:
            batch.step_mc(1000, 3.0, [1, 2], move0=1000 * call)
        except bh.BhmcError as e:
            seen = e.status
            break
    assert seen == bh.ENOMEM_POOL
    states = [batch.replica(r).delta_energy(0, [0.0, 0.0, 0.0])[0] for r in range(2)]
    assert bh.ESTATE in states
    with pytest.raises(bh.BhmcError) as e:
        batch.step_mc(10, 3.0, [1, 2])
    assert e.value.status == bh.ESTATE


def test_positions_and_last_counters(bh, oracle_mod):
    """bhmc_get_positions equals the positions of bhmc_get_charges;
    bhmc_get_counters returns the last evaluation's interaction-list counters."""
    wl = W.colloid(n=800, seed=21)
    ctx = bh.Context(wl, warps=4)
    c0 = ctx.counters()
    assert (c0.visited, c0.accepted, c0.pairs) == (0, 0, 0)
    assert np.array_equal(ctx.positions(), ctx.charges()[1])
    i = 5
    b = wl["xyz"][i] + np.array([0.2, -0.1, 0.3])
    rc, dE, cnt = ctx.delta_energy(i, b)
    assert rc == 0
    last = ctx.counters()
    assert (last.visited, last.accepted, last.pairs) == (cnt.visited, cnt.accepted, cnt.pairs) and cnt.visited > 0
    E, tot = ctx.energy_counters()
    last = ctx.counters()
    assert (last.visited, last.accepted, last.pairs) == (tot.visited, tot.accepted, tot.pairs)


def test_checkpoint_and_resume(bh):
    """A chain stopped after 800 moves, rebuilt from its exported charges (the
    tree is a function of the particle set) and resumed at move 800 with its
    running energy, follows the uninterrupted chain (decisions can differ only
    within the flagged band, since rebuilt moments round differently)."""
    wl = W.edl_hard(n=600, seed=31)
    full = bh.Context(wl, warps=8)
    _, r_full = full.step_mc(1600, 2.0, seed=4, records=True)
    first = bh.Context(wl, warps=8)
    first.step_mc(800, 2.0, seed=4)
    q, x = first.charges()
    n = wl["n_mobile"] + wl["n_fixed"]
    resumed = bh.Context(dict(wl, q=q[:n], xyz=x[:n]), warps=8)
    assert resumed.export_tree() == first.export_tree()
    resumed.set_energy(first.get_energy())
    _, r_res = resumed.step_mc(800, 2.0, seed=4, move0=800, records=True)
    tail = r_full[800:]
    same = tail["outcome"] == r_res["outcome"]
    if same.all():
        assert np.array_equal(tail["r_new"], r_res["r_new"])
        assert np.array_equal(full.charges()[1], resumed.charges()[1])
        assert abs(resumed.get_energy() - full.get_energy()) <= 1e-5 * float(np.abs(tail["dE"]).sum()) + 1e-9
    else:
        k = int(np.argmin(same))
        assert tail["flagged"][k] or r_res["flagged"][k]


def test_bounded_loops_run_out_with_a_status(bh):
    """A host-set budget of two traversal rounds makes the bounded device loops
    run out on ordinary inputs: the trial-move evaluation and the energy pass
    return BHMC_ETIMEOUT, a chain latches it (the next call returns
    BHMC_ESTATE), and nothing faults or waits.  The same system with the
    default budget evaluates normally."""
    wl = W.colloid(n=2000, seed=5)
    i, b = 3, wl["xyz"][3] + 0.1
    ok = bh.Context(wl)
    rc, dE, cnt = ok.delta_energy(i, b)
    assert rc == 0 and cnt.visited > 2
    ok.close()
    wl["params"]["round_limit"] = 2
    ctx = bh.Context(wl)
    rc, dE, cnt = ctx.delta_energy(i, b)
    assert rc == bh.ETIMEOUT
    with pytest.raises(bh.BhmcError) as e:
        ctx.energy()
    assert e.value.status == bh.ETIMEOUT
    with pytest.raises(bh.BhmcError) as e:
        ctx.step_mc(50, 1.0, seed=3)
    assert e.value.status == bh.ETIMEOUT
    with pytest.raises(bh.BhmcError) as e:
        ctx.energy()
    assert e.value.status == bh.ESTATE
    ctx.close()

