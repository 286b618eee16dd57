"""GPU parity at the workloads' full sizes, in the bench's launch configuration
(8 warps per move, AoS moment mirror), on outputs the oracle computes one by one.

  * colloid, N = 1e4 ions (2e4 + 1 charges), theta x p grid: sampled dE and
    interaction-list counters; a 400-move chain compared move by move;
  * 256 replicas with N in [2000, 50000]: one persistent batched launch, four
    sampled replicas compared with the oracle's chains;
  * large colloid, N = 1e6 ions (2e6 + 1 charges), depth up to 20, p = 6:
    sampled dE and a short chain.
"""
import numpy as np
import pytest

from paper_1305_1825_gb300 import workloads as W

pytestmark = pytest.mark.gpu

from tolerances import FLOOR32, REL
BENCH = dict(warps=8, layout=1)


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


def _check_dE(ctx, ref, wl, n, seed):
    rng = np.random.default_rng(seed)
    done = 0
    for _ in range(n):
        i = int(rng.integers(0, wl["n_mobile"]))
        b = wl["xyz"][i] + rng.uniform(-0.5, 0.5, 3)
        rc, dE, cnt = ctx.delta_energy(i, b)
        e = ref.delta_energy(i, b)
        assert rc == e.status
        if rc:
            continue
        done += 1
        assert (cnt.visited, cnt.accepted, cnt.pairs) == (e.visited, e.accepted, e.pairs)
        assert abs(dE - e.dE) <= REL * abs(e.dE) + FLOOR32 * e.abs_sum
    return done


def _compare_chain(rec, orec):
    for t in range(len(orec)):
        assert rec["i"][t] == orec["i"][t] and np.array_equal(rec["r_new"][t], orec["r_new"][t])
        if rec["outcome"][t] != orec["outcome"][t]:
            assert orec["flagged"][t] or rec["flagged"][t], t
            return t
        if orec["outcome"][t] in (0, 1):
            assert abs(rec["dE"][t] - orec["dE"][t]) <= REL * abs(orec["dE"][t]) + FLOOR32 * orec["abs_sum"][t]
    return len(orec)


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
@pytest.mark.parametrize("p", [2, 4, 6])
def test_colloid_1e4_theta_p_grid(bh, oracle_mod, theta, p):
    wl = W.colloid(n=10000, seed=2, theta=theta, p=p)
    ctx = bh.Context(wl, **BENCH)
    ref = _oracle(oracle_mod, wl)
    assert _check_dE(ctx, ref, wl, 25, seed=int(100 * theta) + p) > 15


def test_colloid_1e4_chain(bh, oracle_mod):
    wl = W.colloid(n=10000, seed=2)
    ctx = bh.Context(wl, **BENCH)
    ref = _oracle(oracle_mod, wl)
    st, rec = ctx.step_mc(400, 1.0, seed=2, records=True)
    orec = ref.mc_run(2, 400)
    assert _compare_chain(rec, orec) == 400
    assert ctx.export_tree() == ref.export_tree()


@pytest.mark.parametrize("C", [8, 16])
def test_batch_256_replicas_sampled(bh, oracle_mod, C):
    """The benchmark's 256 replicas in the benchmark's launch configuration:
    sampled replicas' per-move records (proposal, outcome, dE) against the
    oracle chain move by move, up to the first flagged disagreement; positions
    and trees at the end when no decision was flagged."""
    sizes = W.batch_sizes(256, seed=3)
    systems = W.batch(sizes=sizes, C=C)
    batch = bh.Batch(systems, **BENCH)
    seeds = [1000 + r for r in range(256)]
    stats, recs = batch.step_mc(150, 1.0, seeds, records=True)
    assert all(s["moves"] == 150 for s in stats)
    for r in (0, 77, int(np.argmax(sizes)), 255):
        ref = _oracle(oracle_mod, systems[r])
        orec = ref.mc_run(seeds[r], 150, replica=r)
        upto = _compare_chain(recs[r], orec)
        flagged = int(orec["flagged"].sum())
        assert upto == 150 or orec["flagged"][upto] or recs[r]["flagged"][upto]
        assert abs(stats[r]["accepted"] - int((orec["outcome"] == 0).sum())) <= flagged
        if flagged == 0:
            assert upto == 150
            q, x = batch.replica(r).charges()
            assert np.array_equal(x, ref.charges()[1])
            assert batch.replica(r).export_tree() == ref.export_tree()


@pytest.mark.slow
def test_large_colloid_1e6(bh, oracle_mod):
    wl = W.large()
    ctx = bh.Context(wl, **BENCH)
    ref = _oracle(oracle_mod, wl)
    assert _check_dE(ctx, ref, wl, 12, seed=5) > 8
    st, rec = ctx.step_mc(60, 1.0, seed=9, records=True)
    orec = ref.mc_run(9, 60)
    assert _compare_chain(rec, orec) == 60
    q, x = ctx.charges()
    assert np.array_equal(x, ref.charges()[1])


def _check_potentials(ctx, ref, n, seed, wl):
    """Sampled per-charge treecode potentials phi_j (j excluded) against the
    oracle; the macroion, held outside the tree, has the exact sum."""
    phi = ctx.potentials()
    q, x = ref.charges()
    rng = np.random.default_rng(seed)
    m = wl["n_mobile"]
    for j in list(rng.choice(len(q), n, replace=False)) + [m]:
        if wl["params"].get("fixed_direct") and m <= j < m + wl["n_fixed"]:
            assert phi[j] == pytest.approx(ref.phi_direct(x[j], excl=[int(j)]), rel=1e-11)
            continue
        e = ref.phi(x[j], excl=[int(j)])
        assert abs(phi[j] - e.phi) <= REL * abs(e.phi) + FLOOR32 * e.abs_sum, (j, phi[j], e.phi)
    return phi, q


def test_colloid_1e4_potentials_and_energy(bh, oracle_mod):
    wl = W.colloid(n=10000, seed=2)
    ctx = bh.Context(wl, **BENCH)
    ref = _oracle(oracle_mod, wl)
    phi, q = _check_potentials(ctx, ref, 200, seed=7, wl=wl)
    assert ctx.energy() == pytest.approx(0.5 * float(q @ phi), rel=1e-12)


@pytest.mark.slow
def test_large_colloid_1e6_potentials(bh, oracle_mod):
    wl = W.large()
    ctx = bh.Context(wl, **BENCH)
    ref = _oracle(oracle_mod, wl)
    _check_potentials(ctx, ref, 40, seed=8, wl=wl)
