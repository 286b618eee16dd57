"""Radial distribution (RDF) and integrated charge (ICDF) of the double layer
(Sec. 4, Fig. 6 quantities) on the GPU against the oracle:

* snapshot counts (bhmc_radial_counts) equal the oracle's or_radial_counts of
  the same configuration, for one system and for a batch;
* the samples accumulated inside the chains (bhmc_set_radial_sampling) equal
  the oracle chain's snapshots taken after the same moves, bin by bin and
  exactly (integer counts; the charge sums are sums of small integers), for
  the one-move-per-launch chain, the batched persistent kernel and the cluster
  chain, as long as the chains agree move by move."""
import numpy as np
import pytest

from paper_1305_1825_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NB, LO, HI = 46, 32.0, 78.0


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


def _oracle_samples(oracle_mod, wl, seed, n_moves, every, step, move0=0, replica=0):
    """The oracle chain run in pieces that end at the sample points, a snapshot
    after each; returns (counts, charge, samples, flagged before the end)."""
    ref = _oracle(oracle_mod, wl)
    counts, charge = np.zeros(NB, dtype=np.int64), np.zeros(NB)
    m, ns, flagged = move0, 0, 0
    while m < move0 + n_moves:
        nxt = min(((m // every) + 1) * every, move0 + n_moves)
        rec = ref.mc_run(seed, nxt - m, step=step, m0=m, replica=replica)
        flagged += int(rec["flagged"].sum())
        if nxt % every == 0:
            ref.radial_counts(NB, LO, HI, counts, charge)
            ns += 1
        m = nxt
    return counts, charge, ns, flagged


def test_radial_counts_single_and_batch(bh, oracle_mod):
    wl = W.edl_hard(n=800, seed=8)
    ctx = bh.Context(wl, warps=8, layout=1)
    ctx.step_mc(3000, 2.0, seed=1)
    counts = np.zeros(NB, dtype=np.int64)
    charge = np.zeros(NB)
    ctx.radial_counts(counts, charge, LO, HI)
    q, x = ctx.charges()
    snap = dict(wl, xyz=x[:801])
    c, s = _oracle(oracle_mod, snap).radial_counts(NB, LO, HI)
    assert np.array_equal(counts, c) and counts.sum() == 800
    assert np.array_equal(charge, s)
    ctx.radial_counts(counts, charge, LO, HI)  # accumulates
    assert np.array_equal(counts, 2 * c)
    systems = [W.edl_hard(n=n, seed=40 + k) for k, n in enumerate((300, 500))]
    batch = bh.Batch(systems, warps=8)
    batch.step_mc(500, 2.0, [1, 2])
    bc = np.zeros(NB, dtype=np.int64)
    bq = np.zeros(NB)
    batch.radial_counts(bc, bq, LO, HI)
    want = np.zeros(NB, dtype=np.int64)
    for r, wl2 in enumerate(systems):
        q2, x2 = batch.replica(r).charges()
        want += _oracle(oracle_mod, dict(wl2, xyz=x2[:wl2["n_mobile"] + 1])).radial_counts(NB, LO, HI)[0]
    assert np.array_equal(bc, want)


@pytest.mark.parametrize("path", ["plain", "cluster-4", "mala"])
def test_chain_samples_match_oracle(bh, oracle_mod, path):
    wl = W.edl_hard(n=400, seed=21)
    # the Langevin proposals follow the gradient: the FP64 context keeps them
    # within 1e-9 of the oracle's, the FP32 one only within the traversal error
    prec = bh.PREC_F64 if path == "mala" else bh.PREC_F32
    ctx = bh.Context(wl, warps=8, layout=1, precision=prec)
    ctx.set_radial_sampling(NB, LO, HI, every=25)
    if path == "mala":
        ctx.step_mala(300, 2.0, seed=6)
        ref = _oracle(oracle_mod, wl)
        counts, charge, ns = np.zeros(NB, dtype=np.int64), np.zeros(NB), 0
        flagged = 0
        for m in range(0, 300, 25):
            rec = ref.mala_run(6, 25, 2.0, m0=m)
            flagged += int(rec["flagged"].sum())
            ref.radial_counts(NB, LO, HI, counts, charge)
            ns += 1
    else:
        # two calls, split off a sample point: the samples follow the absolute move index
        for m0, n in ((0, 310), (310, 290)):
            if path == "plain":
                ctx.step_mc(n, 2.0, seed=6, move0=m0)
            else:
                ctx.step_mc_spec(n, 2.0, seed=6, move0=m0, proposals=4)
        counts, charge, ns, flagged = _oracle_samples(oracle_mod, wl, 6, 600, 25, 2.0)
    gc, gq, gn = ctx.radial_samples()
    assert gn == ns
    if flagged == 0:
        assert np.array_equal(gc, counts) and np.array_equal(gq, charge)
        assert gc.sum() == ns * 400


def test_batch_samples_match_oracle(bh, oracle_mod):
    systems = [W.edl_hard(n=n, seed=60 + k) for k, n in enumerate((300, 500, 400))]
    batch = bh.Batch(systems, warps=8)
    batch.set_radial_sampling(NB, LO, HI, every=40)
    seeds = [71, 72, 73]
    batch.step_mc(250, 2.0, seeds)
    batch.step_mc(150, 2.0, seeds, move0=250)
    gc, gq, gn = batch.radial_samples()
    for r, wl in enumerate(systems):
        counts, charge, ns, flagged = _oracle_samples(oracle_mod, wl, seeds[r], 400, 40, 2.0, replica=r)
        assert gn[r] == ns == 10
        if flagged == 0:
            assert np.array_equal(gc[r], counts) and np.array_equal(gq[r], charge)


def test_radial_sampling_rejects_bad_arguments(bh):
    ctx = bh.Context(W.edl_hard(n=50, seed=1))
    with pytest.raises(bh.BhmcError):
        ctx.radial_counts(np.zeros(4, dtype=np.int64), np.zeros(4), 10.0, 5.0)
    with pytest.raises(bh.BhmcError):
        ctx.set_radial_sampling(8, 10.0, 5.0, 10)
    with pytest.raises(bh.BhmcError):  # sampling off: nothing to read
        bh.bhmc_get_radial_samples(ctx.h, 8)
