"""Radial distribution (RDF) and integrated charge (ICDF) of the double layer
(Sec. 4, Fig. 6 quantities): the device counts equal numpy's on the same
positions with the same FP64 operations, for one system and for a batch."""
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


def _counts(x, q, nb, lo, hi):
    r = np.sqrt((x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1]) + x[:, 2] * x[:, 2])
    width = (hi - lo) / nb
    t = np.floor((r - lo) / width)
    ok = (r >= lo) & (r < hi) & (t >= 0) & (t < nb)
    c = np.bincount(t[ok].astype(int), minlength=nb)
    s = np.bincount(t[ok].astype(int), weights=q[ok], minlength=nb)
    return c, s


def test_radial_counts_single_and_batch(bh):
    wl = W.edl_hard(n=800, seed=8)
    ctx = bh.Context(wl, warps=8, layout=1)
    ctx.step_mc(3000, 2.0, seed=1)
    nb, lo, hi = 46, 32.0, 78.0
    counts = np.zeros(nb, dtype=np.int64)
    charge = np.zeros(nb)
    ctx.radial_counts(counts, charge, lo, hi)
    q, x = ctx.charges()
    c, s = _counts(x[:800], q[:800], nb, lo, hi)
    assert np.array_equal(counts, c) and counts.sum() == 800
    assert np.allclose(charge, s, rtol=0, atol=1e-9)
    ctx.radial_counts(counts, charge, lo, hi)  # accumulates
    assert np.array_equal(counts, 2 * c)
    systems = [W.edl_hard(n=n, seed=40 + k) for k, n in enumerate((300, 500))]
    batch = bh.Batch(systems, warps=8)
    batch.step_mc(500, 2.0, [1, 2])
    bc = np.zeros(nb, dtype=np.int64)
    bq = np.zeros(nb)
    batch.radial_counts(bc, bq, lo, hi)
    want = np.zeros(nb, dtype=np.int64)
    for r, wl2 in enumerate(systems):
        q2, x2 = batch.replica(r).charges()
        want += _counts(x2[:wl2["n_mobile"]], q2[:wl2["n_mobile"]], nb, lo, hi)[0]
    assert np.array_equal(bc, want)
    k, g, edges, Q = bh.radial_profiles(counts, charge, lo, hi, samples=2, q_fixed=-1600.0)
    assert g.sum() == pytest.approx(1.0) and Q[-1] == pytest.approx(0.0, abs=1e-9)  # the cell is neutral


def test_radial_counts_rejects_bad_bins(bh):
    ctx = bh.Context(W.edl_hard(n=50, seed=1))
    with pytest.raises(bh.BhmcError):
        ctx.radial_counts(np.zeros(4, dtype=np.int64), np.zeros(4), 10.0, 5.0)
