"""RDF and integrated charge of Sec. 4 (Fig. 6) on the host, no GPU.

Oracle pins (or_radial_counts, or_radial_profiles): a uniform density in a
shell gives a flat g whose bins sum to one; the integrated charge of an
electroneutral cell is the fixed charge at the macroion and zero at the cell
wall (Q(a) = Q_M, Q(R_cell) = 0) and, with counterions only, rises outward;
every ion of the cell is counted once and a bin's charge is its count times
the ions' valence.  The library's host-side bhmc_radial_profiles gives the
oracle's profiles on the same counts."""
import numpy as np
import pytest

import oracle
from paper_1305_1825_gb300 import bhmc
from paper_1305_1825_gb300 import workloads as W


def _shell(n, a, b, seed):
    """n ions uniform in the shell a <= r < b (counts made by the oracle)."""
    rng = np.random.default_rng(seed)
    r = (rng.uniform(a ** 3, b ** 3, n)) ** (1.0 / 3.0)
    v = rng.normal(size=(n, 3))
    x = r[:, None] * v / np.linalg.norm(v, axis=1)[:, None]
    params = W.base_params(root_lo=(-64.0,) * 3, root_side=128.0)
    return oracle.System(params, np.ones(n), x, n, 0)


def test_uniform_shell_gives_flat_rdf():
    a, b, nb = 10.0, 50.0, 20
    s = _shell(200000, a, b, 3)
    counts, charge = s.radial_counts(nb, a, b)
    assert counts.sum() == 200000 and np.array_equal(charge, counts.astype(float))
    _, g, _, _ = oracle.radial_profiles(counts, charge, a, b, 1)
    assert abs(g.sum() - 1.0) < 1e-12
    assert np.abs(g * nb - 1.0).max() < 0.03


def test_neutral_double_layer_integrated_charge():
    wl = W.edl_hard(n=500, seed=11)
    n = wl["n_mobile"]
    s = oracle.System(wl["params"], wl["q"], wl["xyz"], n, wl["n_fixed"])
    a, rcell, nb = 30.0, 80.0, 25
    counts, charge = s.radial_counts(nb, a, rcell)
    centres, g, edges, Q = oracle.radial_profiles(counts, charge, a, rcell, 1, q_fixed=float(wl["q"][n]))
    assert counts.sum() == n                        # every ion lies inside the cell, counted once
    assert np.array_equal(charge, 2.0 * counts)     # valence 2
    assert abs(Q[-1]) < 1e-9                        # Q(R_cell) = 0
    assert Q[0] == wl["q"][n] + charge[0]            # Q at the first outer edge
    assert np.all(np.diff(Q) >= 0)                   # counterions only: Q rises outward
    assert np.allclose(edges[-1], rcell) and np.all(np.diff(centres) > 0)


def test_library_profiles_equal_oracle():
    wl = W.edl_hard(n=500, seed=12)
    n = wl["n_mobile"]
    s = oracle.System(wl["params"], wl["q"], wl["xyz"], n, wl["n_fixed"])
    counts, charge = s.radial_counts(30, 32.0, 78.0)
    counts, charge = 7 * counts, 7 * charge  # seven identical samples
    want = oracle.radial_profiles(counts, charge, 32.0, 78.0, 7, q_fixed=-1000.0)
    got = bhmc.radial_profiles(counts, charge, 32.0, 78.0, samples=7, q_fixed=-1000.0)
    for a, b in zip(got, want):
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-12)
    with pytest.raises(bhmc.BhmcError):
        bhmc.radial_profiles(counts, charge, 32.0, 78.0, samples=0)
