"""Host-side conversion of radial counts into the RDF and the integrated charge
of Sec. 4 (Fig. 6), on counts made here with numpy (no GPU): a uniform density
in a shell gives a flat g, the bins of g sum to one, and the integrated charge
of an electroneutral cell is the fixed charge at the macroion and zero at the
cell wall (Q(a) = Q_M, Q(R_cell) = 0)."""
import numpy as np

from paper_1305_1825_gb300 import bhmc
from paper_1305_1825_gb300 import workloads as W


def _counts(r, q, r_lo, r_hi, nbins):
    w = (r_hi - r_lo) / nbins
    k = np.floor((r - r_lo) / w).astype(int)
    ok = (k >= 0) & (k < nbins)
    return np.bincount(k[ok], minlength=nbins).astype(np.int64), np.bincount(k[ok], weights=q[ok], minlength=nbins)


def test_uniform_shell_gives_flat_rdf():
    rng = np.random.default_rng(3)
    a, b, n = 10.0, 50.0, 400000
    r = (rng.uniform(a ** 3, b ** 3, n)) ** (1.0 / 3.0)
    counts, charge = _counts(r, np.ones(n), a, b, 20)
    _, g, _, _ = bhmc.radial_profiles(counts, charge, a, b, samples=1)
    assert abs(g.sum() - 1.0) < 1e-12
    assert np.abs(g * 20 - 1.0).max() < 0.03


def test_neutral_double_layer_integrated_charge():
    wl = W.edl_hard(n=500, seed=11)
    n = wl["n_mobile"]
    r = np.linalg.norm(wl["xyz"][:n], axis=1)
    q = wl["q"][:n]
    a, rcell = 30.0, 80.0
    counts, charge = _counts(r, q, a, rcell, 25)
    centres, g, edges, Q = bhmc.radial_profiles(counts, charge, a, rcell, samples=1, q_fixed=float(wl["q"][n]))
    assert counts.sum() == n                      # every ion lies inside the cell
    assert abs(Q[-1]) < 1e-9                      # Q(R_cell) = 0
    assert Q[0] == wl["q"][n] + charge[0]          # Q at the first outer edge
    assert np.all(np.diff(Q) >= 0)                 # counterions only: Q rises outward
    assert np.allclose(edges[-1], rcell) and np.all(np.diff(centres) > 0)
