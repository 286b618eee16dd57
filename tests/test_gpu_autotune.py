"""The autotuner runs on the GPU and returns a timed, accuracy-checked choice."""
import pytest

from paper_1305_1825_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_autotune_small():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1825_gb300 import autotune
    systems = W.batch(sizes=[2060, 3000, 2500, 4000])
    res = autotune.autotune(systems, [1, 2, 3, 4], C_values=(4, 8), warps_values=(2, 8), moves=20)
    assert len(res["results"]) == 2 * 2 * 2
    assert all(r["moves_per_s"] > 0 for r in res["results"])
    best = res["best"]
    assert res["accuracy"][best["C"]]["E"] <= res["accuracy_bound_E"]
    # dE (a difference of two potentials) at theta = 0.5, p = 4: a few percent at most
    assert 0.0 < res["accuracy"][8]["E"] < 0.05


def test_tune_n0_small():
    """N_0(p) by timing returns a rate for every candidate and picks one of them."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1825_gb300 import autotune
    systems = [W.edl_hard(n=300, seed=90 + k) for k in range(4)]
    res = autotune.tune_n0(systems, [1, 2, 3, 4], p_values=(1, 4), n0_values=(0, 8), moves=40)
    assert set(res) == {1, 4}
    for p in (1, 4):
        assert set(res[p]["rates"]) == {0, 8} and all(v > 0 for v in res[p]["rates"].values())
        assert res[p]["chosen"] in (0, 8)

