"""Which block runs which replica does not change any chain.

The batched kernel places replicas on SMs in one of two ways: with at most two
replicas per SM (more replicas than SMs, at most twice as many) the first block
on each SM takes the next-largest replica and the second block the
size-complement of its sibling's, the largest running alone; otherwise blocks
take replicas largest first from a shared cursor.  Either way every replica
must run exactly once, for all its moves, and each chain must equal the
oracle's chain of that replica (its Philox counter carries the replica index,
not the block)."""
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


def _sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("regime", ["fewer-than-SMs", "pairs-per-SM", "more-than-two-per-SM"])
def test_every_replica_runs_once_and_matches_oracle(bh, oracle_mod, regime):
    sms = _sms()
    n_rep = {"fewer-than-SMs": sms // 2, "pairs-per-SM": sms + sms // 3,
             "more-than-two-per-SM": 2 * sms + 40}[regime]
    rng = np.random.default_rng(n_rep)
    sizes = [int(v) for v in rng.integers(120, 400, n_rep)]
    systems = [W.plain(n=sizes[r], seed=500 + r) for r in range(n_rep)]
    batch = bh.Batch(systems, warps=8, layout=bh.LAYOUT_AOS)
    seeds = [9000 + r for r in range(n_rep)]
    n_moves = 60
    stats, recs = batch.step_mc(n_moves, 1.0, seeds, records=True)
    assert all(s["moves"] == n_moves for s in stats)
    for r in list(rng.choice(n_rep, 5, replace=False)) + [int(np.argmax(sizes)), int(np.argmin(sizes))]:
        ref = oracle_mod.System(systems[r]["params"], systems[r]["q"], systems[r]["xyz"], sizes[r], 0)
        orec = ref.mc_run(seeds[r], n_moves, replica=int(r))
        for t in range(n_moves):
            assert recs[r]["i"][t] == orec["i"][t] and np.array_equal(recs[r]["r_new"][t], orec["r_new"][t])
            if recs[r]["outcome"][t] != orec["outcome"][t]:
                assert orec["flagged"][t] or recs[r]["flagged"][t]
                break
    batch.close()
