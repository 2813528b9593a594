"""The staged proposal's schedule exported by the C-ABI (host code, no GPU)
equals the oracle's, which is built independently from the same definition
(oracle/staged.py) and pinned in test_oracle_staged.py."""
import numpy as np
import pytest

from oracle import staged
import paper_2402_06415_gb300 as ising


@pytest.mark.parametrize("B", [2, 4, 6, 8, 10, 12, 14, 16])
def test_schedule_matches_oracle(B):
    so, ex = ising.ising_proposal_schedule(B, ising.ISING_PROPOSAL_STAGED)
    st = staged.schedule(B)
    assert list(ex) == [1 if kind == "exact" else 0 for kind, _ in st]
    want = np.zeros((B, B), dtype=int)
    for k, (_, sites) in enumerate(st):
        for (i, j) in sites:
            want[i, j] = k
    assert np.array_equal(so, want)


def test_oneshot_schedule_is_one_network_stage():
    so, ex = ising.ising_proposal_schedule(16, ising.ISING_PROPOSAL_ONESHOT)
    assert list(ex) == [0] and not so.any()


@pytest.mark.parametrize("B, kind", [(3, 1), (0, 1), (18, 1), (16, 2)])
def test_schedule_rejects_bad_arguments(B, kind):
    with pytest.raises(ising.IsingError):
        ising.ising_proposal_schedule(B, kind)
