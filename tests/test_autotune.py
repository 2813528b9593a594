"""Autotuner: candidate generation (CPU) and a small tuning run (GPU)."""
import numpy as np
import pytest

import paper_2402_06415_gb300 as ising
from paper_2402_06415_gb300 import autotune


def test_candidates_are_valid_shapes():
    for L in (256, 2048, 16384):
        Wc = ising.ising_words_per_row(L)
        cands = autotune.candidates(L)
        assert cands[0]["kernel"] == ising.ISING_KERNEL_HALF
        for c in cands[1:]:
            assert Wc % c["tile_words"] == 0 and c["tile_words"] % 4 == 0
            assert 1 <= c["k"] <= 8 and 1 <= c["tile_rows"] <= L
    assert len(autotune.candidates(130)) == 1  # ragged rows: half-sweep kernel only


@pytest.mark.gpu
def test_tune_small_lattice(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    monkeypatch.setenv("ISING_TUNE_CACHE", str(tmp_path / "tune.json"))
    L = 2048
    cands = [c for c in autotune.candidates(L) if c["k"] <= 2][:6]
    res = autotune.tune(L, sweeps=4, reps=1, cands=cands)
    assert res["flips_per_ns"] > 0 and res["config"] in [
        {k: c[k] for k in ("kernel", "k", "tile_rows", "tile_words")} for c in cands]
    # cached: a second call returns the same answer without timing
    assert autotune.tune(L, cands=cands) == res
    # the winner and the runner-up give identical chains
    outs = []
    for row in res["table"][:2]:
        with ising.Lattice(L, 0.44, ising.ISING_LAYOUT_BITS, seed=5) as lat:
            lat.set_kernel(row["kernel"], row["k"], row["tile_rows"], row["tile_words"])
            lat.sweep(6, 1)
            outs.append((lat.bits().copy(), lat.series()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1][0], outs[1][1][0])
