"""The single-kernel bench workloads that the profiles' commands run
(`bench.py --workload sw_step | staged_pass | train | xy_step`), at small sizes:
each prints one JSON line with the contract's keys and a sane value.
"""
import json

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bench():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench as b
    return b


def _line(bench, capsys, argv):
    assert bench.main(argv) == 0
    out = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(out) == 1
    d = json.loads(out[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "config"):
        assert k in d, k
    assert d["value"] > 0
    return d


def test_sw_step_workload(bench, capsys):
    d = _line(bench, capsys, ["--workload", "sw_step", "--steps", "2", "--warmup", "3", "--sw-L", "2048"])
    assert d["unit"] == "ms/step" and d["higher_is_better"] is False
    assert d["site_updates_per_ns"] > 0


def test_staged_pass_workload_both_engines(bench, capsys):
    for engine in ("mma_sync", "tcgen05"):
        d = _line(bench, capsys, ["--workload", "staged_pass", "--steps", "2", "--warmup", "3", "--pass-L", "64",
                                  "--nn-engine", engine])
        assert d["config"]["engine"] == engine and d["squares_per_pass"] == 16


def test_train_workload(bench, capsys):
    d = _line(bench, capsys, ["--workload", "train", "--steps", "2", "--warmup", "3"])
    assert set(d["kernels"]) == {"fp32", "bf16_tc"}
    assert d["kernels"]["bf16_tc"]["samples_per_s"] > d["kernels"]["fp32"]["samples_per_s"]


def test_xy_step_workload(bench, capsys):
    for prec in ("32", "64"):
        d = _line(bench, capsys, ["--workload", "xy_step", "--steps", "2", "--warmup", "3", "--xy-L", "256",
                                  "--xy-precision", prec])
        assert d["dtype"] == "f" + prec
