"""The C-ABI library loads, exports every declared entry point, and rejects bad
arguments before touching a GPU (CPU only: no compute calls)."""
import os
import re

import pytest

import paper_2402_06415_gb300 as ising

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ising_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = ising.lib()
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers exactly the declared set
    assert set(ising.EXPORTED) == declared


def test_library_loaded_from_tree():
    lib = ising.lib()
    assert os.path.dirname(os.path.abspath(lib._name)).startswith(ROOT)


@pytest.mark.parametrize("L", [0, 2, 3, 5, 65538, -4])
def test_create_rejects_bad_size(L):
    with pytest.raises(ising.IsingError) as e:
        ising.ising_create(L, 0.4)
    assert e.value.status == ising.ISING_EINVAL
    assert "L must be even" in e.value.message


@pytest.mark.parametrize("beta", [0.0, -1.0, float("nan"), float("inf")])
def test_create_rejects_bad_beta(beta):
    with pytest.raises(ising.IsingError) as e:
        ising.ising_create(64, beta)
    assert e.value.status == ising.ISING_EINVAL


def test_create_rejects_bad_layout():
    with pytest.raises(ising.IsingError) as e:
        ising.ising_create(64, 0.4, layout=7)
    assert e.value.status == ising.ISING_EINVAL


def test_null_context_calls_fail_cleanly():
    lib = ising.lib()
    assert lib.ising_sweep(None, 1, 1) == ising.ISING_EINVAL
    assert b"null context" in lib.ising_last_error()
    assert lib.ising_destroy(None) == ising.ISING_OK


def test_thresholds_match_closed_form():
    from oracle.closed_forms import thresholds_exact

    for beta in [0.3, 0.35, 0.4, 0.4406868, 0.44068679350977147, 0.5, 0.6, 2.0]:
        t4, t8 = ising.ising_thresholds(beta)
        assert t4 == thresholds_exact(beta, 4)
        assert t8 == thresholds_exact(beta, 8)


def test_words_per_row():
    assert ising.ising_words_per_row(4) == 1
    assert ising.ising_words_per_row(64) == 1
    assert ising.ising_words_per_row(66) == 2
    assert ising.ising_words_per_row(16384) == 256


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    """A missing shared library raises instead of silently computing on the CPU."""
    from paper_2402_06415_gb300 import _binding

    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_binding, "LIB_PATH", str(tmp_path / "missing.so"))
    import paper_2402_06415_gb300.build as b

    monkeypatch.setattr(b, "build", lambda *a, **k: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        _binding.lib()
