"""Fixed-point XY sweep (operand-precision study) on the GPU against the CPU
oracle: integer arithmetic throughout, so angles, accepted counts and the
(E2, Mx, My) records are bit-exact."""
import numpy as np
import pytest

import oracle
import paper_2402_06415_gb300 as ising

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    ising.lib()


@pytest.mark.parametrize("qp", [False, True])
@pytest.mark.parametrize("F", [6, 8, 12, 16])
@pytest.mark.parametrize("L", [2, 4, 6, 16, 64, 130])
@pytest.mark.parametrize("beta", [0.3, 1.0 / 0.85, 3.0])
def test_xyfix_bit_exact(qp, F, L, beta):
    seed, n = 900 + L + F, 6
    k = oracle.xyfix_init(L, F, seed)
    with ising.XYFix(L, beta, F, seed=seed, quantise_p=qp) as x:
        assert np.array_equal(x.angles(), k)
        x.sweep(n, 1)
        got = x.angles()
        E2, Mx, My = x.series(n)
        acc_gpu = x.info()["accepted"]
    acc, E2_ref = oracle.xyfix_sweep(k, F, beta, seed, n, qp=qp)
    assert np.array_equal(got, k)
    assert acc_gpu == int(acc.sum())
    assert np.array_equal(E2, E2_ref)
    e, mx, my = oracle.xyfix_observables(k, F)
    assert (Mx[-1], My[-1]) == (mx, my)


def test_xyfix_paper_size_long_chain_and_resume():
    """L = 32 at T = 0.85 (the paper's Tab. S3 setting), F = 8, 3000 sweeps in
    two calls, then a set_angles round trip."""
    L, F, beta, seed = 32, 8, 1.0 / 0.85, 4
    k = oracle.xyfix_init(L, F, seed)
    with ising.XYFix(L, beta, F, seed=seed) as x:
        x.sweep(1000)
        x.sweep(2000, 1)
        got = x.angles()
        E2, _, _ = x.series(2000)
    _, E_ref = oracle.xyfix_sweep(k, F, beta, seed, 3000)
    assert np.array_equal(got, k)
    assert np.array_equal(E2, E_ref[1000:])
    with ising.XYFix(L, beta, F, seed=seed) as x:
        x.set_angles(got)
        assert np.array_equal(x.angles(), got)
        bad = got.copy()
        bad[0, 0] = x.info()["K"]
        with pytest.raises(ising.IsingError):
            x.set_angles(bad)


def test_xyfix_rejects_bad_arguments():
    with pytest.raises(ising.IsingError):
        ising.XYFix(8, 1.0, 5)
    with pytest.raises(ising.IsingError):
        ising.XYFix(8, 1.0, 17)
    with pytest.raises(ising.IsingError):
        ising.XYFix(7, 1.0, 8)
    with pytest.raises(ising.IsingError):
        lib = ising.lib()
        import ctypes
        out = ctypes.c_void_p()
        ising._binding._check(lib.ising_xyfix_create(ctypes.byref(out), 8, 1.0, 8, 2, None))


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("L", [4, 32, 64, 130, 512])
def test_xyfix_kernel_modes_bit_exact(mode, L):
    F, beta, seed, n = 12, 1.0 / 0.85, 77 + L, 7
    k = oracle.xyfix_init(L, F, seed)
    acc, E_ref = oracle.xyfix_sweep(k, F, beta, seed, n)
    with ising.XYFix(L, beta, F, seed=seed) as x:
        x.set_mode(mode)
        x.sweep(3, 3)
        x.sweep(4, 1)
        got = x.angles()
        E2, _, _ = x.series(5)
        info = x.info()
    assert np.array_equal(got, k)
    assert info["accepted"] == int(acc.sum())
    assert np.array_equal(E2, np.concatenate([E_ref[2:3], E_ref[3:]]))
    assert info["launches"] == (2 if mode == 2 else 2 * n + 1 + 4)
