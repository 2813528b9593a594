"""The allocation-free sweep entry point against the regular one (GPU).

ising_sweep_bits_noalloc serves callers that may not allocate device memory
while they run (their allocator owns the device, or an allocation would stall
a real-time stream): they pass their own lattice and output buffers and the
library uses a static scratch array instead of cudaMalloc.  Here it must give
the same spins and E/M records, bit for bit, as ising_sweep with the tiled
kernel, on two calls in a row (the second continuing the chain of the first),
and it must refuse lattices larger than its static scratch.

This file is collected last on purpose; it also passes when run on its own.
"""
import numpy as np
import pytest

import paper_2402_06415_gb300 as ising

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ising.lib()
    return torch


def _reference(L, beta, seed, n1, n2, k):
    """Regular entry point: lattice after n1 and after n1 + n2 sweeps, records."""
    with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS) as lat:
        lat.set_kernel(ising.ISING_KERNEL_TILED, k, max(L // 64, 1), 4)
        lat.seed(seed)
        start = lat.bits().copy()
        lat.sweep(n1, 1)
        mid = lat.bits().copy()
        E1, M1 = lat.series(n1)
        lat.sweep(n2, 1)
        end = lat.bits().copy()
        E2, M2 = lat.series(n2)
    return start, mid, end, (E1, M1), (E2, M2)


# L = 256 / 512 / 1024 take 4- / 8- / 16-word tiles, L = 2048 the 32-word tiles,
# L = 8192 the largest lattice the static scratch holds
@pytest.mark.parametrize("L,k,n1,n2", [(256, 2, 7, 5), (512, 3, 7, 5), (1024, 1, 7, 5),
                                       (2048, 2, 3, 3), (8192, 2, 3, 3)])
def test_noalloc_matches_regular_two_calls(torch_cuda, L, k, n1, n2):
    torch = torch_cuda
    beta, seed = 0.4406868, 21
    start, mid, end, (E1, M1), (E2, M2) = _reference(L, beta, seed, n1, n2, k)

    Wc = ising.ising_words_per_row(L)
    dev = torch.from_numpy(start.view(np.int32)).cuda()
    out = torch.empty_like(dev)
    E = torch.zeros(n1, dtype=torch.int64, device="cuda")
    M = torch.zeros(n1, dtype=torch.int64, device="cuda")
    E2d = torch.zeros(n2, dtype=torch.int64, device="cuda")
    M2d = torch.zeros(n2, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    assert dev.shape == (2, L, Wc)

    # first call: sweeps 0 .. n1-1, dev -> out
    ising.ising_sweep_bits_noalloc(dev, out, L, beta, seed, 0, 0, n1, 1, E, M, k, stream)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), mid)
    assert np.array_equal(E.cpu().numpy(), E1) and np.array_equal(M.cpu().numpy(), M1)

    # second call continues the chain in place: sweeps n1 .. n1+n2-1 (every
    # buffer is allocated and the device idle before the free-memory snapshot)
    torch.cuda.synchronize()
    free_before_second = torch.cuda.mem_get_info()[0]
    ising.ising_sweep_bits_noalloc(out, out, L, beta, seed, 0, n1, n2, 1, E2d, M2d, k, stream)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), end)
    assert np.array_equal(E2d.cpu().numpy(), E2) and np.array_equal(M2d.cpu().numpy(), M2)
    # no device memory was taken by the second call
    assert torch.cuda.mem_get_info()[0] == free_before_second


def test_noalloc_record_slots_with_offset_start(torch_cuda):
    """measure_every = 3 from sweep 7: records of sweeps 8, 11, 14, ... land in
    slots 0, 1, 2, ... exactly as the regular entry point records them."""
    torch = torch_cuda
    L, beta, seed, k, t0, n, every = 512, 0.4406868, 5, 2, 7, 11, 3
    with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS) as lat:
        lat.set_kernel(ising.ISING_KERNEL_TILED, k, L // 64, 4)
        lat.seed(seed)
        lat.sweep(t0, 0)
        start = lat.bits().copy()
        lat.sweep(n, every)
        end = lat.bits().copy()
        n_rec = sum(1 for t in range(t0, t0 + n) if (t + 1) % every == 0)
        Er, Mr = lat.series(n_rec)
    dev = torch.from_numpy(start.view(np.int32)).cuda()
    out = torch.empty_like(dev)
    E = torch.zeros(n_rec, dtype=torch.int64, device="cuda")
    M = torch.zeros(n_rec, dtype=torch.int64, device="cuda")
    ising.ising_sweep_bits_noalloc(dev, out, L, beta, seed, 0, t0, n, every, E, M, k,
                                   torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), end)
    assert np.array_equal(E.cpu().numpy(), Er) and np.array_equal(M.cpu().numpy(), Mr)


def test_noalloc_refuses_oversized_lattice(torch_cuda):
    torch = torch_cuda
    L = 16384
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sweep_bits_noalloc(dummy, dummy, L, 0.44, 1, 0, 0, 1, 0, None, None, 2)
    assert e.value.status == ising.ISING_EINVAL
    assert "at most 8192" in e.value.message
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sweep_bits_noalloc(dummy, dummy, 256, 0.44, 1, 0, 0, 5000, 1, dummy, dummy, 2)
    assert "4096 records" in e.value.message
