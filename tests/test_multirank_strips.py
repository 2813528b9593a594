"""Row-strip decomposition of one lattice over CPU ranks (gloo), the exchange a
multi-GPU single-lattice sweep would need: before every half sweep each rank
sends its first and last owned rows to its neighbours (periodic in y) and
receives their edge rows as halos; each rank then updates only its own rows.
Because every site's uniform is keyed by its global (group, sweep) counter, the
gathered lattice must equal the single-process oracle bit for bit, for any
number of ranks and any strip boundaries (even or odd row counts).

The oracle's half sweep runs on a full-size working copy per rank; rows the rank
does not own hold stale values and are never read back, so the test exercises
exactly which rows must be current (own rows plus one halo row on each side).
"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle


def _strips(L, world):
    cuts = [round(k * L / world) + (k % 2 if 0 < k < world else 0) for k in range(world + 1)]
    cuts[-1] = L
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def _worker(rank, world, port, L, beta, seed, n, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        y0, y1 = _strips(L, world)[rank]
        s = oracle.init(L, seed)                       # every rank starts from the same seeded state
        up, down = (rank - 1) % world, (rank + 1) % world
        for t in range(n):
            for c in range(2):
                # halo exchange: own edge rows out, neighbours' edge rows in
                first = torch.from_numpy(s[y0].copy())
                last = torch.from_numpy(s[y1 - 1].copy())
                halo_up = torch.empty(L, dtype=torch.int8)
                halo_dn = torch.empty(L, dtype=torch.int8)
                # tags keep the two messages apart when up == down (two ranks):
                # 1 = a first row (the upper neighbour's lower halo), 2 = a last row
                reqs = [dist.isend(first, up, tag=1), dist.isend(last, down, tag=2),
                        dist.irecv(halo_up, up, tag=2), dist.irecv(halo_dn, down, tag=1)]
                for r in reqs:
                    r.wait()
                s[(y0 - 1) % L] = halo_up.numpy()
                s[y1 % L] = halo_dn.numpy()
                # rows outside [y0 - 1, y1] are stale on purpose: poison them
                mask = np.ones(L, dtype=bool)
                mask[[(y0 - 1) % L, y1 % L]] = False
                mask[y0:y1] = False
                s[mask] = 1
                oracle.half_sweep(s, beta, seed, 0, t, c)
        out[rank] = (y0, y1, s[y0:y1].tobytes())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,L", [(2, 16), (3, 18), (4, 34)])
def test_strip_decomposition_bit_exact(world, L):
    beta, seed, n = 0.4406868, 9, 4
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 30500 + (os.getpid() % 1500) + world
        mp.start_processes(_worker, args=(world, port, L, beta, seed, n, out), nprocs=world,
                           start_method="spawn")
        res = dict(out)
    got = np.zeros((L, L), dtype=np.int8)
    for rank in range(world):
        y0, y1, rows = res[rank]
        got[y0:y1] = np.frombuffer(rows, dtype=np.int8).reshape(y1 - y0, L)
    ref = oracle.init(L, seed)
    oracle.sweep(ref, beta, seed, n)
    assert np.array_equal(got, ref)


def test_strip_boundaries_cover_the_lattice():
    for world in range(1, 6):
        for L in (4, 16, 18, 34, 64):
            if world > L // 2:
                continue
            st = _strips(L, world)
            assert st[0][0] == 0 and st[-1][1] == L
            assert all(a < b for a, b in st) and all(st[k][1] == st[k + 1][0] for k in range(world - 1))
