"""Staged block proposal on the GPU against the CPU reference (oracle/staged.py).

* The C-ABI schedule equals the oracle's (also checked without a GPU in
  test_staged_schedule.py).
* Per-stage logits of the BF16 tensor-core inference match the float64
  reference with the same bf16-rounded weights at every stage's sites: network
  stages to 1e-2 relative (floor 1), exact stages to 1e-5 (FP32 arithmetic).
* The teacher-forced ln q of each window matches the reference within the
  bound that the logit tolerance implies (|d ln sigma(l) / dl| <= 1 per site).
* FP32 loss and gradients of the staged training objective match the float64
  reference element by element.
* Block passes alone with the staged proposal sample the Boltzmann
  distribution: exact <E>, <M^2> of a 4 x 4 lattice (2 x 2 blocks) and Kaufman's
  <E> on 8 x 8 (4 x 4 blocks), within 3 sigma.
* A briefly trained network with 16 x 16 staged blocks at beta_c accepts
  proposals (acceptance asserted > 0), and sweeps + passes keep the plain
  chain's <E> and <|M|> within 3 sigma on L = 64.
* The batched staged pass equals the single-lattice staged pass bit for bit.
* Both engines of the second convolution (mma.sync, tcgen05) pass the logit,
  ln q and chain tests; their logits agree to FP32 accumulation order.
"""
import numpy as np
import pytest

from oracle import cnn, exact, staged
from oracle.closed_forms import kaufman_energy
import paper_2402_06415_gb300 as ising
from paper_2402_06415_gb300 import learned, stats

pytestmark = pytest.mark.gpu

STAGED = ising.ISING_PROPOSAL_STAGED
BETA_C = 0.4406868
ENGINES = [ising.ISING_NN_ENGINE_MMA_SYNC, ising.ISING_NN_ENGINE_TCGEN05]


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    ising.lib()
    return t


def _windows(L, n, block, seed, beta=BETA_C, sweeps=60):
    rng = np.random.default_rng(seed)
    with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS, seed=seed) as lat:
        lat.sweep(sweeps, 0)
        s = lat.spins()
    w = learned.extract_windows(s, n, block, rng)
    w[:, 0, 0] = w[:, 0, -1] = w[:, -1, 0] = w[:, -1, -1] = 0  # corners are never read
    return w


def _params(seed, scale=2.0):
    p32 = learned.init_params(seed=seed, scale=scale)
    rng = np.random.default_rng(seed + 1)
    for k in p32:
        if k.startswith("b"):
            p32[k] = (0.1 * rng.standard_normal(p32[k].shape)).astype(np.float32)
    return p32, {k: cnn.bf16_round(v.astype(np.float64)) for k, v in p32.items()}


def test_schedule_matches_oracle():
    for B in (2, 4, 8, 16):
        so, ex = ising.ising_proposal_schedule(B, STAGED)
        st = staged.schedule(B)
        assert list(ex) == [1 if kind == "exact" else 0 for kind, _ in st]
        for k, (_, sites) in enumerate(st):
            for (i, j) in sites:
                assert so[i, j] == k


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("block", [16, 8, 4])
def test_stage_logits_match_reference(torch, block, engine):
    p32, pref = _params(3)
    wins = _windows(64, 24, block, seed=5)
    st = staged.schedule(block)
    d = torch.from_numpy(wins).cuda()
    out = torch.zeros((len(wins), block, block), dtype=torch.float32, device="cuda")
    with learned.Trainer(block, params=p32, proposal=STAGED) as tr:
        ising.ising_nn_set_engine(tr.h, engine)
        for k, (kind, sites) in enumerate(st):
            ising.ising_nn_stage_logits(tr.h, d, len(wins), k, BETA_C, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.float64)
            want = staged.stage_logits(pref, wins.astype(np.int64), BETA_C, block, st, k)
            m = np.zeros((block, block), dtype=bool)
            for (i, j) in sites:
                m[i, j] = True
            err = np.abs(got - want)[:, m] / np.maximum(np.abs(want)[:, m], 1.0)
            tol = 1e-2 if kind == "net" else 1e-5
            assert err.max() < tol, (k, kind, err.max())
            assert np.all(got[:, ~m] == 0.0)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("block", [16, 4])
def test_log_q_matches_reference(torch, block, engine):
    p32, pref = _params(7)
    wins = _windows(64, 16, block, seed=8)
    st = staged.schedule(block)
    with learned.Trainer(block, params=p32, proposal=STAGED) as tr:
        ising.ising_nn_set_engine(tr.h, engine)
        d = torch.from_numpy(wins).cuda()
        out = torch.zeros(len(wins), dtype=torch.float32, device="cuda")
        ising.ising_nn_log_q(tr.h, d, len(wins), BETA_C, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
    w64 = wins.astype(np.int64)
    want = staged.log_q_many(pref, w64, BETA_C, block, st)
    # bound implied by the logit tolerance: sum over sites of 1e-2 max(|l|, 1)
    # (network stages) and 1e-5 max(|l|, 1) (exact stages), plus FP32 rounding
    bound = np.zeros(len(wins))
    for k, (kind, sites) in enumerate(st):
        lg = staged.stage_logits(pref, w64, BETA_C, block, st, k)
        rel = 1e-2 if kind == "net" else 1e-5
        for (i, j) in sites:
            bound += rel * np.maximum(np.abs(lg[:, i, j]), 1.0)
    bound += 1e-5 * np.abs(want) + 1e-3
    assert np.all(np.abs(got - want) <= bound), (got - want, bound)
    assert np.all(want < 0)


@pytest.mark.parametrize("proposal", [ising.ISING_PROPOSAL_ONESHOT, STAGED])
def test_loss_and_gradients_elementwise(torch, proposal):
    block = 4
    p32 = learned.init_params(seed=6)
    for k in p32:  # avoid exact ReLU kinks at 0 and give the biases some weight
        p32[k] = p32[k] + (0.05 * np.random.default_rng(60).standard_normal(p32[k].shape)).astype(np.float32)
    wins = _windows(32, 24, block, seed=7)
    with learned.Trainer(block, params=p32, proposal=proposal) as tr:
        d = torch.from_numpy(wins).cuda()
        loss, g = ising.ising_nn_loss_grad(tr.h, d, len(wins))
    p64 = {k: v.astype(np.float64) for k, v in p32.items()}
    if proposal == STAGED:
        want_loss, want_g = staged.staged_loss_and_grads(p64, wins, block)
    else:
        F = block + 2
        want_loss, want_g = cnn.loss_and_grads(p64, staged.stage_frame(wins, staged.ring_mask(block)),
                                               wins[:, 1:F - 1, 1:F - 1].astype(np.float64))
    assert abs(loss - want_loss) < 1e-5 * abs(want_loss)
    G = ising.nn_unflatten(g)
    for k in want_g:
        ref = want_g[k]
        scale = 1e-2 * np.abs(ref).max()
        err = np.abs(G[k] - ref) / np.maximum(np.abs(ref), scale)
        assert err.max() < 1e-4, (k, err.max())


@pytest.mark.parametrize("proposal,block", [(ising.ISING_PROPOSAL_ONESHOT, 4), (STAGED, 4), (STAGED, 16)])
def test_tensor_core_gradients_elementwise(torch, proposal, block):
    """The BF16 tensor-core training kernel, element by element, against the
    float64 objective whose 32 -> 32 convolution operands are rounded to BF16
    at the same points (oracle/staged.py, bf16_operands): what is left is FP32
    accumulation order and the odd operand rounded from an FP32 instead of a
    float64 value, so every element within 5e-3 of max(|ref|, a tenth of the
    tensor's largest element), the loss within 1e-4.  Against the exact
    objective the layer-3 gradients (one rounded operand) stay within 2e-2 of
    the tensor's largest element; the layer-2 and layer-1 gradients also see
    ReLU masks that the rounding flips near zero (oracle pin in
    test_oracle_staged.py) and are checked against the exact objective only to
    0.15 of the largest element."""
    p32 = learned.init_params(seed=6)
    for k in p32:
        p32[k] = p32[k] + (0.05 * np.random.default_rng(60).standard_normal(p32[k].shape)).astype(np.float32)
    wins = _windows(64, 24, block, seed=7)
    with learned.Trainer(block, params=p32, proposal=proposal) as tr:
        ising.ising_nn_set_train_precision(tr.h, ising.ISING_NN_TRAIN_BF16_TC)
        d = torch.from_numpy(wins).cuda()
        loss, g = ising.ising_nn_loss_grad(tr.h, d, len(wins))
        with pytest.raises(ising.IsingError):
            ising.ising_nn_set_train_precision(tr.h, 2)
    p64 = {k: v.astype(np.float64) for k, v in p32.items()}
    st = None if proposal == STAGED else [("net", [(i, j) for i in range(block) for j in range(block)])]
    emu_loss, emu_g = staged.staged_loss_and_grads(p64, wins, block, st, bf16_operands=True)
    ex_loss, ex_g = staged.staged_loss_and_grads(p64, wins, block, st)
    assert abs(loss - emu_loss) < 1e-4 * abs(emu_loss), (loss, emu_loss)
    G = ising.nn_unflatten(g)
    for k in emu_g:
        ref = emu_g[k]
        scale = 0.1 * np.abs(ref).max()
        err = np.abs(G[k] - ref) / np.maximum(np.abs(ref), scale)
        assert err.max() < 5e-3, (k, err.max())
        assert np.abs(ref).max() > 0
    for k in ex_g:
        ref = ex_g[k]
        d = np.abs(G[k] - ref).max() / np.abs(ref).max()
        assert d < (2e-2 if k in ("W3", "b3") else 0.15), (k, d)


def test_tensor_core_training_lowers_loss_and_accepts(torch):
    """Training the staged 16 x 16 proposal with the tensor-core kernel lowers
    the loss like the FP32 kernel, and the trained network's block moves are
    accepted on a beta_c lattice."""
    wins = learned.generate_windows([64, 128], BETA_C, 3072, 16, seed=71, thermalise=2000, thin=40)
    with learned.Trainer(16, seed=72, proposal=STAGED) as tr:
        ising.ising_nn_set_train_precision(tr.h, ising.ISING_NN_TRAIN_BF16_TC)
        losses = tr.fit(wins, epochs=2, batch=256, lr=2e-3, seed=73)
        blob = tr.blob()
    assert np.mean(losses[-5:]) < 0.9 * np.mean(losses[:5])
    with ising.Lattice(64, BETA_C, ising.ISING_LAYOUT_BITS, seed=74) as lat:
        ising.ising_nn_load(lat.ctx, blob)
        ising.ising_set_proposal(lat.ctx, STAGED)
        lat.sweep(2000, 0)
        ising.ising_block_pass(lat.ctx, 200, 16)
        p, a = ising.ising_block_stats(lat.ctx)
    assert a > 0.01 * p, (a, p)


def test_adam_and_bf16_export_match_reference(torch):
    """Three Adam steps with the oracle's gradients on both sides: FP32 master
    weights vs the float64 Adam, and the BF16 blob = bf16(master weights)."""
    block = 4
    p32 = learned.init_params(seed=40)
    p64 = {k: v.astype(np.float64) for k, v in p32.items()}
    m = {k: np.zeros_like(v) for k, v in p64.items()}
    v = {k: np.zeros_like(x) for k, x in p64.items()}
    wins = _windows(32, 16, block, seed=41)
    lr = 3e-3
    with learned.Trainer(block, params=p32) as tr:
        for t in (1, 2, 3):
            _, g = staged.staged_loss_and_grads(p64, wins[5 * t:5 * t + 5], block,
                                                [("net", [(i, j) for i in range(block) for j in range(block)])])
            g32 = {k: x.astype(np.float32) for k, x in g.items()}
            ising.ising_nn_apply_grads(tr.h, ising.nn_flatten(g32), lr)
            p64, m, v = staged.adam_step(p64, {k: x.astype(np.float64) for k, x in g32.items()}, m, v, t, lr)
        got = tr.params()
        blob = tr.blob()
    for k in p64:
        err = np.abs(got[k].astype(np.float64) - p64[k])
        assert err.max() < 2e-6 * max(1.0, np.abs(p64[k]).max()), (k, err.max())
    flat = ising.nn_flatten(got)
    want_blob = (cnn.bf16_round(flat.astype(np.float64)).astype(np.float32).view(np.uint32) >> 16)
    assert np.array_equal(blob.astype(np.uint32), want_blob)


def test_engines_agree_on_stage_logits(torch):
    """Same windows, same weights: the two layer-2 engines differ only in the
    order of the FP32 accumulation of the same FP16 products."""
    block = 16
    p32, _ = _params(17)
    wins = _windows(128, 64, block, seed=18)
    st = staged.schedule(block)
    d = torch.from_numpy(wins).cuda()
    got = {}
    with learned.Trainer(block, params=p32, proposal=STAGED) as tr:
        for engine in ENGINES:
            ising.ising_nn_set_engine(tr.h, engine)
            outs = []
            for k, (kind, _) in enumerate(st):
                if kind != "net":
                    continue
                out = torch.zeros((len(wins), block, block), dtype=torch.float32, device="cuda")
                ising.ising_nn_stage_logits(tr.h, d, len(wins), k, BETA_C, out)
                outs.append(out.cpu().numpy())
            got[engine] = np.stack(outs)
        with pytest.raises(ising.IsingError):
            ising.ising_nn_set_engine(tr.h, 2)
    a, b = got[ENGINES[0]], got[ENGINES[1]]
    assert np.abs(a).max() > 1.0
    assert np.abs(a - b).max() <= 1e-4 * max(1.0, np.abs(a).max())


def _block_only_chain(L, block, beta, blob, n, seed, engine=ising.ISING_NN_ENGINE_MMA_SYNC):
    Es, M2 = [], []
    with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS, seed=seed) as lat:
        ising.ising_nn_load(lat.ctx, blob)
        ising.ising_set_proposal(lat.ctx, STAGED)
        ising.ising_set_nn_engine(lat.ctx, engine)
        for _ in range(n):
            ising.ising_block_pass(lat.ctx, 1, block)
            E, M = lat.measure()
            Es.append(E)
            M2.append(M * M)
        prop, acc = ising.ising_block_stats(lat.ctx)
    return np.array(Es, float), np.array(M2, float), prop, acc


def test_staged_block_moves_exact_on_4x4(torch):
    L, block, beta, n = 4, 2, 0.44, 12000
    ex = exact.averages(L, beta)
    with learned.Trainer(block, params=learned.init_params(seed=9, scale=1.0), proposal=STAGED) as tr:
        blob = tr.blob()
    Es, M2, prop, acc = _block_only_chain(L, block, beta, blob, n, 11)
    e, de = stats.mean_and_error(Es[200:])
    m, dm = stats.mean_and_error(M2[200:])
    assert abs(e - ex["E"]) < 3 * de, (e, de, ex["E"])
    assert abs(m - ex["M2"]) < 3 * dm, (m, dm, ex["M2"])
    assert prop == n * 4 and 0 < acc < prop


@pytest.mark.parametrize("engine", ENGINES)
def test_staged_block_moves_match_kaufman_8x8(torch, engine):
    L, block, beta, n = 8, 4, BETA_C, 12000
    with learned.Trainer(block, params=learned.init_params(seed=14, scale=1.0), proposal=STAGED) as tr:
        blob = tr.blob()
    Es, _, prop, acc = _block_only_chain(L, block, beta, blob, n, 15, engine)
    e, de = stats.mean_and_error(Es[300:])
    want = kaufman_energy(L, beta) * L * L
    assert acc > 0.02 * prop
    assert abs(e - want) < 3 * de, (e, de, want)


@pytest.fixture(scope="module")
def trained16(torch):
    """A staged 16 x 16 network trained briefly at beta_c (tens of seconds)."""
    wins = learned.generate_windows([64, 128], BETA_C, 6144, 16, seed=51, thermalise=2000, thin=40)
    with learned.Trainer(16, seed=52, proposal=STAGED) as tr:
        losses = tr.fit(wins, epochs=2, batch=256, lr=2e-3, seed=53)
        blob = tr.blob()
    return blob, losses


def test_trained_staged_16x16_accepts_and_keeps_the_chain(torch, trained16):
    blob, losses = trained16
    assert np.mean(losses[-5:]) < np.mean(losses[:5])
    L, block, beta = 64, 16, BETA_C
    res, rates = {}, []
    for mode in ("plain", "staged"):
        Es, Ms = [], []
        for seed in range(61, 69):
            with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS, seed=seed) as lat:
                every = 0
                if mode == "staged":
                    ising.ising_nn_load(lat.ctx, blob)
                    ising.ising_set_proposal(lat.ctx, STAGED)
                    every = 1
                ising.ising_sweep_blocks(lat.ctx, 500, 0, block, every)
                ising.ising_sweep_blocks(lat.ctx, 3000, 1, block, every)
                E, M = lat.series(3000)
                Es.append(stats.mean_and_error(E / (L * L)))
                Ms.append(stats.mean_and_error(np.abs(M) / (L * L)))
                if mode == "staged":
                    p, a = ising.ising_block_stats(lat.ctx)
                    rates.append(a / p)
        res[mode] = (stats.combine_runs([a for a, _ in Es], [b for _, b in Es]),
                     stats.combine_runs([a for a, _ in Ms], [b for _, b in Ms]))
    assert min(rates) > 0.01, rates
    for idx in (0, 1):
        (a, da), (b, db) = res["plain"][idx], res["staged"][idx]
        assert abs(a - b) < 3 * np.hypot(da, db), (idx, res)
    e_exact = kaufman_energy(L, beta)
    (b, db) = res["staged"][0]
    assert abs(b - e_exact) < 3 * db, (b, db, e_exact)


@pytest.mark.parametrize("engine", ENGINES)
def test_batch_staged_pass_equals_single_lattice_pass(torch, engine):
    Ls, betas, block, seed = [32, 64], np.array([0.38, 0.42, 0.46]), 8, 5
    with learned.Trainer(block, params=learned.init_params(seed=13), proposal=STAGED) as tr:
        blob = tr.blob()
    with ising.Batch(Ls, betas, 1000, seed=seed) as b:
        ising.ising_batch_nn_load(b.h, blob)
        ising.ising_batch_set_proposal(b.h, STAGED)
        ising.ising_batch_set_nn_engine(b.h, engine)
        ising.ising_batch_block_pass(b.h, 3, block)
        got = {(l, i): b.spins(l, i) for l in range(2) for i in range(3)}
        pb, ab = ising.ising_batch_block_stats(b.h)
    tot_p = tot_a = 0
    for l, L in enumerate(Ls):
        for i in range(3):
            with ising.Lattice(L, betas[i], ising.ISING_LAYOUT_BITS) as lat:
                ising.ising_set_replica(lat.ctx, l * 3 + i)
                lat.seed(seed)
                ising.ising_nn_load(lat.ctx, blob)
                ising.ising_set_proposal(lat.ctx, STAGED)
                ising.ising_set_nn_engine(lat.ctx, engine)
                ising.ising_block_pass(lat.ctx, 3, block)
                assert np.array_equal(lat.spins(), got[(l, i)]), (l, i)
                p_, a_ = ising.ising_block_stats(lat.ctx)
                tot_p += p_
                tot_a += a_
    assert (pb, ab) == (tot_p, tot_a) and ab > 0
