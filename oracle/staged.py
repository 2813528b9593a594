"""CPU reference of the staged (autoregressive) block proposal, and of Adam.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): only the tests, the smoke
check and the benchmark's CPU legs may import it.  Plain numpy in float64.

The paper has no learned proposal (its Monte Carlo is single-site Metropolis,
Results A and Supplementary "Detail of the MC calculation"); this is the block
move the build adds to the same chain, written from its definition.

A B x B square (interior sites (i, j), i = row, 0 <= i, j < B) is redrawn
conditioned on the four edges of the ring around it, like the one-shot
proposal of ``oracle/cnn.py``, but site by site in *stages*:

* Site classes (local to the square): 0 = i even and j even; 1 = i and j odd
  with ((i - 1) / 2 + (j - 1) / 2) even; 2 = the other i, j odd sites;
  3 = i + j odd.  A class-3 site has no class-3 neighbour, and no two class-2
  sites are neighbours or share a neighbour.
* Depth d = min(i, j, B-1-i, B-1-j) (distance from the ring); band = d // 2.
* Schedule.  Known sites start as the ring edges (the corners are never used).
  For band k = 0, 1, ...: a *network* stage with the unknown class-0 sites of
  band k, a network stage with the unknown class-1 sites of band k, then the
  *closure*: repeat { if some unknown sites have all four neighbours known, an
  exact stage with all of them; else if some unknown class-2 sites are exactly
  drawable (every unknown neighbour n has all its other neighbours known), an
  exact stage with all of them; else stop }.  A final closure draws whatever is
  left.
* Network stage: the CNN of ``oracle/cnn.py`` on a frame whose channel 0 is
  the known spins (0 elsewhere) and channel 1 the known mask; logit l_i of
  every site of the stage.
* Exact stage: the conditional of s_i given the known sites with its unknown
  neighbours summed out (each such neighbour n has all its other neighbours
  known, with sum h_n):
      l_i = sum_{known n} 2 beta s_n
            + sum_{unknown n} [log cosh(beta (h_n + 1)) - log cosh(beta (h_n - 1))].
  This is the exact log-odds of p(s_i = +1 | known) (a heat-bath draw when no
  neighbour is unknown), so these stages add nothing to the mismatch between
  the proposal and the Boltzmann conditional.
* Every stage draws its sites with the quantised probability of
  ``cnn.quantise``: s_i = +1 iff u_i < P_i; q(x) = prod over all sites of
  (P_i or 2^32 - P_i) / 2^32, the P_i of each stage computed from the sites of
  x known before that stage.  The same product evaluated on the current
  interior (teacher forcing) gives q(old).
* Metropolis-Hastings: accept with min(1, exp(-beta dE) q(old) / q(new)), dE
  over the bonds that touch the interior.

Training of the staged proposal: maximum likelihood, loss = mean over windows
of sum over network stages of sum over the stage's sites of BCE(l_i, (s_i+1)/2)
with the stage's known mask on the input.

Adam (Kingma & Ba, "Adam: a method for stochastic optimization", ICLR 2015,
Algorithm 1): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

from . import cnn

NB = ((-1, 0), (1, 0), (0, -1), (0, 1))
TWO32 = 4294967296.0


def site_class(B: int, i: int, j: int) -> int:
    if (i + j) % 2 == 1:
        return 3
    if i % 2 == 0:
        return 0
    return 1 if ((i - 1) // 2 + (j - 1) // 2) % 2 == 0 else 2


def depth(B: int, i: int, j: int) -> int:
    return min(i, j, B - 1 - i, B - 1 - j)


def ring_mask(B: int) -> np.ndarray:
    """(B+2) x (B+2) bool: the four ring edges (no corners)."""
    F = B + 2
    m = np.zeros((F, F), dtype=bool)
    m[0, 1:-1] = m[-1, 1:-1] = m[1:-1, 0] = m[1:-1, -1] = True
    return m


def _nbrs(i, j):
    """frame coordinates of the four neighbours of interior site (i, j)"""
    return [(i + 1 + dy, j + 1 + dx) for dy, dx in NB]


def _all_nbrs_known(known, i, j):
    return all(known[a, b] for a, b in _nbrs(i, j))


def _exactly_drawable(known, i, j):
    """every unknown neighbour of (i, j) has all its other neighbours known"""
    fi, fj = i + 1, j + 1
    for a, b in _nbrs(i, j):
        if known[a, b]:
            continue
        for dy, dx in NB:
            c, d = a + dy, b + dx
            if (c, d) != (fi, fj) and not known[c, d]:
                return False
    return True


def schedule(B: int):
    """[(kind, [(i, j), ...])] in drawing order; kind 'net' or 'exact'."""
    known = ring_mask(B)
    unknown = {(i, j) for i in range(B) for j in range(B)}
    stages = []

    def add(kind, sites):
        sites = sorted(sites)
        stages.append((kind, sites))
        for (i, j) in sites:
            known[i + 1, j + 1] = True
            unknown.discard((i, j))

    def closure():
        while True:
            x = [(i, j) for (i, j) in unknown if _all_nbrs_known(known, i, j)]
            if x:
                add("exact", x)
                continue
            y = [(i, j) for (i, j) in unknown
                 if site_class(B, i, j) == 2 and _exactly_drawable(known, i, j)]
            if y:
                add("exact", y)
                continue
            return

    n_bands = (B // 2 + 1) // 2
    for k in range(n_bands):
        for cls in (0, 1):
            s = [(i, j) for (i, j) in unknown
                 if site_class(B, i, j) == cls and depth(B, i, j) // 2 == k]
            if s:
                add("net", s)
        closure()
    closure()
    assert not unknown, "schedule left sites undrawn"
    return stages


def known_before(B: int, stages, k: int) -> np.ndarray:
    """(B+2)^2 bool known mask before stage k."""
    m = ring_mask(B)
    for kind, sites in stages[:k]:
        for (i, j) in sites:
            m[i + 1, j + 1] = True
    return m


def _lcosh(x):
    return np.logaddexp(x, -x)


def exact_logodds(win, known, beta, i, j):
    """Log-odds of s_i = +1 for the exact stage; win is one window ((B+2)^2
    spins) or a stack of them (..., B+2, B+2)."""
    win = np.asarray(win, dtype=np.float64)
    fi, fj = i + 1, j + 1
    l = np.zeros(win.shape[:-2])
    for a, b in _nbrs(i, j):
        if known[a, b]:
            l = l + 2.0 * beta * win[..., a, b]
        else:
            h = np.zeros(win.shape[:-2])
            for dy, dx in NB:
                c, d = a + dy, b + dx
                if (c, d) != (fi, fj):
                    assert known[c, d], "exact stage with an undetermined neighbour"
                    h = h + win[..., c, d]
            l = l + _lcosh(beta * (h + 1.0)) - _lcosh(beta * (h - 1.0))
    return l


def stage_frame(win, known):
    """Network input (2, F, F) (or (N, 2, F, F) for a stack): known spins,
    known mask."""
    win = np.asarray(win, dtype=np.float64)
    x0 = np.where(known, win, 0.0)
    x1 = np.broadcast_to(known.astype(np.float64), x0.shape)
    return np.stack([x0, x1], axis=-3)


def stage_logits(params, win, beta, B, stages, k):
    """Logits (B, B) (or (N, B, B)) of stage k for window(s) win (only the
    stage's sites are meaningful for an exact stage; the rest are 0 there)."""
    kind, sites = stages[k]
    known = known_before(B, stages, k)
    win = np.asarray(win)
    single = win.ndim == 2
    w = win[None] if single else win
    if kind == "net":
        out = cnn.forward(params, stage_frame(w, known))
    else:
        out = np.zeros((w.shape[0], B, B))
        for (i, j) in sites:
            out[:, i, j] = exact_logodds(w, known, beta, i, j)
    return out[0] if single else out


def _log_term(P, s):
    return np.log(P if s > 0 else TWO32 - P) - np.log(TWO32)


def log_q_many(params, wins, beta, B, stages=None):
    """Teacher-forced natural log of the quantised staged proposal density of
    the interior of each window of the stack wins (N, B+2, B+2)."""
    stages = stages or schedule(B)
    wins = np.asarray(wins)
    tot = np.zeros(wins.shape[0])
    for k, (kind, sites) in enumerate(stages):
        P = cnn.quantise(stage_logits(params, wins, beta, B, stages, k)).astype(np.float64)
        for (i, j) in sites:
            s = wins[:, i + 1, j + 1]
            tot += np.log(np.where(s > 0, P[:, i, j], TWO32 - P[:, i, j])) - np.log(TWO32)
    return tot


def log_q(params, win, beta, B, stages=None):
    """Teacher-forced natural log of the quantised staged proposal density of
    the interior of win given its ring (one window, site by site)."""
    stages = stages or schedule(B)
    tot = 0.0
    for k, (kind, sites) in enumerate(stages):
        P = cnn.quantise(stage_logits(params, win, beta, B, stages, k))
        for (i, j) in sites:
            tot += _log_term(int(P[i, j]), win[i + 1, j + 1])
    return float(tot)


def propose(params, win, beta, B, u, stages=None):
    """Draw a new interior from the staged proposal with uniforms u (B x B
    uint32); returns (new interior (B, B) int8, natural log q(new))."""
    stages = stages or schedule(B)
    w = np.array(win, dtype=np.int64)
    w[1:-1, 1:-1] = 0
    lq = 0.0
    for k, (kind, sites) in enumerate(stages):
        P = cnn.quantise(stage_logits(params, w, beta, B, stages, k))
        for (i, j) in sites:
            s = 1 if int(u[i, j]) < int(P[i, j]) else -1
            w[i + 1, j + 1] = s
            lq += _log_term(int(P[i, j]), s)
    return w[1:-1, 1:-1].astype(np.int8), float(lq)


def block_mh(spins, ox, oy, B, params, beta, u_sample, u_accept, stages=None):
    """One staged block MH update in place (interior origin (ox, oy), periodic).
    Returns True if accepted."""
    fr, old = cnn.frame(spins, ox, oy, B)
    L = spins.shape[0]
    F = B + 2
    ys = (oy - 1 + np.arange(F)) % L
    xs = (ox - 1 + np.arange(F)) % L
    win = spins[np.ix_(ys, xs)].astype(np.int64)
    win[~(ring_mask(B) | _interior(B))] = 0  # corners are never read
    new, lq_new = propose(params, win, beta, B, u_sample, stages)
    lq_old = log_q(params, win, beta, B, stages)
    dE = cnn.block_energy_change(spins, ox, oy, B, new)
    log_alpha = -beta * dE + lq_old - lq_new
    if log_alpha >= 0 or u_accept < np.exp(log_alpha):
        spins[np.ix_(ys[1:-1], xs[1:-1])] = new
        return True
    return False


def _interior(B):
    m = np.zeros((B + 2, B + 2), dtype=bool)
    m[1:-1, 1:-1] = True
    return m


# ---------------------------------------------------------------------------
# training of the staged proposal
# ---------------------------------------------------------------------------

def masked_loss_and_grads(params, frames, targets, tmask, bf16_operands=False):
    """Mean over samples of sum over tmask sites of BCE(logit, (t+1)/2) and
    its gradients.  frames (N, 2, F, F), targets (N, B, B) +-1, tmask (N, B, B).

    bf16_operands: the same objective with the operands of the 32 -> 32
    convolution rounded to bfloat16 where a BF16-operand / FP32-accumulate
    tensor-core implementation rounds them (BF16 weights with FP32
    accumulation): W2, the layer-1 output h1 (forward and weight gradient),
    the layer-2 output h2 (which layer 3 and its gradient read) and dL/dz2
    (input and weight gradients of layer 2; the bias gradient sums it
    unrounded).  Everything else stays float64."""
    r = cnn.bf16_round if bf16_operands else (lambda a: a)
    W2 = r(params["W2"])
    x0 = frames
    z1 = cnn.conv3x3(x0, params["W1"], params["b1"])
    h1 = r(np.maximum(z1, 0.0))
    z2 = cnn.conv3x3(h1, W2, params["b2"])
    h2 = r(np.maximum(z2, 0.0))
    z3 = cnn.conv3x3(h2, params["W3"], params["b3"])
    logits = z3[:, 0, 1:-1, 1:-1]
    y = (targets.astype(np.float64) + 1.0) / 2.0
    w = tmask.astype(np.float64)
    N = frames.shape[0]
    loss = (w * (np.maximum(logits, 0) - logits * y + np.log1p(np.exp(-np.abs(logits))))).sum() / N
    g = w * (1.0 / (1.0 + np.exp(-logits)) - y) / N
    gz3 = np.zeros_like(z3)
    gz3[:, 0, 1:-1, 1:-1] = g
    gh2, gW3, gb3 = cnn.conv3x3_backward(h2, params["W3"], gz3)
    gz2 = gh2 * (z2 > 0)
    gh1, gW2, _ = cnn.conv3x3_backward(h1, W2, r(gz2))
    gb2 = gz2.sum(axis=(0, 2, 3))
    gz1 = gh1 * (z1 > 0)
    _, gW1, gb1 = cnn.conv3x3_backward(x0, params["W1"], gz1)
    return loss, {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3}


def training_samples(windows, B, stages=None):
    """Expand windows (N, F, F) int8 into one (frame, target, mask) sample per
    (window, network stage); the loss over them, times the number of network
    stages, is the mean over windows of -log q_net."""
    stages = stages or schedule(B)
    net = [k for k, (kind, _) in enumerate(stages) if kind == "net"]
    frs, tg, tm = [], [], []
    for win in windows:
        w = np.asarray(win, dtype=np.int64)
        for k in net:
            known = known_before(B, stages, k)
            frs.append(stage_frame(w, known))
            tg.append(w[1:-1, 1:-1])
            m = np.zeros((B, B), dtype=bool)
            for (i, j) in stages[k][1]:
                m[i, j] = True
            tm.append(m)
    return np.stack(frs), np.stack(tg), np.stack(tm)


def staged_loss_and_grads(params, windows, B, stages=None, bf16_operands=False):
    """Loss = mean over windows of sum over network stages of the masked BCE
    (bf16_operands as in masked_loss_and_grads)."""
    frs, tg, tm = training_samples(windows, B, stages)
    n_net = frs.shape[0] // len(windows)
    loss, g = masked_loss_and_grads(params, frs, tg, tm, bf16_operands)
    return loss * n_net, {k: v * n_net for k, v in g.items()}


def adam_step(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t = 1, 2, ...) in float64; returns new (params, m, v)."""
    P, Mo, Vo = {}, {}, {}
    for k in params:
        Mo[k] = b1 * m[k] + (1.0 - b1) * grads[k]
        Vo[k] = b2 * v[k] + (1.0 - b2) * grads[k] ** 2
        mh = Mo[k] / (1.0 - b1 ** t)
        vh = Vo[k] / (1.0 - b2 ** t)
        P[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return P, Mo, Vo
