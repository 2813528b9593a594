"""CPU reference of the learned block proposal (plain numpy, float64).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  Not in the paper (whose MC
is single-site Metropolis); this is the block proposal the build adds on top
of the checkerboard sweep, written from its definition:

* Network: three 3 x 3 convolutions with zero ('same') padding on a
  (B+2) x (B+2) frame around a B x B block: 2 -> C -> C -> 1 channels, ReLU after
  the first two.  Input channel 0 = boundary spins (+-1) on the four edges of
  the ring around the block (corners and interior 0), channel 1 = 1 on those
  edge sites.  The logits of the B x B interior are the inner part of the
  output.
* Proposal: p_i = sigmoid(logit_i), quantised to an integer P_i in
  [1, 2^32 - 1]; a new interior spin is +1 iff u_i < P_i.  The proposal
  density is q(x) = prod_i (x_i = +1 ? P_i : 2^32 - P_i) / 2^32.
* Metropolis-Hastings: accept the new interior with probability
  min(1, exp(-beta dE) q(x_old) / q(x_new)), dE counting every bond that touches
  the interior (boundary unchanged, so q(.|boundary) is the same both ways).
* Training: maximum likelihood, loss = mean over blocks of
  sum_i BCE(logit_i, (x_i + 1) / 2), gradients by hand (backward convolutions).
"""
from __future__ import annotations

import numpy as np


def init_params(C: int = 32, seed: int = 0, scale: float = 1.0) -> dict:
    """He-style random initialisation (float64)."""
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.standard_normal((C, 2, 3, 3)) * np.sqrt(2.0 / 18) * scale,
        "b1": np.zeros(C),
        "W2": rng.standard_normal((C, C, 3, 3)) * np.sqrt(2.0 / (9 * C)) * scale,
        "b2": np.zeros(C),
        "W3": rng.standard_normal((1, C, 3, 3)) * np.sqrt(1.0 / (9 * C)) * scale,
        "b3": np.zeros(1),
    }
    return p


def _pad(x):
    return np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))


def conv3x3(x, W, b):
    """x (N, Cin, H, W) -> (N, Cout, H, W), zero padding 1; plain sum over taps."""
    N, Ci, H, Wd = x.shape
    Co = W.shape[0]
    xp = _pad(x)
    out = np.zeros((N, Co, H, Wd))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + H, dx:dx + Wd]  # (N, Ci, H, W)
            out += np.einsum("nchw,oc->nohw", patch, W[:, :, dy, dx])
    return out + b[None, :, None, None]


def conv3x3_backward(x, W, gout):
    """Gradients of conv3x3(x, W, b) for upstream gradient gout."""
    N, Ci, H, Wd = x.shape
    xp = _pad(x)
    gW = np.zeros_like(W)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + H, dx:dx + Wd]
            gW[:, :, dy, dx] = np.einsum("nohw,nchw->oc", gout, patch)
            gxp[:, :, dy:dy + H, dx:dx + Wd] += np.einsum("nohw,oc->nchw", gout, W[:, :, dy, dx])
    gb = gout.sum(axis=(0, 2, 3))
    return gxp[:, :, 1:-1, 1:-1], gW, gb


def forward(params, frames, keep=False):
    """frames (N, 2, B+2, B+2) -> logits (N, B, B) (and the activations)."""
    z1 = conv3x3(frames, params["W1"], params["b1"])
    h1 = np.maximum(z1, 0.0)
    z2 = conv3x3(h1, params["W2"], params["b2"])
    h2 = np.maximum(z2, 0.0)
    z3 = conv3x3(h2, params["W3"], params["b3"])
    logits = z3[:, 0, 1:-1, 1:-1]
    if keep:
        return logits, (frames, z1, h1, z2, h2, z3)
    return logits


def loss_and_grads(params, frames, interior):
    """Mean over blocks of sum_i BCE(logit_i, (s_i+1)/2) and its gradients."""
    logits, (x0, z1, h1, z2, h2, z3) = forward(params, frames, keep=True)
    y = (interior.astype(np.float64) + 1.0) / 2.0
    N = frames.shape[0]
    # BCE with logits, numerically stable
    loss = (np.maximum(logits, 0) - logits * y + np.log1p(np.exp(-np.abs(logits)))).sum() / N
    g = (1.0 / (1.0 + np.exp(-logits)) - y) / N
    gz3 = np.zeros_like(z3)
    gz3[:, 0, 1:-1, 1:-1] = g
    gh2, gW3, gb3 = conv3x3_backward(h2, params["W3"], gz3)
    gz2 = gh2 * (z2 > 0)
    gh1, gW2, gb2 = conv3x3_backward(h1, params["W2"], gz2)
    gz1 = gh1 * (z1 > 0)
    _, gW1, gb1 = conv3x3_backward(x0, params["W1"], gz1)
    return loss, {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3}


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (ties to even)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def frame(spins, ox, oy, B):
    """Input frame (2, B+2, B+2) and interior (B, B) of the block whose
    interior starts at (ox, oy) (periodic)."""
    L = spins.shape[0]
    F = B + 2
    ys = (oy - 1 + np.arange(F)) % L
    xs = (ox - 1 + np.arange(F)) % L
    win = spins[np.ix_(ys, xs)].astype(np.float64)
    mask = np.zeros((F, F))
    mask[0, 1:-1] = mask[-1, 1:-1] = mask[1:-1, 0] = mask[1:-1, -1] = 1.0
    fr = np.stack([win * mask, mask])
    return fr, spins[np.ix_(ys[1:-1], xs[1:-1])].copy()


def quantise(logits):
    """P_i = clamp(round(sigmoid(logit) 2^32), 1, 2^32 - 1) as integers."""
    z = np.asarray(logits, dtype=np.float64)
    p = 0.5 * (1.0 + np.tanh(0.5 * z))  # sigmoid without overflow
    P = np.rint(p * 4294967296.0)
    return np.clip(P, 1, 4294967295).astype(np.int64)


def log_q(P, x):
    """log of the quantised proposal density of interior x (+-1)."""
    num = np.where(x > 0, P, 4294967296 - P).astype(np.float64)
    return float(np.log(num).sum() - x.size * np.log(4294967296.0))


def block_energy_change(spins, ox, oy, B, new_interior):
    """E(new) - E(old) over the bonds that touch the block interior."""
    L = spins.shape[0]
    F = B + 2
    ys = (oy - 1 + np.arange(F)) % L
    xs = (ox - 1 + np.arange(F)) % L
    win = spins[np.ix_(ys, xs)].astype(np.int64)

    def e(w):
        # bonds with at least one end in the interior [1, B]^2 of the window
        tot = 0
        for y in range(F):
            for x in range(F):
                for (yy, xx) in ((y, x + 1), (y + 1, x)):
                    if yy >= F or xx >= F:
                        continue
                    a_in = 1 <= y <= B and 1 <= x <= B
                    b_in = 1 <= yy <= B and 1 <= xx <= B
                    if a_in or b_in:
                        tot -= w[y, x] * w[yy, xx]
        return tot

    new = win.copy()
    new[1:-1, 1:-1] = new_interior
    return e(new) - e(win)


def block_mh(spins, ox, oy, B, params, beta, u_sample, u_accept):
    """One exact block MH update in place.  u_sample: B x B uint32 uniforms for
    the draw, u_accept in [0, 1).  Returns True if accepted."""
    fr, old = frame(spins, ox, oy, B)
    P = quantise(forward(params, fr[None])[0])
    new = np.where(u_sample.astype(np.int64) < P, 1, -1).astype(np.int8)
    dE = block_energy_change(spins, ox, oy, B, new)
    log_alpha = -beta * dE + log_q(P, old) - log_q(P, new)
    if log_alpha >= 0 or u_accept < np.exp(log_alpha):
        L = spins.shape[0]
        ys = (oy + np.arange(B)) % L
        xs = (ox + np.arange(B)) % L
        spins[np.ix_(ys, xs)] = new
        return True
    return False
