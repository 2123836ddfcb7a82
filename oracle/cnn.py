"""CPU oracle for the learned proposal stage (FP64).

TEST INFRASTRUCTURE ONLY (tests, smoke, benchmark baselines).

The network is a small circular-padded CNN on the torus: four 3x3
convolutions with 32 channels and ReLU between them, 3 input channels per
site, and one logit per site.  The inputs are the spin s_i, w to the right and
w downwards, all +-1; the paper's problem data is Eq. 2 with J = -w.  The
logit scores "flip this spin".  The paper has no learned component (its Cosm
rule is unpublished, Section III); this stage and its readings are this
project's.

Parameters are one flat float vector in this order, each convolution weight
laid out (out channel, in channel, ky, kx):
    W1 [32,3,3,3], b1 [32], W2 [32,32,3,3], b2 [32],
    W3 [32,32,3,3], b3 [32], W4 [1,32,3,3], b4 [1]

Convolution on the torus: out[y, x] = b + sum W[o, c, ky, kx] * in[c, (y+ky-1)
mod Y, (x+kx-1) mod X].  The forward pass is done with torch CPU float64 ops
(conv2d with circular padding), which the tests pin against a direct numpy
loop; gradients come from autograd, pinned by finite differences.

Training target (reading of the gauge symmetry): for an input state s and a
low-energy reference state r of the same instance, y_i = [s_i != r'_i], where
r' is r or -r, whichever is closer to s in Hamming distance (on a tie, the one
that keeps site 0).  The loss is the
mean binary cross-entropy with logits.

Proposals (exact acceptance): sites with logit > 0 are proposed for flipping,
restricted to square tiles of side b (the last tile of a row or column may be
smaller); tiles whose (tx + ty) is even go first, then the odd ones.  With the
number of tiles along each side 1 or even, same-parity tiles share no edge
even across the periodic boundary, so their decisions are independent.  A tile's proposal B is accepted iff its exact energy change
dE_B = -2 sum_{i in B, j not in B, j ~ i} w_ij s_i s_j is <= 0 (flipping B
reverses the sign of exactly its boundary terms of H = sum w_ij s_i s_j).
"""
from __future__ import annotations

import numpy as np

CH = 32
SHAPES = [("W1", (CH, 3, 3, 3)), ("b1", (CH,)), ("W2", (CH, CH, 3, 3)), ("b2", (CH,)),
          ("W3", (CH, CH, 3, 3)), ("b3", (CH,)), ("W4", (1, CH, 3, 3)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(params):
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = np.asarray(params[o:o + k]).reshape(shp)
        o += k
    return out


def init_params(seed, scale=1.0):
    """Seeded starting weights: the shared input generator (synth)."""
    import synth
    return synth.cnn_init_params(seed, scale)


def features(spins, w_right, w_down):
    """[B, 3, Y, X] float64 input: (s, w_right, w_down)."""
    s = np.asarray(spins, dtype=np.float64)
    B = s.shape[0]
    Y, X = w_right.shape
    f = np.empty((B, 3, Y, X))
    f[:, 0] = s.reshape(B, Y, X)
    f[:, 1] = w_right[None]
    f[:, 2] = w_down[None]
    return f


def _torch():
    import torch
    return torch


def forward(params, spins, w_right, w_down, return_all=False):
    """Logits [B, Y, X] (float64).  return_all: also the input features, the
    hidden pre-activations p1..p3 and activations h1..h3."""
    torch = _torch()
    F = torch.nn.functional
    p = {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)) for k, v in unflatten(params).items()}
    x = torch.from_numpy(features(spins, w_right, w_down))

    def conv(t, W, b):
        return F.conv2d(F.pad(t, (1, 1, 1, 1), mode="circular"), W, b)

    p1 = conv(x, p["W1"], p["b1"])
    h1 = torch.relu(p1)
    p2 = conv(h1, p["W2"], p["b2"])
    h2 = torch.relu(p2)
    p3 = conv(h2, p["W3"], p["b3"])
    h3 = torch.relu(p3)
    z = conv(h3, p["W4"], p["b4"])[:, 0]
    if return_all:
        return {"x": x.numpy(), "p1": p1.numpy(), "h1": h1.numpy(), "p2": p2.numpy(), "h2": h2.numpy(),
                "p3": p3.numpy(), "h3": h3.numpy(), "z": z.numpy()}
    return z.numpy()


def loss_and_grad(params, spins, targets, w_right, w_down):
    """Mean BCE-with-logits and its gradient w.r.t. the flat parameters (float64)."""
    torch = _torch()
    F = torch.nn.functional
    theta = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    parts, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        parts[name] = theta[o:o + k].reshape(shp)
        o += k
    x = torch.from_numpy(features(spins, w_right, w_down))

    def conv(t, W, b):
        return F.conv2d(F.pad(t, (1, 1, 1, 1), mode="circular"), W, b)

    h1 = torch.relu(conv(x, parts["W1"], parts["b1"]))
    h2 = torch.relu(conv(h1, parts["W2"], parts["b2"]))
    h3 = torch.relu(conv(h2, parts["W3"], parts["b3"]))
    z = conv(h3, parts["W4"], parts["b4"])[:, 0]
    y = torch.from_numpy(np.asarray(targets, dtype=np.float64).reshape(z.shape))
    loss = F.binary_cross_entropy_with_logits(z, y)
    loss.backward()
    return float(loss.item()), theta.grad.numpy().copy()


def flip_targets(spins, reference):
    """Gauge-aligned flip targets y = [s != r'] with r' = +-r closest to s."""
    s = np.asarray(spins)
    r = np.asarray(reference)
    diff = (s != r)
    d2 = diff.sum(axis=-1, keepdims=True) * 2
    n = s.shape[-1]
    # a tie (exactly n/2 differ) is broken by site 0 so that r and -r agree
    flip_ref = (d2 > n) | ((d2 == n) & diff[..., :1])
    return np.where(flip_ref, ~diff, diff).astype(np.uint8)


# ---------------------------------------------------------------- proposals
def propose_tiles(spins, logits, w_right, w_down, tile):
    """Tile proposals with exact acceptance (see module docstring).

    spins int8 [B, n] (modified copy returned), logits [B, Y, X] or [B, n].
    Returns (new_spins, accepted [B] number of accepted tiles).
    """
    Y, X = w_right.shape
    s = np.array(spins, dtype=np.int8).reshape(-1, Y, X).copy()
    z = np.asarray(logits).reshape(-1, Y, X)
    B = s.shape[0]
    ntx, nty = -(-X // tile), -(-Y // tile)
    if (ntx != 1 and ntx % 2) or (nty != 1 and nty % 2):
        raise ValueError("tile counts per dimension must be 1 or even (independent same-parity tiles)")
    acc = np.zeros(B, dtype=np.int64)
    for phase in (0, 1):
        for b in range(B):
            for ty in range(nty):
                for tx in range(ntx):
                    if (tx + ty) % 2 != phase:
                        continue
                    y0, y1 = ty * tile, min(Y, (ty + 1) * tile)
                    x0, x1 = tx * tile, min(X, (tx + 1) * tile)
                    m = z[b, y0:y1, x0:x1] > 0
                    if not m.any():
                        continue
                    inB = np.zeros((Y, X), dtype=bool)
                    inB[y0:y1, x0:x1] = m
                    dE = 0
                    for yy, xx in zip(*np.nonzero(inB)):
                        si = int(s[b, yy, xx])
                        for (jy, jx, w) in (
                                (yy, (xx + 1) % X, int(w_right[yy, xx])),
                                (yy, (xx - 1) % X, int(w_right[yy, (xx - 1) % X])),
                                ((yy + 1) % Y, xx, int(w_down[yy, xx])),
                                ((yy - 1) % Y, xx, int(w_down[(yy - 1) % Y, xx]))):
                            if not inB[jy, jx]:
                                dE += -2 * w * si * int(s[b, jy, jx])
                    if dE <= 0:
                        s[b][inB] = -s[b][inB]
                        acc[b] += 1
    return s.reshape(B, -1), acc


def propose_global(spins, logits, w_right, w_down):
    """Whole-lattice proposal (warm start): flip every site with logit > 0,
    accept iff the exact energy does not increase."""
    Y, X = w_right.shape
    s = np.array(spins, dtype=np.int8).reshape(-1, Y, X).copy()
    z = np.asarray(logits).reshape(-1, Y, X)
    acc = np.zeros(s.shape[0], dtype=np.int64)

    def energy(t):
        t = t.astype(np.int64)
        return int((w_right * t * np.roll(t, -1, axis=1)).sum() + (w_down * t * np.roll(t, -1, axis=0)).sum())

    for b in range(s.shape[0]):
        m = z[b] > 0
        if not m.any():
            continue
        cand = s[b].copy()
        cand[m] = -cand[m]
        if energy(cand) <= energy(s[b]):
            s[b] = cand
            acc[b] = 1
    return s.reshape(s.shape[0], -1), acc


# ---------------------------------------------------------------- clusters
def _energy_grid(s, w_right, w_down):
    """H = sum over the 2n torus edges of w_ij s_i s_j (Eq. 2 with J = -w, h = 0)."""
    t = np.asarray(s, dtype=np.int64)
    return int((w_right * t * np.roll(t, -1, axis=1)).sum() + (w_down * t * np.roll(t, -1, axis=0)).sum())


def torus_components(mask):
    """Connected components of the True sites of mask [Y, X] under 4-neighbour
    adjacency on the torus: a list of lists of (y, x), found by breadth-first
    search from each unvisited site in increasing index order."""
    Y, X = mask.shape
    seen = np.zeros_like(mask, dtype=bool)
    comps = []
    for y0 in range(Y):
        for x0 in range(X):
            if not mask[y0, x0] or seen[y0, x0]:
                continue
            comp, queue = [], [(y0, x0)]
            seen[y0, x0] = True
            while queue:
                y, x = queue.pop()
                comp.append((y, x))
                for yy, xx in ((y, (x + 1) % X), (y, (x - 1) % X), ((y + 1) % Y, x), ((y - 1) % Y, x)):
                    if mask[yy, xx] and not seen[yy, xx]:
                        seen[yy, xx] = True
                        queue.append((yy, xx))
            comps.append(comp)
    return comps


def component_dE(s_grid, comp, w_right, w_down):
    """Energy change of flipping the sites of one component, as the
    difference of the whole-lattice energies (the definition)."""
    t = np.array(s_grid, dtype=np.int8)
    e0 = _energy_grid(t, w_right, w_down)
    for y, x in comp:
        t[y, x] = -t[y, x]
    return _energy_grid(t, w_right, w_down) - e0


def droplet_targets(spins, reference, w_right, w_down):
    """Training targets of the cluster form of the learned stage (a reading of
    the block-flip proposals, not in the paper): with r' = +-r gauge-aligned
    to s (as flip_targets), the sites where s and r' differ split into
    connected components on the torus; y_i = 1 iff i lies in a component whose
    flip alone lowers the energy of s (dE < 0).  Such a component is an exact
    multi-spin move from s towards the better state.  uint8 [B, n]."""
    Y, X = w_right.shape
    d = flip_targets(spins, reference).reshape(-1, Y, X).astype(bool)
    s = np.asarray(spins, dtype=np.int8).reshape(-1, Y, X)
    out = np.zeros(d.shape, dtype=np.uint8)
    for b in range(d.shape[0]):
        for comp in torus_components(d[b]):
            if component_dE(s[b], comp, w_right, w_down) < 0:
                for y, x in comp:
                    out[b, y, x] = 1
    return out.reshape(d.shape[0], -1)


def propose_clusters(spins, logits, w_right, w_down):
    """Cluster proposals: every connected component of the sites with logit > 0
    is flipped iff its flip alone does not raise the energy (dE <= 0).
    Components are never adjacent, so their flips are independent and the
    accepted ones can be applied together.  Returns (new spins [B, n],
    accepted components [B])."""
    Y, X = w_right.shape
    s = np.array(spins, dtype=np.int8).reshape(-1, Y, X).copy()
    z = np.asarray(logits).reshape(-1, Y, X)
    acc = np.zeros(s.shape[0], dtype=np.int64)
    for b in range(s.shape[0]):
        base = s[b].copy()
        for comp in torus_components(z[b] > 0):
            if component_dE(base, comp, w_right, w_down) <= 0:
                for y, x in comp:
                    s[b, y, x] = -s[b, y, x]
                acc[b] += 1
    return s.reshape(s.shape[0], -1), acc


def transcribe(spins, shift, w_right, w_down):
    """Partner cluster moves (a reading of block flips with blocks taken from
    another trial instead of the network): configuration t of a batch of B
    takes partner p = (t + shift) mod B; every component of the disagreement
    between s_t and the gauge-aligned s_p whose flip alone lowers the energy
    of s_t is flipped (droplet_targets), all partners read before any move.
    Returns (new spins [B, n], flipped components [B])."""
    s = np.asarray(spins, dtype=np.int8)
    B = s.shape[0]
    partner = s[(np.arange(B) + shift) % B]
    y = droplet_targets(s, partner, w_right, w_down)
    Y, X = w_right.shape
    d = flip_targets(s, partner).reshape(B, Y, X).astype(bool)
    comps = np.zeros(B, dtype=np.int64)
    for b in range(B):
        sg = s[b].reshape(Y, X)
        comps[b] = sum(component_dE(sg, c, w_right, w_down) < 0 for c in torus_components(d[b]))
    return np.where(y.astype(bool), -s, s).astype(np.int8), comps
