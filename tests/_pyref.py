"""Independent pure-Python restatements used to pin the C oracle on tiny cases.

* ``philox`` follows the Philox4x32-10 round function of Salmon et al. (SC'11)
  with Python integers; it is pinned by the published known-answer vectors.
* ``anneal_full_energy`` is the Metropolis sweep written from its definition,
  with the energy change of a flip taken as H(s') - H(s) by evaluating Eq. 2
  on the whole edge list before and after (no local fields, no CSR), and the
  acceptance probability exp(-beta dE) compared against u / 2^B through the
  threshold T = floor(exp(-beta dE) 2^B), B = 32 (or 16 in the 16-bit draw
  mode).
"""
import math

import numpy as np

MASK = 0xFFFFFFFF


def philox(ctr, key, rounds=10):
    c = [int(v) & MASK for v in ctr]
    k0, k1 = int(key[0]) & MASK, int(key[1]) & MASK
    for _ in range(rounds):
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & MASK, p1 & MASK, ((p0 >> 32) ^ c[3] ^ k1) & MASK, p0 & MASK]
        k0 = (k0 + 0x9E3779B9) & MASK
        k1 = (k1 + 0xBB67AE85) & MASK
    return c


def draw(a, b, t, seed):
    out = philox((a, b, t >> 2, 0), (seed & MASK, (seed >> 32) & MASK))
    return out[t & 3]


def draw16(a, b, t, seed):
    """16-bit draw mode: trial t takes the low (t even) or high (t odd) half of
    word (t mod 8) // 2 of the block at counter (a, b, t // 8, 0)."""
    out = philox((a, b, t // 8, 0), (seed & MASK, (seed >> 32) & MASK))
    word = out[(t % 8) // 2]
    return (word >> 16) if t % 2 else (word & 0xFFFF)


def energy(edges, s):
    i, j, w = edges
    return int(sum(int(w[e]) * int(s[i[e]]) * int(s[j[e]]) for e in range(len(w))))


def anneal_full_energy(X, Y, edges, betas, seed, trials, sweep_offset=0, init=None, draw_bits=32):
    n = X * Y
    out = np.zeros((trials, n), dtype=np.int8)
    for t in range(trials):
        if init is not None:
            s = [1 if v > 0 else -1 for v in init[t]]
        else:
            s = [1 if (draw(i, 0xFFFFFFFF, t, seed) >> 31) else -1 for i in range(n)]
        for jj, beta in enumerate(betas):
            k = (sweep_offset + jj) & MASK
            for colour in (0, 1):
                for i in range(n):
                    if ((i % X) + (i // X)) % 2 != colour:
                        continue
                    e0 = energy(edges, s)
                    s[i] = -s[i]
                    dE = energy(edges, s) - e0
                    s[i] = -s[i]
                    if dE <= 0:
                        flip = True
                    else:
                        B = draw_bits
                        thr = min(math.floor(math.exp(-beta * dE) * 2.0 ** B), 2 ** B - 1)
                        u = draw16(i, k, t, seed) if B == 16 else draw(i, k, t, seed)
                        flip = u < thr
                    if flip:
                        s[i] = -s[i]
        out[t] = s
    return out


def graph_energy(n, edges, h, s):
    """Eq. 2 with fields from an edge list (i, j, J): -sum J s_i s_j - sum h s."""
    i, j, Jv = edges
    e = -sum(int(Jv[k]) * int(s[i[k]]) * int(s[j[k]]) for k in range(len(Jv)))
    if h is not None:
        e -= sum(int(h[q]) * int(s[q]) for q in range(n))
    return e


def first_fit_colouring(n, adj):
    """Smallest colour not taken by an earlier neighbour, sites in index order."""
    colour = [0] * n
    for v in range(n):
        taken = {colour[u] for u in adj[v] if u < v}
        c = 0
        while c in taken:
            c += 1
        colour[v] = c
    return colour


def anneal_graph_full_energy(n, edges, h, colour, betas, seed, trials, sweep_offset=0):
    """The Metropolis sweep over colour classes in order, each flip judged by
    the difference of whole-graph energies (Eq. 2 with fields)."""
    out = np.zeros((trials, n), dtype=np.int8)
    ncol = max(colour) + 1
    for t in range(trials):
        s = [1 if (draw(q, 0xFFFFFFFF, t, seed) >> 31) else -1 for q in range(n)]
        for jj, beta in enumerate(betas):
            k = (sweep_offset + jj) & MASK
            for c in range(ncol):
                for q in range(n):
                    if colour[q] != c:
                        continue
                    e0 = graph_energy(n, edges, h, s)
                    s[q] = -s[q]
                    dE = graph_energy(n, edges, h, s) - e0
                    s[q] = -s[q]
                    if dE <= 0:
                        flip = True
                    else:
                        thr = min(math.floor(math.exp(-beta * dE) * 2.0 ** 32), 2 ** 32 - 1)
                        flip = draw(q, k, t, seed) < thr
                    if flip:
                        s[q] = -s[q]
        out[t] = s
    return out
