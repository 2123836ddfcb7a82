"""Seeded synthetic inputs for the tests, the benchmark and the smoke run.

This module only *generates inputs*: toroidal ±1 instances in CSR form, inverse
temperature schedules and starting spin configurations.  It holds none of the
annealing arithmetic (no energies, no acceptance rule, no random stream used by
the method), so both the CUDA path and the CPU oracle may import it.

Instance recipe (stands in for the Gset toroidal instances G72/G77/G81, which
are 4-regular periodic square grids with i.i.d. weights w_ij in {-1,+1}; paper
Section I and Appendix A):

* the torus is X columns by Y rows, site i = y*X + x;
* every site owns its right edge (x+1 mod X) and its down edge (y+1 mod Y), so
  |E| = 2n, matching the |V|/|E| columns of Table I;
* each edge weight is +1 or -1 with probability 1/2, drawn with numpy's PCG64
  generator seeded by ``inst_seed`` (right edges first, then down edges, both
  in site order);
* the CSR handed to the library stores J = -w (the paper's Ising coupling,
  Eq. 2), four entries per row sorted by column.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "torus_weights",
    "torus_csr",
    "torus_instance",
    "linear_betas",
    "random_spins",
    "batched_config",
    "cnn_init_params",
    "random_graph",
    "graph_from_edges",
]


def torus_weights(X: int, Y: int, inst_seed: int):
    """Return (w_right, w_down), each int8 [Y, X] with entries in {-1, +1}."""
    rng = np.random.Generator(np.random.PCG64(int(inst_seed)))
    bits = rng.integers(0, 2, size=(2, Y, X), dtype=np.int8)
    w = (2 * bits - 1).astype(np.int8)
    return w[0].copy(), w[1].copy()


def torus_csr(X: int, Y: int, w_right: np.ndarray, w_down: np.ndarray):
    """CSR (row_ptr int64[n+1], col int32[nnz], J int8[nnz]) of the torus.

    J holds -w (Eq. 2 with J_ij = -w_ij).  Each row lists its four neighbours
    sorted by column index (right, left, down, up for equal columns, which only
    happen when a side is 2).  Works for any X, Y >= 1 (tiny or odd dimensions
    are produced on purpose by the validation tests).
    """
    n = X * Y
    y, x = np.divmod(np.arange(n, dtype=np.int64), X)
    wr = np.asarray(w_right, dtype=np.int64)
    wd = np.asarray(w_down, dtype=np.int64)
    cols = np.stack([y * X + (x + 1) % X, y * X + (x - 1) % X,
                     ((y + 1) % Y) * X + x, ((y - 1) % Y) * X + x], axis=1)
    ws = np.stack([wr[y, x], wr[y, (x - 1) % X], wd[y, x], wd[(y - 1) % Y, x]], axis=1)
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    ws = np.take_along_axis(ws, order, axis=1)
    row_ptr = np.arange(n + 1, dtype=np.int64) * 4
    return row_ptr, cols.reshape(-1).astype(np.int32), (-ws).reshape(-1).astype(np.int8)


def torus_instance(X: int, Y: int, inst_seed: int):
    """Convenience: dict with X, Y, n, w_right, w_down and the CSR arrays."""
    wr, wd = torus_weights(X, Y, inst_seed)
    row_ptr, col, J = torus_csr(X, Y, wr, wd)
    return {
        "X": X, "Y": Y, "n": X * Y, "inst_seed": inst_seed,
        "w_right": wr, "w_down": wd,
        "row_ptr": row_ptr, "col": col, "J": J,
    }


def linear_betas(beta0: float, beta1: float, S: int) -> np.ndarray:
    """Inverse temperatures for S sweeps, linear from beta0 to beta1 inclusive.

    beta_k = beta0 + (beta1 - beta0) * k / (S - 1); a single sweep uses beta0.
    """
    if S <= 0:
        return np.zeros(0, dtype=np.float64)
    if S == 1:
        return np.array([beta0], dtype=np.float64)
    k = np.arange(S, dtype=np.float64)
    return beta0 + (beta1 - beta0) * k / float(S - 1)


def random_spins(T: int, n: int, seed: int) -> np.ndarray:
    """int8 [T, n] configuration with entries in {-1, +1} (PCG64, seeded)."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    return (2 * rng.integers(0, 2, size=(T, n), dtype=np.int8) - 1).astype(np.int8)


def batched_config(count: int = 96, base_seed: int = 100):
    """The uneven batch of tori: shapes {50,100,140,200}x100, 32..512 trials,
    2,000..20,000 sweeps, instance seeds base_seed + k.

    Returns a list of dicts (X, Y, inst_seed, trials, sweeps, seed).
    """
    out = []
    widths = [50, 100, 140, 200]
    for k in range(count):
        out.append({
            "X": widths[k % 4], "Y": 100, "inst_seed": base_seed + k,
            "trials": 32 * (1 << (k % 5)),
            "sweeps": 2000 + (k * 1889) % 18001,
            "seed": 5000 + k,
        })
    return out


# Parameter shapes of the learned stage's network, in the order of its flat
# FP32 parameter vector: W1[32,3,3,3] b1 W2[32,32,3,3] b2 W3[32,32,3,3] b3
# W4[1,32,3,3] b4.
CNN_SHAPES = [
    ("W1", (32, 3, 3, 3)), ("b1", (32,)),
    ("W2", (32, 32, 3, 3)), ("b2", (32,)),
    ("W3", (32, 32, 3, 3)), ("b3", (32,)),
    ("W4", (1, 32, 3, 3)), ("b4", (1,)),
]


def cnn_init_params(seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded starting weights (float64 [19681]): normal with standard deviation
    scale * sqrt(2 / fan_in) for the convolution weights, zero biases (PCG64)."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    parts = []
    for name, shp in CNN_SHAPES:
        if name.startswith("b"):
            parts.append(np.zeros(shp))
        else:
            fan_in = shp[1] * shp[2] * shp[3]
            parts.append(rng.normal(0.0, scale * np.sqrt(2.0 / fan_in), size=shp))
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float64)


def graph_from_edges(n: int, i, j, w, h=None):
    """Symmetric CSR of an undirected graph: edges (i[e], j[e]) with weight
    w[e] (i != j, no repeats); returns a dict with n, row_ptr int64, col int32
    (rows sorted by column), J int8 = -w (the Ising coupling of Eq. 2) and the
    fields h (int8 [n] or None)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    w = np.asarray(w, dtype=np.int64)
    src = np.concatenate([i, j])
    dst = np.concatenate([j, i])
    ww = np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return {"n": int(n), "row_ptr": row_ptr, "col": dst.astype(np.int32), "J": (-ww).astype(np.int8),
            "h": None if h is None else np.asarray(h, dtype=np.int8), "w": ww.astype(np.int8)}


def random_graph(n: int, m: int, seed: int, weights: str = "pm1", hmax: int = 0):
    """A random simple graph with n vertices and m distinct edges (PCG64), in
    the form of graph_from_edges.  weights: "pm1" (w = +-1, like the Gset
    random and toroidal graphs), "one" (w = +1) or "int" (w in +-{1, 2, 3});
    hmax > 0 adds integer fields h_i in [-hmax, hmax]."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    if m > n * (n - 1) // 2:
        raise ValueError("too many edges")
    seen = set()
    ii, jj = [], []
    while len(ii) < m:
        a, b = (int(v) for v in rng.integers(0, n, size=2))
        if a == b:
            continue
        key = (min(a, b), max(a, b))
        if key in seen:
            continue
        seen.add(key)
        ii.append(key[0])
        jj.append(key[1])
    if weights == "one":
        w = np.ones(m, dtype=np.int64)
    elif weights == "int":
        w = rng.integers(1, 4, size=m) * (2 * rng.integers(0, 2, size=m) - 1)
    else:
        w = 2 * rng.integers(0, 2, size=m) - 1
    h = rng.integers(-hmax, hmax + 1, size=n) if hmax > 0 else None
    return graph_from_edges(n, ii, jj, w, h)
