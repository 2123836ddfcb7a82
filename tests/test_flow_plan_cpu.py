"""Host logic of the persistent kernel's work split (ising_flow_split, no GPU):
every stacked site word belongs to exactly one CTA, the ranges are balanced
to within one word of weight, the 16-bit mode splits at row boundaries, and
the local-row and segment counts match an independent count."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def ia():
    import __graft_entry__
    from paper_2505_18508_gb300 import build
    build.build()
    import paper_2505_18508_gb300 as ia
    return ia


def _weights(Y, T, G, blk, weighted):
    groups = (T + G - 1) // G
    w = []
    for g in range(groups):
        live = min(G, T - g * G)
        w += [(live + blk - 1) // blk if weighted else 1] * Y
    return np.array(w, dtype=np.int64)


def _local_rows(split, Y, H):
    lrmax = segmax = 0
    for j in range(len(split) - 1):
        lr = nseg = 0
        rows = {}
        for wd in range(split[j], split[j + 1]):
            rows.setdefault(wd // H, 0)
            rows[wd // H] += 1
        groups = {}
        for r in rows:
            groups.setdefault(r // Y, []).append(r)
        for g, rs in groups.items():
            whole = len(rs) == Y and all(rows[r] == H for r in rs)
            lr += len(rs) + (0 if whole else 2)
            nseg += 1
        lrmax, segmax = max(lrmax, lr), max(segmax, nseg)
    return lrmax, segmax


CASES = [
    # X, Y, trials, group trials, draw bits, SMs, weighted
    (200, 100, 1024, 32, 32, 152, True),
    (200, 100, 1024, 32, 16, 152, True),
    (100, 100, 1000, 32, 32, 152, True),
    (8, 6, 37, 32, 32, 152, True),
    (8, 6, 37, 32, 32, 152, False),
    (24, 16, 3000, 8, 32, 152, True),
    (50, 50, 64, 32, 32, 7, True),
    (200, 100, 33, 32, 32, 152, True),
    (64, 48, 96, 32, 16, 152, True),
]


@pytest.mark.parametrize("X,Y,T,G,bits,sms,weighted", CASES)
def test_flow_split_invariants(ia, X, Y, T, G, bits, sms, weighted):
    _check_split(ia, X, Y, T, G, bits, sms, weighted)


def test_flow_split_invariants_random_shapes(ia):
    """The same invariants on 120 random shapes: even sides 4..400, every
    group width and both draw modes, 1..160 SMs, and up to 5,000 trials
    (capped so a case stacks at most 60,000 site words)."""
    rng = np.random.default_rng(2026)
    for _ in range(120):
        bits = int(rng.choice([32, 16]))
        blk = 8 if bits == 16 else 4
        X = 2 * int(rng.integers(2, 201))
        Y = 2 * int(rng.integers(2, 201))
        G = blk * int(rng.integers(1, 32 // blk + 1))
        groups_max = max(1, 60000 // (Y * (X // 2)))
        T = int(rng.integers(1, min(5000, groups_max * G) + 1))
        sms = int(rng.integers(1, 161))
        _check_split(ia, X, Y, T, G, bits, sms, bool(rng.integers(0, 2)))


def _check_split(ia, X, Y, T, G, bits, sms, weighted):
    H = X // 2
    split, lrmax, segmax = ia.flow_split(Y, X, T, G, bits, sms, weighted)
    w = _weights(Y, T, G, 8 if bits == 16 else 4, weighted)
    RT = w.shape[0]
    P = min(sms, RT)
    W = RT * H
    assert split.shape[0] == P + 1 and split[0] == 0 and split[-1] == W
    assert np.all(np.diff(split) > 0)                       # every CTA gets words, none twice
    if bits == 16:
        assert np.all(split % H == 0)                        # row boundaries in the 16-bit mode
    # weight of each range against the ideal share (one word of slack per end;
    # row-boundary splits may miss by up to a row)
    word_w = np.repeat(w, H)
    cumw = np.concatenate([[0], np.cumsum(word_w)])
    share = cumw[-1] / P
    slack = (H if bits == 16 else 1) * w.max() + w.max()
    loads = cumw[split[1:]] - cumw[split[:-1]]
    assert np.all(np.abs(loads - share) <= slack + 1e-9)
    assert (lrmax, segmax) == _local_rows(split, Y, H)


def test_flow_split_headline_balance(ia):
    split, lrmax, segmax = ia.flow_split(100, 200, 1024)
    sizes = np.diff(split)
    assert split.shape[0] == 153 and set(sizes.tolist()) <= {2105, 2106}
    assert segmax <= 2


def test_flow_split_arguments(ia):
    for kw in (dict(draw_bits=8), dict(group_trials=0), dict(group_trials=33)):
        args = dict(Y=10, X=20, trials=64)
        args.update(kw)
        with pytest.raises(ia.IsingError):
            ia.flow_split(**args)


# ---------------------------------------------------------------- batched schedule

def _batch_cfg():
    import synth
    cfg = synth.batched_config()
    return [(c["X"], c["Y"]) for c in cfg], [c["trials"] for c in cfg], [c["sweeps"] for c in cfg]


def test_batch_schedule_covers_every_group_longest_first(ia):
    shapes, trials, sweeps = _batch_cfg()
    per_sm, threads, G, units = ia.batch_schedule(shapes, trials, sweeps)
    assert (per_sm, threads) == (1, 1024)        # large tori: one 1,024-thread CTA per SM
    assert np.all(G % 4 == 0) and np.all((G >= 4) & (G <= 32))
    want = {(q, g) for q in range(len(shapes)) for g in range((trials[q] + G[q] - 1) // G[q])}
    got = [tuple(u) for u in units.tolist()]
    assert len(got) == len(want) and set(got) == want
    # longest first: n (S + 1) x (3 + Philox blocks of the unit), non-increasing
    Gi = [int(v) for v in G]
    cost = [_unit_cost(shapes, sweeps, trials, Gi, q, g, 4) for q, g in got]
    assert all(a >= b for a, b in zip(cost, cost[1:]))
    # every 32-trial unit of this batch fits in a CTA's average share: all 32
    share = sum(x * y * s * t for (x, y), s, t in zip(shapes, sweeps, trials)) / (152 * per_sm)
    assert max(x * y * s * 32 for (x, y), s in zip(shapes, sweeps)) <= share
    assert Gi == [32] * len(shapes)


def _unit_cost(shapes, sweeps, trials, G, q, g, blk):
    n = shapes[q][0] * shapes[q][1]
    live = min(G[q], trials[q] - g * G[q])
    return n * (sweeps[q] + 1) * (3 + (live + blk - 1) // blk)


def _lpt_makespan(costs, ctas):
    """List scheduling in the given order onto `ctas` identical CTAs."""
    import heapq
    busy = [0.0] * ctas
    for c in costs:
        heapq.heapreplace(busy, busy[0] + c)
    return max(busy)


@pytest.mark.parametrize("case", ["8x200x100", "mixed", "8x200x100_16bit"])
def test_batch_schedule_unit_width_minimises_the_makespan(ia, case):
    """Instances whose 32-trial unit exceeds a CTA's average share take the
    unit width (a multiple of the Philox block) whose longest-first schedule
    ends first, ties to the wider; the others keep 32.  Checked against a
    separate list-scheduling simulation of every candidate width."""
    draw_bits = 16 if case.endswith("16bit") else 32
    blk = 8 if draw_bits == 16 else 4
    if case.startswith("8x200x100"):
        shapes, trials, sweeps = [(200, 100)] * 8, [512] * 8, [30000] * 8
    else:
        shapes = [(200, 100)] * 4 + [(50, 100)] * 20
        trials, sweeps = [512] * 4 + [64] * 20, [20000] * 4 + [2000] * 20
    per_sm, _, G, units = ia.batch_schedule(shapes, trials, sweeps, draw_bits=draw_bits)
    ctas = 152 * per_sm
    total = sum(x * y * s * t for (x, y), s, t in zip(shapes, sweeps, trials))
    large = [x * y * s * 32 > total / ctas for (x, y), s in zip(shapes, sweeps)]
    assert any(large)
    spans = {}
    for g in range(32, blk - 1, -blk):
        Gc = [g if large[q] else 32 for q in range(len(shapes))]
        cs = sorted((_unit_cost(shapes, sweeps, trials, Gc, q, k, blk)
                     for q in range(len(shapes)) for k in range(-(-trials[q] // Gc[q]))), reverse=True)
        spans[g] = _lpt_makespan(cs, ctas)
    best = min(spans.values())
    g_want = max(g for g, v in spans.items() if v == best)
    Gi = [int(v) for v in G]
    assert Gi == [g_want if large[q] else 32 for q in range(len(shapes))]
    assert units.shape[0] == sum(-(-t // g) for t, g in zip(trials, Gi))
    if case == "8x200x100":
        assert g_want == 28 and units.shape[0] == 152        # 18 x 28 + 8 trials per instance
        assert spans[28] < spans[32] < spans[24]


def test_batch_schedule_small_tori_take_two_ctas_per_sm(ia):
    shapes = [(20, 20)] * 8
    per_sm, threads, G, units = ia.batch_schedule(shapes, [64] * 8, [500] * 8)
    assert (per_sm, threads) == (2, 512)
    assert units.shape[0] == sum((64 + g - 1) // g for g in G)


def test_batch_schedule_fixed_shapes_and_16_bit(ia):
    shapes, trials, sweeps = _batch_cfg()
    per_sm, threads, G, _ = ia.batch_schedule(shapes, trials, sweeps, group_trials=8, ctas_per_sm=2)
    assert (per_sm, threads) == (2, 512) and np.all(G == 8)
    _, _, G16, _ = ia.batch_schedule(shapes, trials, sweeps, draw_bits=16)
    assert np.all(G16 % 8 == 0)
    with pytest.raises(ia.IsingError):
        ia.batch_schedule(shapes, trials, sweeps, draw_bits=16, group_trials=12)
    with pytest.raises(ia.IsingError):
        ia.batch_schedule([(5, 8)], [32], [10])


def test_batch_schedule_degenerate_batches(ia):
    per_sm, threads, G, units = ia.batch_schedule([], [], [])
    assert G.shape == (0,) and units.shape == (0, 2)
    _, _, G, units = ia.batch_schedule([(8, 8)], [0], [10])            # no trials: no units
    assert units.shape == (0, 2)
    _, _, G, units = ia.batch_schedule([(8, 8), (200, 100)], [0, 5], [10, 0])
    assert [tuple(u) for u in units.tolist()] == [(1, 0)]             # 5 trials, no sweeps: one unit
    _, _, G, units = ia.batch_schedule([(200, 100)], [3], [100])
    assert G.tolist() == [32] and units.tolist() == [[0, 0]]           # every width gives one unit: the widest


def test_batch_schedule_random_batches(ia):
    """40 random uneven batches (1-20 tori of even sides 4..200, 1-600
    trials, 1-3,000 sweeps, both draw modes): every unit once, longest first
    under the cost model, and each large instance's width the one whose
    list schedule ends first (ties to the wider), per a separate simulation."""
    rng = np.random.default_rng(11)
    for _ in range(40):
        m = int(rng.integers(1, 21))
        bits = int(rng.choice([32, 16]))
        blk = 8 if bits == 16 else 4
        shapes = [(2 * int(rng.integers(2, 101)), 2 * int(rng.integers(2, 101))) for _ in range(m)]
        trials = [int(rng.integers(1, 601)) for _ in range(m)]
        sweeps = [int(rng.integers(1, 3001)) for _ in range(m)]
        per_sm, _, G, units = ia.batch_schedule(shapes, trials, sweeps, draw_bits=bits)
        Gi = [int(v) for v in G]
        got = [tuple(u) for u in units.tolist()]
        assert sorted(got) == sorted((q, g) for q in range(m) for g in range(-(-trials[q] // Gi[q])))
        cost = [_unit_cost(shapes, sweeps, trials, Gi, q, g, blk) for q, g in got]
        assert all(a >= b for a, b in zip(cost, cost[1:]))
        ctas = 152 * per_sm
        total = sum(x * y * s * t for (x, y), s, t in zip(shapes, sweeps, trials))
        large = [x * y * s * 32 > total / ctas for (x, y), s in zip(shapes, sweeps)]
        if not any(large):
            assert Gi == [32] * m
            continue
        spans = {}
        for g in range(32, blk - 1, -blk):
            Gc = [g if large[q] else 32 for q in range(m)]
            cs = sorted((_unit_cost(shapes, sweeps, trials, Gc, q, k, blk)
                         for q in range(m) for k in range(-(-trials[q] // Gc[q]))), reverse=True)
            spans[g] = _lpt_makespan(cs, ctas)
        best = min(spans.values())
        g_want = max(g for g, v in spans.items() if v == best)
        assert Gi == [g_want if large[q] else 32 for q in range(m)]
