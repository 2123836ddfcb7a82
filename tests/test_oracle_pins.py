"""Pins for the CPU oracle, each against something other than the oracle itself.

* Philox4x32-10: the published known-answer vectors (golden file).
* Thresholds: a 60-digit decimal evaluation of floor(exp(-beta d) 2^32).
* Eq. 1 / Eq. 2: the edge-list forms, the identity cut = (W - H)/2, flip symmetry.
* The annealer: a pure-Python restatement that evaluates dE as a difference of
  whole-lattice energies (bit-exact on tiny tori), brute force over all 2^16
  states of a 4x4 torus, the exact Boltzmann distribution at fixed beta,
  zero-temperature monotonicity, gauge invariance, resume, and incremental
  versus recomputed local fields.
* Eq. 3-5: the printed rows of Table I.
* The 16-bit draw mode (a variant of this project): its thresholds against a
  high-precision evaluation of floor(exp(-beta d) 2^16), its draws against
  the Python Philox, the whole annealer against the full-energy restatement,
  and the Boltzmann distribution at fixed beta.
"""
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
import synth
from tests import _pyref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


# ---------------------------------------------------------------- Philox
@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers_c(ctr, key, expect):
    assert oracle.philox4x32_10(ctr, key) == expect


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers_python(ctr, key, expect):
    assert _pyref.philox(ctr, key) == expect


def test_philox_c_matches_python_on_random_counters():
    rng = np.random.default_rng(7)
    for _ in range(200):
        ctr = [int(v) for v in rng.integers(0, 2**32, 4, dtype=np.uint64)]
        key = [int(v) for v in rng.integers(0, 2**32, 2, dtype=np.uint64)]
        assert oracle.philox4x32_10(ctr, key) == _pyref.philox(ctr, key)


# ---------------------------------------------------------------- thresholds
def _exact_threshold(beta, d):
    getcontext().prec = 60
    v = (-(Decimal(beta) * d)).exp() * (Decimal(2) ** 32)
    f = int(v)  # floor for v >= 0
    return min(f, 2**32 - 1), v


def test_thresholds_against_high_precision():
    betas = np.concatenate([synth.linear_betas(0.1, 3.0, 997), [1e-12, 1e-3, 7.5, 40.0]])
    T4, T8 = oracle.thresholds(betas)
    for k, b in enumerate(betas):
        for d, T in ((4, T4[k]), (8, T8[k])):
            exact, v = _exact_threshold(float(b), d)
            # FP64 exp is within a few ulp; only values within 1e-5 of an integer may round either way
            if abs(v - int(v)) > Decimal("1e-5") and abs(v - int(v) - 1) > Decimal("1e-5"):
                assert int(T) == exact, (b, d, int(T), exact)
            else:
                assert abs(int(T) - exact) <= 1


def test_threshold_limits_and_order():
    T4, T8 = oracle.thresholds(np.array([1e-300, 0.5, 3.0, 6.0, np.inf]))
    assert T4[0] == 2**32 - 1 and T8[0] == 2**32 - 1          # beta -> 0: always accept
    assert T4[-1] == 0 and T8[-1] == 0                       # beta = inf: never accept uphill
    assert all(T8 <= T4)
    assert all(np.diff(T4.astype(np.int64)) <= 0)
    # exp(-24) * 2^32 = 0.162...: floors to 0 at beta = 3 for dE = 8
    assert T8[2] == 0 and T4[2] == int(math.floor(math.exp(-12.0) * 2**32))
    with pytest.raises(ValueError):
        oracle.thresholds(np.array([0.0]))
    with pytest.raises(ValueError):
        oracle.thresholds(np.array([np.nan]))


def _exact_threshold16(beta, d):
    getcontext().prec = 60
    v = (-(Decimal(beta) * d)).exp() * (Decimal(2) ** 16)
    return min(int(v), 2**16 - 1), v


def test_thresholds16_against_high_precision():
    betas = np.concatenate([synth.linear_betas(0.1, 3.0, 997), [1e-12, 1e-3, 1.5, 7.5, 40.0]])
    T4, T8 = oracle.thresholds(betas, draw_bits=16)
    for k, b in enumerate(betas):
        for d, T in ((4, T4[k]), (8, T8[k])):
            exact, v = _exact_threshold16(float(b), d)
            if abs(v - int(v)) > Decimal("1e-9") and abs(v - int(v) - 1) > Decimal("1e-9"):
                assert int(T) == exact, (b, d, int(T), exact)
            else:
                assert abs(int(T) - exact) <= 1


def test_thresholds16_limits():
    T4, T8 = oracle.thresholds(np.array([1e-300, 0.5, 2.0, np.inf]), draw_bits=16)
    assert T4[0] == 2**16 - 1 and T8[0] == 2**16 - 1
    assert T4[-1] == 0 and T8[-1] == 0
    # beta 2: exp(-8) 2^16 = 21.98..., exp(-16) 2^16 = 0.0074...
    assert T4[2] == 21 and T8[2] == 0
    # beta 0.5: exp(-2) 2^16 = 8869.2..., exp(-4) 2^16 = 1200.3...
    assert T4[1] == 8869 and T8[1] == 1200
    assert all(T8 <= T4)


def test_draw16_matches_python_philox_halves():
    rng = np.random.default_rng(17)
    for _ in range(300):
        i, k = (int(v) for v in rng.integers(0, 2**32, 2, dtype=np.uint64))
        t = int(rng.integers(0, 4096))
        seed = int(rng.integers(0, 2**63, dtype=np.uint64))
        assert oracle.decision_draw(i, k, t, seed, 16) == _pyref.draw16(i, k, t, seed)
        assert oracle.decision_draw(i, k, t, seed, 32) == _pyref.draw(i, k, t, seed)
    # the eight trials of one block cover its four words, low half first
    blk = _pyref.philox((5, 9, 3, 0), (0x11, 0x22))
    halves = [w >> (16 * h) & 0xFFFF for w in blk for h in (0, 1)]
    assert [oracle.decision_draw(5, 9, 24 + j, 0x22_0000_0011, 16) for j in range(8)] == halves


# ---------------------------------------------------------------- Eq. 1 / Eq. 2
@pytest.mark.parametrize("X,Y,seed", [(4, 4, 1), (6, 4, 2), (10, 8, 3), (50, 50, 1)])
def test_cut_energy_identities(X, Y, seed):
    inst = synth.torus_instance(X, Y, seed)
    edges = oracle.torus_edges(X, Y, inst["w_right"], inst["w_down"])
    W = int(edges[2].sum())
    S = synth.random_spins(20, X * Y, seed + 100)
    for s in S:
        c = oracle.cut_csr(inst, s)
        h = oracle.energy_csr(inst, s)
        assert c == int(oracle.cut_eq1(edges, s))            # Eq. 1 over the edge list
        assert h == int(oracle.energy_eq2(edges, s))         # Eq. 2 over the edge list
        assert 2 * c == W - h                                 # cut = (W - H)/2
        assert oracle.cut_csr(inst, -s) == c                  # global flip symmetry
    # |E| = 2n on the torus (Table I: |E| = 2|V|)
    assert len(edges[2]) == 2 * X * Y


def test_paper_cut_energy_pairs_have_integer_weight_sums():
    # The best cuts 7008, 9940, 14060 are printed with energies -14022, -19672,
    # -28086 (Section III).  With cut = (W - H)/2, W = H + 2 cut must be an
    # integer sum of |E| = 2n weights of +-1, i.e. of the parity of |E|.
    for cut, H, nE in ((7008, -14022, 20000), (9940, -19672, 28000), (14060, -28086, 40000)):
        W = H + 2 * cut
        assert abs(W) <= nE and (W - nE) % 2 == 0


# ---------------------------------------------------------------- brute force
def test_brute_force_4x4_and_low_temperature_anneal():
    inst = synth.torus_instance(4, 4, 11)
    edges = oracle.torus_edges(4, 4, inst["w_right"], inst["w_down"])
    Emin, Cmax, E, C = oracle.brute_force(edges, 16)
    W = int(edges[2].sum())
    assert 2 * Cmax == W - Emin
    betas = synth.linear_betas(0.1, 3.0, 400)
    spins, cuts = oracle.anneal(inst, betas, seed=5, t_count=64)
    assert cuts.max() == Cmax
    assert (cuts == Cmax).mean() > 0.5
    for s, c in zip(spins, cuts):
        assert oracle.cut_csr(inst, s) == c


# ---------------------------------------------------------------- pure-Python equality
@pytest.mark.parametrize("bits", [32, 16])
@pytest.mark.parametrize("X,Y,seed,S,trials", [(4, 4, 3, 6, 5), (6, 4, 4, 4, 4), (4, 6, 5, 5, 3), (4, 4, 6, 3, 17)])
def test_oracle_equals_full_energy_restatement(X, Y, seed, S, trials, bits):
    inst = synth.torus_instance(X, Y, seed)
    edges = oracle.torus_edges(X, Y, inst["w_right"], inst["w_down"])
    betas = synth.linear_betas(0.2, 1.5, S)
    ref = _pyref.anneal_full_energy(X, Y, edges, betas, seed=0x1234_5678_9ABC, trials=trials,
                                    sweep_offset=7, draw_bits=bits)
    got, cuts = oracle.anneal(inst, betas, seed=0x1234_5678_9ABC, t_count=trials, sweep_offset=7,
                              draw_bits=bits)
    np.testing.assert_array_equal(got, ref)
    for s, c in zip(got, cuts):
        assert c == int(oracle.cut_eq1(edges, s))


# ---------------------------------------------------------------- Boltzmann
@pytest.mark.parametrize("bits", [32, 16])
def test_fixed_beta_samples_follow_boltzmann(bits):
    """Each Metropolis update leaves exp(-beta H) invariant, so after many sweeps
    independent trials sample the exact distribution (chi-square on energies).
    The 16-bit mode quantises each acceptance probability down by < 2^-16."""
    inst = synth.torus_instance(4, 4, 21)
    edges = oracle.torus_edges(4, 4, inst["w_right"], inst["w_down"])
    _, _, E, _ = oracle.brute_force(edges, 16)
    beta = 0.45
    p_state = oracle.boltzmann(E, beta)
    levels, inv = np.unique(E, return_inverse=True)
    p_level = np.bincount(inv, weights=p_state)
    trials = 6000
    spins, _ = oracle.anneal(inst, np.full(60, beta), seed=99, t_count=trials, draw_bits=bits)
    got = np.array([oracle.energy_csr(inst, s) for s in spins])
    obs = np.array([(got == L).sum() for L in levels], dtype=np.float64)
    exp = p_level * trials
    keep = exp >= 5
    chi2 = (((obs[keep] - exp[keep]) ** 2) / exp[keep]).sum() + 0.0
    dof = keep.sum() - 1
    # 99.99% quantile of chi-square ~ dof + 6 sqrt(2 dof) for these dof
    assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (chi2, dof)
    # the mean energy must match too (a flipped dE sign would push it far up)
    assert abs(got.mean() - (p_state * E).sum()) < 0.25


def test_zero_temperature_never_increases_energy():
    inst = synth.torus_instance(10, 8, 31)
    s0 = synth.random_spins(8, 80, 3)
    cur = s0
    prev = np.array([oracle.energy_csr(inst, s) for s in cur])
    for k in range(12):
        cur, _ = oracle.anneal(inst, np.array([np.inf]), seed=4, t_count=8, sweep_offset=k, init=cur)
        e = np.array([oracle.energy_csr(inst, s) for s in cur])
        assert (e <= prev).all()
        prev = e


# ---------------------------------------------------------------- invariances
def test_gauge_transform_is_exact():
    X, Y = 8, 6
    inst = synth.torus_instance(X, Y, 41)
    rng = np.random.default_rng(5)
    tau = (2 * rng.integers(0, 2, size=(Y, X)) - 1).astype(np.int8)
    wr = inst["w_right"] * tau * np.roll(tau, -1, axis=1)
    wd = inst["w_down"] * tau * np.roll(tau, -1, axis=0)
    row_ptr, col, J = synth.torus_csr(X, Y, wr, wd)
    inst2 = dict(inst, w_right=wr, w_down=wd, row_ptr=row_ptr, col=col, J=J)
    s0 = synth.random_spins(6, X * Y, 8)
    betas = synth.linear_betas(0.3, 2.0, 40)
    a, _ = oracle.anneal(inst, betas, seed=12, t_count=6, init=s0)
    b, _ = oracle.anneal(inst2, betas, seed=12, t_count=6, init=s0 * tau.reshape(-1))
    np.testing.assert_array_equal(b, a * tau.reshape(-1))
    for sa, sb in zip(a, b):
        assert oracle.energy_csr(inst, sa) == oracle.energy_csr(inst2, sb)


def test_resume_is_exact():
    inst = synth.torus_instance(12, 10, 51)
    betas = synth.linear_betas(0.1, 3.0, 50)
    full, fcut = oracle.anneal(inst, betas, seed=77, t_count=9)
    half, _ = oracle.anneal(inst, betas[:20], seed=77, t_count=9)
    rest, rcut = oracle.anneal(inst, betas[20:], seed=77, t_count=9, sweep_offset=20, init=half)
    np.testing.assert_array_equal(full, rest)
    np.testing.assert_array_equal(fcut, rcut)


def test_trial_subsets_are_independent():
    inst = synth.torus_instance(8, 8, 61)
    betas = synth.linear_betas(0.1, 3.0, 30)
    allt, allc = oracle.anneal(inst, betas, seed=3, t_count=13)
    part, pc = oracle.anneal(inst, betas, seed=3, t_begin=5, t_count=6)
    np.testing.assert_array_equal(allt[5:11], part)
    np.testing.assert_array_equal(allc[5:11], pc)


def test_incremental_fields_match_recomputed():
    inst = synth.torus_instance(14, 10, 71)
    betas = synth.linear_betas(0.1, 3.0, 60)
    oracle.anneal(inst, betas, seed=9, t_count=4, check_fields=True)


def test_zero_sweeps_returns_initial_state():
    inst = synth.torus_instance(6, 6, 81)
    s, c = oracle.anneal(inst, np.zeros(0), seed=2, t_count=8)
    for t in range(8):
        for i in range(36):
            bit = _pyref.draw(i, 0xFFFFFFFF, t, 2) >> 31
            assert s[t, i] == (1 if bit else -1)
        assert c[t] == oracle.cut_csr(inst, s[t])


# ---------------------------------------------------------------- Eq. 3-5
def _table1():
    rows = []
    for line in open(os.path.join(GOLDEN, "table1_campaigns.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append(dict(inst=f[0], target=f[1], S=int(f[2]), succ=int(f[3]), n=int(f[4]),
                         stt=float(f[5]), ttt=float(f[6]), ges=float(f[7]), speedup=float(f[8]),
                         flag=f[9], proj_ms=float(f[10]), proj_txt=f[10]))
    return rows


def _sig3(x):
    return float(f"{x:.3g}")


@pytest.mark.parametrize("row", _table1(), ids=lambda r: f"{r['inst']}-{r['target']}")
def test_table1_sweeps_to_target(row):
    Ps = row["succ"] / row["n"]
    if row["flag"] == "garbled":
        assert _sig3(oracle.sweeps_to_target(row["S"], Ps)) != row["stt"]
        assert _sig3(oracle.sweeps_to_target(100000, Ps)) == row["stt"]
    else:
        assert _sig3(oracle.sweeps_to_target(row["S"], Ps)) == row["stt"]
    # projected column: STT x 2 ns, printed with one or two significant digits
    proj = row["stt"] * 2e-9 * 1e3
    assert any(float(f"{proj:.{d}g}") == row["proj_ms"] for d in (1, 2)), (proj, row["proj_txt"])
    if not math.isnan(row["speedup"]):
        assert _sig3(row["ges"] / row["ttt"]) == row["speedup"]


def test_repetitions_edge_cases():
    assert oracle.repetitions(1.0) == 1.0
    assert oracle.repetitions(0.999) == 1.0
    assert math.isinf(oracle.repetitions(0.0))
    assert oracle.target_cut(14060) == 14046       # Table I: ">= 14045.94"
    assert oracle.target_cut(7008) == 7001          # ">= 7000.99"
    assert oracle.target_cut(9940) == 9931          # ">= 9930.06"


# ---------------------------------------------------------------- trajectory read-out
@pytest.mark.parametrize("S,every", [(30, 10), (31, 10), (7, 1), (5, 9)])
def test_trace_points_equal_prefix_runs(S, every):
    """Each traced cut is the Eq. 1 cut of the configuration a separate run of
    the first j sweeps ends in; the best is their maximum, its configuration
    the first reaching it."""
    inst = synth.torus_instance(8, 6, 91)
    edges = oracle.torus_edges(8, 6, inst["w_right"], inst["w_down"])
    betas = synth.linear_betas(0.1, 2.5, S)
    T = 9
    spins, cuts, trace, best, bspins = oracle.anneal_trace(inst, betas, 5, every, t_count=T)
    pts = list(range(every, S + 1, every))
    if not pts or pts[-1] != S:
        pts.append(S)
    assert trace.shape == (len(pts), T)
    prefix = []
    for p, j in enumerate(pts):
        sj, cj = oracle.anneal(inst, betas[:j], 5, t_count=T)
        prefix.append(sj)
        np.testing.assert_array_equal(trace[p], cj)
        for t in range(T):
            assert trace[p, t] == int(oracle.cut_eq1(edges, sj[t]))
    np.testing.assert_array_equal(trace[-1], cuts)
    np.testing.assert_array_equal(best, trace.max(axis=0))
    first = trace.argmax(axis=0)
    for t in range(T):
        np.testing.assert_array_equal(bspins[t], prefix[first[t]][t])
        assert int(oracle.cut_eq1(edges, bspins[t])) == best[t]


def test_best_so_far_is_bounded_by_brute_force():
    inst = synth.torus_instance(4, 4, 11)
    edges = oracle.torus_edges(4, 4, inst["w_right"], inst["w_down"])
    _, Cmax, _, _ = oracle.brute_force(edges, 16)
    betas = synth.linear_betas(0.1, 3.0, 200)
    _, cuts, _, best, _ = oracle.anneal_trace(inst, betas, 3, 7, t_count=40)
    assert (best >= cuts).all() and (best <= Cmax).all()
    # with no sweeps the best is the starting configuration's cut
    s0, c0, tr, b0, bs0 = oracle.anneal_trace(inst, np.zeros(0), 3, 5, t_count=4)
    assert tr.shape == (0, 4)
    np.testing.assert_array_equal(b0, c0)
    np.testing.assert_array_equal(bs0, s0)
