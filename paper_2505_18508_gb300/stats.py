"""Time-to-target statistics of a batch of trials (host side, Section III,
Eq. 3-5), used by the benchmark to turn final cuts into P_s, r, STT and TTT.

* target: the smallest integer cut at or above q * best (the paper quotes
  its 99.9% targets as real thresholds); computed exactly with a rational q;
* P_s: the fraction of trials whose final cut reaches the target;
* r (Eq. 3): repetitions for 99% confidence, ln(0.01) / ln(1 - P_s), at
  least 1; P_s = 1 gives 1 and P_s = 0 gives infinity ("not reached");
* STT = sweeps per trial x r (Eq. 4); TTT = time per trial x r (Eq. 5).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

CONFIDENCE = 0.99


def target_cut(best: int, quality: float = 0.999) -> int:
    q = Fraction(str(quality))
    num = q.numerator * int(best)
    return -((-num) // q.denominator)          # ceiling of q * best, exactly


def success_probability(cuts, target: int) -> float:
    c = np.asarray(cuts).reshape(-1)
    if c.size == 0:
        return 0.0
    return float(np.count_nonzero(c >= target)) / float(c.size)


def repetitions(p_s: float) -> float:
    if p_s >= 1.0:
        return 1.0
    if p_s <= 0.0:
        return math.inf
    return max(1.0, math.log(1.0 - CONFIDENCE) / math.log1p(-p_s))


def sweeps_to_target(sweeps_per_trial: float, p_s: float) -> float:
    return sweeps_per_trial * repetitions(p_s)


def time_to_target(seconds_per_trial: float, p_s: float) -> float:
    return seconds_per_trial * repetitions(p_s)
