"""Closed forms printed in the paper, used to pin the oracle.

* p(theta) = erfc(theta/sqrt 2)/2 (Results, "Spike encoding statistics", and Methods,
  "Input encoding").
* Cascade noise statistics (Eq. cascade): p_1 = P(Bin(C, p_0) >= K_L),
  p_{l+1} = P(Bin(B_l, p_l) >= K_I), where B_l is the fan-in of level l+1.
* SNR_A(W) = sqrt(W) (p_sig - p_noise) / sqrt(p_noise (1 - p_noise)) (Eq. snr_A).
"""
from __future__ import annotations

import math


def p_fire(theta: float) -> float:
    """Per-channel fire probability of the delta encoder on zero-mean unit Gaussian z."""
    return 0.5 * math.erfc(theta / math.sqrt(2.0))


def binom_tail(n: int, p: float, k: int) -> float:
    """P(Bin(n, p) >= k), by direct summation."""
    if k <= 0:
        return 1.0
    return sum(math.comb(n, j) * p ** j * (1.0 - p) ** (n - j) for j in range(k, n + 1))


def cascade(p0: float, leaf_fanin: int, fanins, k_leaf: int, k_internal: int) -> list:
    """Per-level fire probabilities [p_1 (leaf), p_2, ..., p_root] of Eq. cascade.

    ``fanins`` lists the fan-in of each level above the leaves, bottom-up."""
    p = binom_tail(leaf_fanin, p0, k_leaf)
    out = [p]
    for b in fanins:
        p = binom_tail(b, p, k_internal)
        out.append(p)
    return out


def snr_binary(width: int, p_sig: float, p_noise: float) -> float:
    """Eq. snr_A: matched-filter S/N of a Bernoulli root output over a width-W boxcar."""
    return math.sqrt(width) * (p_sig - p_noise) / math.sqrt(p_noise * (1.0 - p_noise))
