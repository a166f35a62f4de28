"""Host-side statistics for QMC energy series (error bars by reblocking).

The paper's driver writes per-block energies and analyses them by reblocking
(Flyvbjerg & Petersen, J. Chem. Phys. 91, 461 (1989)): the series is
repeatedly averaged in pairs; the naive standard error of the blocked series
grows until blocks are longer than the autocorrelation time and then
plateaus.  The error bar is taken at the first blocking level whose error
estimate agrees, within its own uncertainty, with every later one.
"""
from __future__ import annotations

import numpy as np


def reblock(series):
    """[(level, nblocks, stderr, stderr_of_stderr)] for successive pairwise blockings."""
    x = np.asarray(series, dtype=np.float64)
    out = []
    level = 0
    while x.size >= 2:
        n = x.size
        se = x.std(ddof=1) / np.sqrt(n)
        out.append((level, n, se, se / np.sqrt(2.0 * (n - 1))))
        if n < 4:
            break
        x = 0.5 * (x[: n // 2 * 2 : 2] + x[1 : n // 2 * 2 : 2])
        level += 1
    return out


def error_bar(series):
    """Plateau estimate of the standard error of the mean of a correlated series."""
    levels = reblock(series)
    if not levels:
        return float("nan")
    usable = [lv for lv in levels if lv[1] >= 8]      # too few blocks carry no information
    for i, (_, n, se, dse) in enumerate(usable):
        if all(abs(se - s2) <= 2.0 * (dse + d2) for (_, _, s2, d2) in usable[i + 1:]):
            return float(se)
    return float(max(lv[2] for lv in usable)) if usable else float(levels[0][2])


def energy_series(sums):
    """E_k = ENumer_k / EDenom_k from the estimator sums [nmeas, 4]."""
    sums = np.asarray(sums)
    return sums[:, 0] / sums[:, 1]
