import numpy as np

from paper_2406_16238_b300.analysis import error_bar, reblock


def test_reblocking_recovers_the_error_of_an_ar1_series():
    rng = np.random.default_rng(0)
    phi, n = 0.9, 2 ** 16
    x = np.empty(n)
    x[0] = 0.0
    eps = rng.standard_normal(n)
    for i in range(1, n):
        x[i] = phi * x[i - 1] + eps[i]
    # exact variance of the mean of an AR(1) series: sigma^2/(1-phi^2) * (1+phi)/(1-phi) / n
    exact = np.sqrt(1.0 / (1 - phi ** 2) * (1 + phi) / (1 - phi) / n)
    eb = error_bar(x)
    assert 0.7 * exact < eb < 1.3 * exact
    naive = x.std(ddof=1) / np.sqrt(n)
    assert eb > 2.5 * naive


def test_uncorrelated_series():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(4096)
    eb = error_bar(x)
    assert abs(eb - 1 / 64) < 0.3 / 64
    assert reblock(x)[0][1] == 4096
