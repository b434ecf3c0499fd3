"""The seeded input recipes (host only, no GPU): the cfg5 serving mix follows
its stated distribution, is reproducible from its seed, and the cfg4
right-hand-side coefficients are the stated N(0, 1) draws of seed 3."""
import numpy as np

from paper_2201_05413_gb300.workloads import multi_rhs_coefficients, serving_requests


def test_serving_mix_follows_the_cfg5_recipe():
    reqs = serving_requests(10000, seed=4)
    assert len(reqs) == 10000
    dims = np.array([r["dim"] for r in reqs])
    assert abs((dims == 2).mean() - 0.70) < 0.02          # 70 % 2D, 30 % 3D
    deg = np.array([r["degree"] for r in reqs])
    assert set(deg) == {1, 2} and abs((deg == 1).mean() - 0.5) < 0.02
    ks = np.array([r["k"] for r in reqs])
    assert ks.min() == 1 and ks.max() == 8 and abs(ks.mean() - 4.5) < 0.1
    c2 = np.array([r["cells"] for r in reqs if r["dim"] == 2])
    c3 = np.array([r["cells"] for r in reqs if r["dim"] == 3])
    assert c2.min() >= 32 and c2.max() <= 1024 and c3.min() >= 16 and c3.max() <= 128
    # log-uniform: the median of n sits near the geometric mean of the range
    assert abs(np.log(np.median(c2)) - 0.5 * np.log(32 * 1024)) < 0.1
    assert abs(np.log(np.median(c3)) - 0.5 * np.log(16 * 128)) < 0.1
    for r in reqs[:50]:
        ncoef = 10 if r["dim"] == 2 else 4
        assert r["coef"].shape == (r["k"], ncoef)
        assert r["jitter"] == (1 if r["dim"] == 2 else 0)
    assert [r["seed"] for r in reqs[:5]] == [0, 1, 2, 3, 4]  # mesh seed = request index


def test_serving_mix_is_reproducible_and_arrivals_poisson():
    a = serving_requests(200, seed=4, rate_per_s=2.0)
    b = serving_requests(200, seed=4, rate_per_s=2.0)
    assert [(r["dim"], r["cells"], r["k"]) for r in a] == [(r["dim"], r["cells"], r["k"]) for r in b]
    assert all(np.array_equal(x["coef"], y["coef"]) for x, y in zip(a, b))
    t = np.array([r["t"] for r in a])
    assert np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    assert 0.35 < gaps.mean() < 0.65  # exponential gaps of mean 1 / rate


def test_cfg4_coefficients():
    c = multi_rhs_coefficients(32)
    assert c.shape == (32, 10)
    assert np.array_equal(c, np.random.default_rng(3).standard_normal((32, 10)))
