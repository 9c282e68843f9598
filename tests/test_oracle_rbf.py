"""Pins of the oracle RBF interpolant (the interpolated initial guess of Sec. 5): it interpolates the data
at the sampled points, reproduces functions linear in the standardised features (its polynomial part),
and equals scipy's RBFInterpolator with the cubic kernel and a degree-1 polynomial on the same features."""
import numpy as np
import pytest

from oracle import rbf as ORBF


def _samples(K=14, R=4, N=5, seed=0):
    rng = np.random.default_rng(seed)
    ss = np.exp(rng.uniform(0.0, 6.0, (K, R)))
    sa = rng.uniform(0.05, 0.5, (K, R))
    sol = rng.standard_normal((K, N))
    return ss, sa, sol


def test_interpolates_the_samples():
    ss, sa, sol = _samples()
    f = ORBF.Rbf(ss, sa, sol)
    for k in range(len(ss)):
        assert np.allclose(f(ss[k], sa[k]), sol[k], rtol=0, atol=1e-9 * np.abs(sol).max())


def test_reproduces_linear_functions_of_the_features():
    ss, sa, _ = _samples(K=16)
    X = ORBF.features(ss, sa)
    a = np.random.default_rng(1).standard_normal(X.shape[1])
    data = np.stack([X @ a + 2.5, -(X @ a)], axis=1)
    f = ORBF.Rbf(ss, sa, data)
    rng = np.random.default_rng(2)
    for _ in range(5):
        qs = np.exp(rng.uniform(0.0, 6.0, 4))
        qa = rng.uniform(0.05, 0.5, 4)
        x = ORBF.features(qs, qa)
        assert np.allclose(f(qs, qa), [x @ a + 2.5, -(x @ a)], atol=1e-9)


def test_matches_scipy_rbf_interpolator():
    interp = pytest.importorskip("scipy.interpolate")
    ss, sa, sol = _samples(K=20)
    f = ORBF.Rbf(ss, sa, sol)
    Xs = (ORBF.features(ss, sa) - f.mean) / f.scale
    ref = interp.RBFInterpolator(Xs, sol, kernel="cubic", degree=1)
    rng = np.random.default_rng(3)
    for _ in range(5):
        qs = np.exp(rng.uniform(0.0, 6.0, 4))
        qa = rng.uniform(0.05, 0.5, 4)
        x = (ORBF.features(qs, qa) - f.mean) / f.scale
        assert np.allclose(f(qs, qa), ref(x[None, :])[0], rtol=1e-9, atol=1e-11)
