"""Noise-free likelihood and the Fisher-Gaussian posterior for (lambda, beta, psi, t_c) with the
other parameters at their injected values (Sec. 3.3, without the stochastic sampler): the
noise-free log-likelihood -1/2 <s(theta) - s(theta0)|s(theta) - s(theta0)> agrees with its
quadratic Fisher form near theta0, and draws from N(theta0, F^-1) give -2 log L ~ chi^2_4."""
import numpy as np
import pytest

from paper_2602_12011_gb300 import workloads as W

pytestmark = pytest.mark.gpu

IDX = [7, 8, 9, 10]   # lambda, beta, psi, t_c


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2602_12011_gb300 import build as B
    from paper_2602_12011_gb300 import _lib as L
    B.build()
    T = 2.0 ** 20
    k0, nb = W.grid(T)
    th0 = W.theta_injection(T)
    d = L.Detector(W.LISA, T, k0, nb)
    d.inject(th0, W.MODE_ALL, None)           # noise-free data s(theta0)
    return L, d, th0


def test_noise_free_loglike_is_zero_at_truth(setup):
    L, d, th0 = setup
    r = L.loglike([d], th0[None, :], W.MODE_ALL, dhhh=True)
    hh = r["dhhh"][0, :, :, 1].sum()
    assert abs(r["logl"][0]) <= 1e-10 * (2 * hh)


def test_noise_free_loglike_matches_fisher_quadratic_form(setup):
    L, d, th0 = setup
    cov, _ = L.fisher_gaussian([d], th0, W.MODE_ALL, IDX)
    F = np.linalg.inv(cov)
    rng = np.random.default_rng(4)
    sig = np.sqrt(np.diag(cov))
    th = np.repeat(th0[None, :], 12, axis=0)
    dirs = rng.standard_normal((12, 4)) * sig * 0.5
    th[:, IDX] += dirs
    ll = L.loglike([d], th, W.MODE_ALL)["logl"]
    quad = -0.5 * np.einsum("ni,ij,nj->n", dirs, F, dirs)
    np.testing.assert_allclose(ll, quad, rtol=2e-2)


def test_fisher_gaussian_draws_give_chi2(setup):
    L, d, th0 = setup
    z = np.random.default_rng(5).standard_normal((512, 4))
    cov, samples = L.fisher_gaussian([d], th0, W.MODE_ALL, IDX, z)
    assert np.all(np.linalg.eigvalsh(cov) > 0)
    np.testing.assert_array_equal(samples[:, [0, 1, 2, 3, 4, 5, 6]], np.repeat(th0[None, :7], 512, axis=0))
    emp = np.cov((samples[:, IDX] - th0[IDX]).T)
    np.testing.assert_allclose(np.diag(emp), np.diag(cov), rtol=0.2)
    ll = L.loglike([d], samples, W.MODE_ALL)["logl"]
    chi2 = -2 * ll
    assert abs(chi2.mean() - 4.0) < 0.6            # chi^2 with 4 dof: mean 4, std of mean 0.125
    assert abs(chi2.var() - 8.0) < 3.0
