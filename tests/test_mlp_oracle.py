"""Pins of the FP64 network oracle (oracle/mlp.py)."""
import math

import numpy as np
from scipy.special import erf

from oracle import mlp
from tests import pins


def test_gelu_tanh_form_against_erf_form():
    """The tanh form approximates z Phi(z) (Hendrycks and Gimpel) to 1e-3."""
    z = np.linspace(-6, 6, 2001)
    exact = 0.5 * z * (1 + erf(z / math.sqrt(2)))
    assert np.max(np.abs(mlp.gelu(z) - exact)) < 1e-3
    assert mlp.gelu(0.0) == 0.0
    assert abs(mlp.gelu(1.0) - 0.8411919906082768) < 1e-15  # the tanh form at 1


def test_gelu_grad_differences():
    z = np.linspace(-5, 5, 101)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-7, atol=1e-8)


def test_backward_central_differences():
    rng = np.random.default_rng(0)
    n_in, hid, n_out, B = 7, 5, 4, 3
    n_p = hid * n_in + hid + hid * hid + hid + n_out * hid + n_out
    p = rng.standard_normal(n_p) * 0.5
    U = rng.standard_normal((B, n_in))
    dY = rng.standard_normal((B, n_out))
    Y, cache = mlp.forward(p, U, n_in, hid, n_out)
    g = mlp.backward(p, cache, dY, n_in, hid, n_out)
    f = lambda q: np.array([float(np.sum(mlp.forward(q, U, n_in, hid, n_out)[0] * dY))])
    fd = pins.central_diff(f, p, h=1e-3)[0]
    np.testing.assert_allclose(g, fd, rtol=1e-8, atol=1e-9)


def test_inputs_normalisation():
    pd0 = np.array([0.5, 0.0, 0.2])
    qd0 = np.array([0.15, 0.0, 0.06])
    pd = np.array([[0.6, 0.0, 0.2]])
    qd = np.array([[0.12, 0.0, 0.066]])
    U = mlp.inputs(pd, qd, pd0, qd0, 8)
    np.testing.assert_allclose(U[0], [1.0, 0.0, 0.0, -1.0, 0.0, 0.5, 0.0, 0.0], atol=1e-12)

