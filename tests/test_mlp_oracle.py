"""Pins of the FP64 network oracle (oracle/mlp.py)."""
import math

import pytest

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



# --- the output map point() and the loss: a two-bus lossless line whose
# flows, rows and violations are textbook closed forms (Sec. IV-A's
# constraint violation; the output map and loss of the learned warm start)

XK = 0.2  # series reactance of the lossless line (r = 0, b = 0, tap 1, no shift)


def _two_bus(rate):
    from tests.test_oracle_pins import tiny
    g = tiny(2, [(0, 1, 0.0, XK, 0.0, 1.0, 0.0, rate)], [(0, 0.07, 12.0, 0.5)], [(1, 0.6, 0.18)])
    # asymmetric generator limits, so that a dropped half-range factor or a
    # mid-point of the wrong limits shows
    return g.copy(gen_pmin=np.array([0.2]), gen_pmax=np.array([1.8]),
                  gen_qmin=np.array([-0.6]), gen_qmax=np.array([1.0]))


def _y(nb, ng, ya, yv, yp, yq, fill=7.0):
    """Network output with the four blocks at offsets 0, nbp, 2 nbp, 2 nbp + ngp
    (nbp, ngp = nb, ng rounded up to 128) and every padding entry = fill."""
    nbp, ngp = mlp.pad(nb), mlp.pad(ng)
    y = np.full(2 * nbp + 2 * ngp, fill)
    y[:nb] = ya
    y[nbp:nbp + nb] = yv
    y[2 * nbp:2 * nbp + ng] = yp
    y[2 * nbp + ngp:2 * nbp + ngp + ng] = yq
    return y


def _lossless_flows(va, vm):
    d = va[0] - va[1]
    vf, vt = vm
    s = vf * vt * math.sin(d) / XK
    c = vf * vt * math.cos(d) / XK
    return d, (s, vf * vf / XK - c), (-s, vt * vt / XK - c)  # (P, Q) at the from and to ends


def test_point_output_map_two_bus(oracle_mod):
    """va = s ya with va_ref = 0, vm = mid + yv, pg/qg = mid + half range * y,
    and p, q = the textbook lossless-line flows at (va, vm)."""
    g = _two_bus(rate=2.0)
    O = oracle_mod.Oracle(g)
    y = _y(2, 1, ya=[0.3, -0.5], yv=[0.05, -0.02], yp=[0.25], yq=[-0.4])
    x = mlp.point(g, y, 0.4, O)
    va, vm, pg, qg = x[0:2], x[2:4], x[4], x[5]
    assert va[0] == 0.0 and va[1] == pytest.approx(-0.2, abs=1e-16)  # bus 0 is the reference
    np.testing.assert_allclose(vm, [1.05, 0.98], rtol=0, atol=1e-15)
    assert pg == pytest.approx(1.0 + 0.8 * 0.25, abs=1e-15)   # mid 1.0, half range 0.8
    assert qg == pytest.approx(0.2 + 0.8 * -0.4, abs=1e-15)   # mid 0.2, half range 0.8
    _, (pf, qf), (pt, qt) = _lossless_flows(va, vm)
    # arcs: 0 = the from-end of branch 0, 1 = its to-end; x = [.., p0, p1, q0, q1]
    np.testing.assert_allclose(x[6:10], [pf, pt, qf, qt], rtol=1e-14, atol=1e-15)


def test_point_ignores_padding():
    """Changing only the padding of y leaves the point unchanged (the blocks
    are read at the padded offsets)."""
    import oracle
    g = _two_bus(rate=2.0)
    O = oracle.Oracle(g)
    a = mlp.point(g, _y(2, 1, [0.1, 0.2], [0.0, 0.01], [0.5], [0.5], fill=7.0), 1.0, O)
    b = mlp.point(g, _y(2, 1, [0.1, 0.2], [0.0, 0.01], [0.5], [0.5], fill=-3.0), 1.0, O)
    np.testing.assert_array_equal(a, b)


def test_loss_two_bus_known_violations(oracle_mod):
    """loss = c2 pg^2 + c1 pg + c0 + w (sum of squared row violations + sum of
    squared bound violations), with every row and violation written out by
    hand: the flow rows vanish (p, q are the flows), the balance rows are
    Pd + sum p - pg and Qd + sum q - qg, the thermal rows p^2 + q^2 - rate^2
    violate a small rating, vm and pg are pushed past their bounds."""
    rate = 0.5
    g = _two_bus(rate=rate)
    O = oracle_mod.Oracle(g)
    ya, yv, yp, yq = [0.0, -0.25], [0.15, -0.03], [1.25], [0.1]
    y = _y(2, 1, ya, yv, yp, yq)
    s = 0.8
    va = np.array([0.0, s * ya[1]])
    vm = 1.0 + np.array(yv)
    pg = 1.0 + 0.8 * yp[0]   # 2.0: 0.2 above pmax
    qg = 0.2 + 0.8 * yq[0]
    d, (pf, qf), (pt, qt) = _lossless_flows(va, vm)
    pd, qd = 0.6, 0.18
    rows = np.array([
        0.0,                      # reference angle
        0.0, 0.0, 0.0, 0.0,       # flow rows P_fr, Q_fr, P_to, Q_to
        d,                        # angle difference
        pf - pg, pd + pt,         # P balance at buses 0, 1
        qf - qg, qd + qt,         # Q balance
        pf * pf + qf * qf - rate * rate, pt * pt + qt * qt - rate * rate])  # thermal
    gl = np.array([0, 0, 0, 0, 0, -math.pi / 6, 0, 0, 0, 0, -np.inf, -np.inf])
    gu = np.array([0, 0, 0, 0, 0, math.pi / 6, 0, 0, 0, 0, 0, 0])
    xv = np.array([va[0], va[1], vm[0], vm[1], pg, qg, pf, pt, qf, qt])
    xl = np.array([-np.inf, -np.inf, 0.9, 0.9, 0.2, -0.6, -rate, -rate, -rate, -rate])
    xu = np.array([np.inf, np.inf, 1.1, 1.1, 1.8, 1.0, rate, rate, rate, rate])
    rho = np.maximum(gl - rows, 0) + np.maximum(rows - gu, 0)
    r = np.maximum(xl - xv, 0) + np.maximum(xv - xu, 0)
    assert r[2] == pytest.approx(0.05) and r[4] == pytest.approx(0.2)
    assert rho[10] > 0 and rho[11] > 0 and rho[6] > 0  # thermal and balance rows violated
    w = 1e3
    want = 0.07 * pg * pg + 12.0 * pg + 0.5 + w * (float(rho @ rho) + float(r @ r))
    got = mlp.loss(g, y, s, w, O, (xl, xu, gl, gu))
    assert got == pytest.approx(want, rel=1e-13)
    # with the oracle's own bounds the same value (its bounds follow Listing 3)
    assert mlp.loss(g, y, s, w, O, O.bounds()) == pytest.approx(want, rel=1e-13)
