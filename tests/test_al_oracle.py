"""Pins of the augmented-Lagrangian oracle (oracle/al.py) against what the
mathematics fixes, on CPU."""
import numpy as np

from oracle import al
from paper_2510_12897_b300 import synth
from tests import pins


def test_gradient_central_differences(oracle_mod):
    """G = grad f + J^T mu equals Richardson central differences of L(x;
    lambda) in every coordinate, at a point with active, inactive and
    violated rows (multi-period, general terms)."""
    g = synth.multi_period(synth.case30(general=True), 2, seed=4, ramp_ratio=0.2)
    O = oracle_mod.Oracle(g)
    A = al.AugLagOracle(O, rho=7.0, lr=1e-3)
    rng = np.random.default_rng(3)
    x = synth.random_point(g, rng)
    lam = rng.standard_normal(O.m)
    G = A.gradient(x, lam)
    fd = pins.central_diff(lambda v: np.array([A.value(v, lam)]), x, h=1e-5)[0]
    np.testing.assert_allclose(G, fd, rtol=1e-6, atol=1e-6 * max(1.0, float(np.max(np.abs(G)))))


def test_inside_bounds_no_penalty(oracle_mod):
    """With lambda = 0 at a point whose rows all lie strictly inside their
    bounds, mu = 0 and L = f; lambda = mu is then a fixed point of the
    update. The point: a Newton power-flow solution with p, q set to the
    flows (balance and flow rows zero), inside the angle and thermal limits."""
    g = synth.case30()
    g = g.copy(br_rate_a=np.full(g.nbranch, 10.0), br_angmin=np.full(g.nbranch, -1.5),
               br_angmax=np.full(g.nbranch, 1.5))
    O = oracle_mod.Oracle(g)
    xl, xu, gl, gu = O.bounds()
    x = power_flow_point(g)
    c = O.cons(x)
    assert np.all(c >= gl - 1e-9) and np.all(c <= gu + 1e-9)
    A = al.AugLagOracle(O, rho=3.0, lr=1e-3)
    lam = np.zeros(O.m)
    mu, _ = A.mu(x, lam)
    assert np.max(np.abs(mu)) <= 3.0 * 1e-9
    assert abs(A.value(x, lam) - O.obj(x)) <= 1e-9 * max(1.0, abs(O.obj(x)))
    lam2, _ = A.update(x, mu)
    np.testing.assert_allclose(lam2, mu, atol=1e-8)


def power_flow_point(g):
    """x at a Newton power-flow solution (textbook polar Newton-Raphson on the
    dense Y-bus): voltages from the solution, generator outputs from the
    injections, p and q the branch flows."""
    Pd, Qd = pins.bus_demand(g)
    V = pins.newton_pf(g, np.full(g.ngen, Pd.sum() / g.ngen))
    Y, Yf, Yt = pins.ybus(g)
    S = V * np.conj(Y @ V)
    G = pins.groups(g)
    x = np.zeros(G["q"].stop)
    x[G["va"]] = np.angle(V)
    x[G["vm"]] = np.abs(V)
    Sg = S + Pd + 1j * Qd
    x[G["pg"]] = Sg.real[g.gen_bus]
    x[G["qg"]] = Sg.imag[g.gen_bus]
    Sf = V[g.br_f] * np.conj(Yf @ V)
    St = V[g.br_t] * np.conj(Yt @ V)
    x[G["p"]] = np.concatenate([Sf.real, St.real])
    x[G["q"]] = np.concatenate([Sf.imag, St.imag])
    return x
