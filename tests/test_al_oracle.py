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


class _FreeRows:
    """A problem with one free row (mu = 0) whose gradient is supplied by a
    callable of the call count: isolates the oracle's Adam step."""

    def __init__(self, n, grad_of_call):
        self.n, self.calls, self.grad_of_call = n, 0, grad_of_call

    def bounds(self):
        return np.full(self.n, -1e30), np.full(self.n, 1e30), np.array([-np.inf]), np.array([np.inf])

    def jac_pattern(self):
        return np.array([0]), np.array([0])

    def cons(self, x):
        return np.zeros(1)

    def jac(self, x):
        return np.zeros(1)

    def obj(self, x):
        return 0.0

    def grad(self, x):
        self.calls += 1
        return self.grad_of_call(self.calls)


def test_adam_constant_gradient_moves_lr_per_step():
    """A constant gradient c makes the bias-corrected moments exactly c and
    c^2 (Kingma and Ba, Sec. 3), so every step moves x by lr against the sign
    of c, up to eps / |c| and the FP32 rounding of the scale (3 x 2^-24)."""
    rng = np.random.default_rng(0)
    c = rng.uniform(0.5, 5.0, 64) * rng.choice([-1.0, 1.0], 64)
    A = al.AugLagOracle(_FreeRows(64, lambda k: c), rho=1.0, lr=1e-3)
    x0 = rng.standard_normal(64)
    for k in (1, 5, 40):
        A.k, A.m1, A.m2 = 0, np.zeros(64), np.zeros(64)
        xk, _ = A.iterate(x0, np.zeros(1), k)
        np.testing.assert_allclose(xk, x0 - k * 1e-3 * np.sign(c), rtol=0, atol=k * 1e-3 * 5e-7)


def test_adam_sign_flip_closed_form():
    """Gradients c then -c: after the second step m_hat = (0.9 * 0.1 - 0.1) c
    / (1 - 0.9^2) = -c / 19 and v_hat = c^2 (the two (1 - 0.999) c^2 terms
    over 1 - 0.999^2), so the two steps sum to -lr sign(c) (1 - 1/19)."""
    rng = np.random.default_rng(1)
    c = rng.uniform(0.5, 5.0, 32) * rng.choice([-1.0, 1.0], 32)
    A = al.AugLagOracle(_FreeRows(32, lambda k: c if k == 1 else -c), rho=1.0, lr=2e-3)
    x0 = rng.standard_normal(32)
    x2, _ = A.iterate(x0, np.zeros(1), 2)
    np.testing.assert_allclose(x2, x0 - 2e-3 * np.sign(c) * (1.0 - 1.0 / 19.0), rtol=0, atol=2e-3 * 1e-6)
