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


# ---- the projected Newton-CG step (NewtonOracle, pcg)

def test_newton_system_is_the_gradients_derivative(oracle_mod):
    """K v (K = H(x; mu, 1) + rho J^T D J, H assembled symmetric from its
    lower triangle) equals Richardson central differences of the AL gradient
    G along v, at a point where every row's s stays on its side of its bounds
    over the differencing interval (so D is constant there); several
    directions, multi-period general grid."""
    g = synth.multi_period(synth.case30(general=True), 2, seed=4, ramp_ratio=0.2)
    O = oracle_mod.Oracle(g)
    A = al.NewtonOracle(O, rho=7.0, lr=1e-3)
    rng = np.random.default_rng(5)
    x = synth.random_point(g, rng)
    lam = rng.standard_normal(O.m)
    G, K, D, _, _ = A.system(x, lam)
    assert 0 < D.sum() < O.m  # active and inactive rows
    xl, xu, gl, gu = O.bounds()
    for k in range(4):
        v = rng.standard_normal(O.n)
        h = 1e-6
        s_lo = O.cons(x - h * v) + lam / A.rho
        s_hi = O.cons(x + h * v) + lam / A.rho
        Dl = ((s_lo < gl) | (s_lo > gu)).astype(float)
        Dh = ((s_hi < gl) | (s_hi > gu)).astype(float)
        assert np.array_equal(Dl, D) and np.array_equal(Dh, D)
        d1 = (A.gradient(x + h * v, lam) - A.gradient(x - h * v, lam)) / (2 * h)
        d2 = (A.gradient(x + h / 2 * v, lam) - A.gradient(x - h / 2 * v, lam)) / h
        fd = (4 * d2 - d1) / 3
        Kv = K @ v
        np.testing.assert_allclose(Kv, fd, rtol=1e-5, atol=1e-5 * max(1.0, float(np.max(np.abs(Kv)))))


def test_pcg_solves_spd_systems():
    """On a symmetric positive definite system the preconditioned CG reaches
    numpy's dense solution over the free entries (the others stay zero); on
    an indefinite one whose first direction has negative curvature it
    returns that direction."""
    rng = np.random.default_rng(7)
    n = 40
    A0 = rng.standard_normal((n, n))
    K = A0 @ A0.T + n * np.eye(n)
    G = rng.standard_normal(n)
    F = rng.uniform(size=n) > 0.2
    Mj = np.diag(K).copy()
    p = al.pcg(lambda v: K @ v, G, F, Mj, 200)
    ff = np.flatnonzero(F)
    want = np.linalg.solve(K[np.ix_(ff, ff)], -G[ff])
    np.testing.assert_allclose(p[ff], want, rtol=1e-10, atol=1e-12)
    assert np.all(p[~F] == 0.0)
    Kneg = -np.eye(n)
    Fall = np.ones(n, bool)
    p1 = al.pcg(lambda v: Kneg @ v, G, Fall, np.ones(n), 10)
    np.testing.assert_array_equal(p1, -G)


def test_newton_steps_never_raise_L_and_reach_feasibility(oracle_mod):
    """The step never increases L(x; lambda); an outer loop of ten Newton
    steps per multiplier update (rho 1000) takes the 30-bus grid from the
    flat start to a max row violation below 1e-4 in twelve updates (a
    first-order loop stalls near 0.06 on the 2,000-bus grid)."""
    g = synth.secure_ratings(synth.case30())
    O = oracle_mod.Oracle(g)
    A = al.NewtonOracle(O, rho=1000.0, lr=1e-3)
    xl, xu, _, _ = O.bounds()
    nb, ng, nl = g.nbus, g.ngen, g.nbranch
    x = np.concatenate([np.zeros(nb), np.clip(np.ones(nb), xl[nb:2 * nb], xu[nb:2 * nb]),
                        0.5 * (xl[2 * nb:2 * nb + 2 * ng] + xu[2 * nb:2 * nb + 2 * ng]), np.zeros(4 * nl)])
    lam = np.zeros(O.m)
    viol0 = A.stats(x, lam)[1]
    for outer in range(12):
        for _ in range(10):
            L0 = A.value(x, lam)
            x, st, _ = A.newton_step(x, lam, 100)
            assert st[2] <= L0 + 1e-12 * max(1.0, abs(L0))
        lam, st = A.update(x, lam)
    assert A.stats(x, lam)[1] < 1e-4 < 0.5 < viol0
