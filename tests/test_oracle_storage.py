"""Pins of the oracle's multi-period model with storage (Sec. III-C-2).

The storage rows are pinned by what they mean, not by their formulas: a
charge/discharge schedule integrated by a plain recurrence leaves every
state-of-charge row at zero; the converter-loss row vanishes where ps solves
the loss balance as a quadratic (numpy's roots), and its loss term is
r |I|^2 with I = conj(S / V) computed in complex arithmetic; units draw ps,
qs from their bus's balance rows and change nothing else; the
complementarity row is the product sc sd; sizes and bounds follow from the
model's definition; derivatives against central differences.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2510_12897_b300 import synth
from tests import pins
from tests.test_oracle_pins import dense_lower


def grid(T=4, general=True):
    return synth.with_storage(synth.multi_period(synth.case30(general=general), T, seed=3, ramp_ratio=0.2))


def slices(g):
    """Storage variable groups (ps, qs, sc, sd, se) and row groups (soc,
    loss, thermal, compl) of a single multi-period instance with storage."""
    T, ns = g.nperiod, g.storage.nstor
    base_x = T * (2 * g.nbus + 2 * g.ngen + 4 * g.nbranch)
    base_c = T * (1 + 7 * g.nbranch + 2 * g.nbus) + g.ngen * (T - 1)
    X = {k: slice(base_x + i * ns * T, base_x + (i + 1) * ns * T) for i, k in enumerate(("ps", "qs", "sc", "sd", "se"))}
    R = {k: slice(base_c + i * ns * T, base_c + (i + 1) * ns * T) for i, k in enumerate(("soc", "loss", "th", "cmp"))}
    return X, R


def test_storage_sizes(oracle_mod):
    g = grid()
    T, ns = g.nperiod, g.storage.nstor
    O, O0 = oracle_mod.Oracle(g), oracle_mod.Oracle(g.copy(storage=None))
    Oc = oracle_mod.Oracle(g, compl=True)
    assert O.n - O0.n == 5 * ns * T
    assert O.m - O0.m == 3 * ns * T and Oc.m - O.m == ns * T
    # balance +2, state of charge 3 (first period) or 4, losses 5, thermal 2
    assert O.nnzj - O0.nnzj == ns * (2 * T + 3 + 4 * (T - 1) + 5 * T + 2 * T)
    assert Oc.nnzj - O.nnzj == 2 * ns * T
    # (ps, vm), (ps, ps), (qs, vm), (qs, qs); complementarity (sd, sc)
    assert O.nnzh - O0.nnzh == 4 * ns * T and Oc.nnzh - O.nnzh == ns * T
    assert synth.n_vars(g) == O.n


def test_storage_placement_recipe():
    """Units at the buses with the largest 10% of base load, energy 1.5 x
    that load, 2-hour ratings (the synthetic recipe)."""
    g = synth.multi_period(synth.case2k(), 4, seed=1)
    s = synth.with_storage(g).storage
    pd = np.zeros(g.nbus)
    np.add.at(pd, g.load_bus, g.load_pd[0])
    assert s.nstor == round(0.1 * np.count_nonzero(pd))
    assert pd[s.bus].min() >= np.sort(pd)[-s.nstor]
    np.testing.assert_allclose(s.energy_rating, 1.5 * pd[s.bus])
    np.testing.assert_allclose(s.charge_rating, s.energy_rating / 2.0)


def test_state_of_charge_trajectory(oracle_mod):
    """se integrated by the recurrence se_t = se_{t-1} + dt (eta_c sc_t -
    sd_t / eta_d) from the initial energy: every state-of-charge row equals
    its bound (e_init in the first period, 0 after)."""
    g = grid(T=6)
    st = g.storage
    O = oracle_mod.Oracle(g)
    X, R = slices(g)
    rng = np.random.default_rng(4)
    x = synth.random_point(g, rng)
    T, ns = g.nperiod, st.nstor
    sc = rng.uniform(0, st.charge_rating, (T, ns))
    sd = rng.uniform(0, st.discharge_rating, (T, ns))
    se = np.empty((T, ns))
    prev = st.e_init.copy()
    for t in range(T):
        prev = prev + st.dt * (st.eta_c * sc[t] - sd[t] / st.eta_d)
        se[t] = prev
    x[X["sc"]], x[X["sd"]], x[X["se"]] = sc.ravel(), sd.ravel(), se.ravel()
    c = O.cons(x)
    gl = O.bounds()[2]
    np.testing.assert_allclose(c[R["soc"]], gl[R["soc"]], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(gl[R["soc"]][:ns], st.e_init)
    assert np.all(gl[R["soc"]][ns:] == 0)


def test_loss_row_is_series_resistance_loss(oracle_mod):
    """Loss term = r |I|^2 with I = conj(S / V), S = ps + j qs, V = vm e^{j va}:
    with ps the root of the loss balance ps + sd - sc = r (ps^2 + qs^2) / vm^2
    (numpy's roots of the quadratic), the loss row sits at p_loss = 0."""
    g = grid(T=3)
    st = g.storage
    O = oracle_mod.Oracle(g)
    X, R = slices(g)
    rng = np.random.default_rng(8)
    x = synth.random_point(g, rng)
    T, ns, nb = g.nperiod, st.nstor, g.nbus
    vm = x[nb * T:2 * nb * T].reshape(T, nb)
    va = x[:nb * T].reshape(T, nb)
    qs = x[X["qs"]].reshape(T, ns)
    net = (x[X["sc"]] - x[X["sd"]]).reshape(T, ns)  # ps - loss must equal this
    ps = np.empty((T, ns))
    for t in range(T):
        for k in range(ns):
            a = st.r[k] / vm[t, st.bus[k]] ** 2
            roots = np.roots([a, -1.0, net[t, k] + a * qs[t, k] ** 2])
            ps[t, k] = roots[np.argmin(np.abs(roots - net[t, k]))].real
    x[X["ps"]] = ps.ravel()
    c = O.cons(x)
    np.testing.assert_allclose(c[R["loss"]], 0.0, atol=1e-14)
    # the loss term itself, r |I|^2, in complex arithmetic
    V = vm * np.exp(1j * va)
    I = np.conj((ps + 1j * qs) / V[:, st.bus])
    loss = st.r * np.abs(I) ** 2
    x2 = x.copy()
    x2[X["sc"]] = 0.0
    x2[X["sd"]] = 0.0
    np.testing.assert_allclose(-(O.cons(x2)[R["loss"]] - ps.ravel()), loss.ravel(), rtol=1e-13)


def test_storage_draws_from_its_bus(oracle_mod):
    """Every row outside the storage groups equals the model without
    storage, except the units' buses' balance rows, which grow by ps and qs."""
    g = grid(T=3)
    st = g.storage
    O, O0 = oracle_mod.Oracle(g), oracle_mod.Oracle(g.copy(storage=None))
    X, R = slices(g)
    x = synth.random_point(g, np.random.default_rng(2))
    c, c0 = O.cons(x), O0.cons(x[:O0.n])
    T, nb, nl, ns = g.nperiod, g.nbus, g.nbranch, st.nstor
    expect = c0.copy()
    pb = T * (1 + 5 * nl)
    ps = x[X["ps"]].reshape(T, ns)
    qs = x[X["qs"]].reshape(T, ns)
    for t in range(T):
        for k in range(ns):
            expect[pb + nb * t + st.bus[k]] += ps[t, k]
            expect[pb + nb * T + nb * t + st.bus[k]] += qs[t, k]
    np.testing.assert_allclose(c[:O0.m], expect, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(c[R["th"]], x[X["ps"]] ** 2 + x[X["qs"]] ** 2, rtol=1e-15)


def test_complementarity_and_bounds(oracle_mod):
    g = grid(T=3)
    st = g.storage
    O = oracle_mod.Oracle(g, compl=True)
    X, R = slices(g)
    x = synth.random_point(g, np.random.default_rng(6))
    np.testing.assert_array_equal(O.cons(x)[R["cmp"]], x[X["sc"]] * x[X["sd"]])
    xl, xu, gl, gu = O.bounds()
    T = g.nperiod
    rep = lambda a: np.tile(a, T)  # noqa: E731
    np.testing.assert_array_equal(xl[X["ps"]], -rep(st.thermal_rating))
    np.testing.assert_array_equal(xu[X["ps"]], rep(st.thermal_rating))
    np.testing.assert_array_equal(xl[X["qs"]], rep(st.qmin))
    np.testing.assert_array_equal(xu[X["qs"]], rep(st.qmax))
    assert np.all(xl[X["sc"]] == 0) and np.all(xl[X["sd"]] == 0) and np.all(xl[X["se"]] == 0)
    np.testing.assert_array_equal(xu[X["sc"]], rep(st.charge_rating))
    np.testing.assert_array_equal(xu[X["sd"]], rep(st.discharge_rating))
    np.testing.assert_array_equal(xu[X["se"]], rep(st.energy_rating))
    np.testing.assert_array_equal(gl[R["loss"]], rep(st.p_loss))
    np.testing.assert_array_equal(gu[R["th"]], rep(st.thermal_rating ** 2))
    assert np.all(np.isneginf(gl[R["th"]])) and np.all(np.isneginf(gl[R["cmp"]])) and np.all(gu[R["cmp"]] == 0)


@pytest.mark.parametrize("compl", [False, True])
def test_storage_jacobian_differences(oracle_mod, compl):
    g = grid(T=3)
    O = oracle_mod.Oracle(g, compl=compl)
    x = synth.random_point(g, np.random.default_rng(5))
    r, c = O.jac_pattern()
    J = sp.coo_matrix((O.jac(x), (r, c)), shape=(O.m, O.n)).toarray()
    fd = pins.central_diff(O.cons, x)
    np.testing.assert_allclose(J, fd, rtol=1e-8, atol=1e-8)
    mask = np.zeros((O.m, O.n), bool)
    mask[r, c] = True
    assert np.max(np.abs(fd[~mask])) < 1e-9


@pytest.mark.parametrize("compl", [False, True])
def test_storage_hessian_differences(oracle_mod, compl):
    g = grid(T=3)
    O = oracle_mod.Oracle(g, compl=compl)
    rng = np.random.default_rng(19)
    x = synth.random_point(g, rng)
    lam = rng.standard_normal(O.m)
    jr, jc = O.jac_pattern()

    def grad_L(y):
        return 0.6 * O.grad(y) + sp.coo_matrix((O.jac(y), (jr, jc)), shape=(O.m, O.n)).T @ lam

    fd = pins.central_diff(grad_L, x)
    hr, hc = O.hess_pattern()
    H = dense_lower(hr, hc, O.hess(x, lam, 0.6), O.n)
    np.testing.assert_allclose(H, 0.5 * (fd + fd.T), rtol=1e-7, atol=1e-7)
    mask = np.zeros((O.n, O.n), bool)
    mask[hr, hc] = True
    mask |= mask.T
    assert np.max(np.abs(fd[~mask])) < 1e-8


def test_storage_rejections(oracle_mod):
    g = grid(T=2)
    with pytest.raises(ValueError, match="polar"):
        oracle_mod.Oracle(g, form="rect")
    bad = g.copy(storage=synth.replace(g.storage, bus=np.array([0, g.nbus], np.int32)))
    with pytest.raises(ValueError, match="bus"):
        oracle_mod.Oracle(bad)
    bad = g.copy(storage=synth.replace(g.storage, eta_c=np.zeros(g.storage.nstor)))
    with pytest.raises(ValueError, match="efficienc"):
        oracle_mod.Oracle(bad)
