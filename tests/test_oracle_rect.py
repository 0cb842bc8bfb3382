"""Pins of the oracle's rectangular form (form = :rect, Sec. III-C-1).

The rectangular model keeps the polar model's physics and changes only the
coordinates of the voltages, so most pins tie it to things fixed elsewhere:
the dense admittance-matrix evaluation and the Newton power flow of
tests/pins.py, the polar oracle at the same physical point (itself pinned by
tests/test_oracle_pins.py), trigonometric closed forms of the angle rows, and
one exact identity: every rectangular row is at most quadratic in x, so the
second-order Taylor expansion of the Lagrangian with the oracle's gradient,
Jacobian and Hessian is exact for any step, not only a small one.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2510_12897_b300 import synth
from tests import pins
from tests.test_oracle_pins import dense_lower, point, three_bus


def rect_rows(g):
    """Slices of the rectangular form's row groups (one period)."""
    nl, nb = len(g.br_f), g.nbus
    sizes = [("ref", 1), ("fpf", nl), ("fqf", nl), ("fpt", nl), ("fqt", nl), ("ang", nl),
             ("pb", nb), ("qb", nb), ("thf", nl), ("tht", nl), ("anl", nl), ("vm", nb)]
    out, o = {}, 0
    for k, s in sizes:
        out[k] = slice(o, o + s)
        o += s
    return out


def to_rect(g, x):
    """The rectangular point of a polar one (single period): vr = vm cos va,
    vi = vm sin va in the places of va, vm; everything else unchanged."""
    G = pins.groups(g)
    y = x.copy()
    va, vm = x[G["va"]], x[G["vm"]]
    y[G["va"]] = vm * np.cos(va)
    y[G["vm"]] = vm * np.sin(va)
    return y


def rect_point(g, seed):
    return to_rect(g, point(g, seed))


CASES = {"three": lambda: three_bus(True), "case30": lambda: synth.case30(),
         "case30g": lambda: synth.case30(general=True)}


@pytest.mark.parametrize("gen", [False, True])
def test_rect_sizes_closed_form(oracle_mod, gen):
    g = synth.case30(general=gen)
    O = oracle_mod.Oracle(g, form="rect")
    nb, nl, ng = g.nbus, g.nbranch, g.ngen
    pairs = {(min(a, b), max(a, b)) for a, b in zip(g.br_f, g.br_t)}
    assert O.n == 2 * nb + 2 * ng + 4 * nl
    assert O.m == 1 + 8 * nl + 3 * nb
    # flows 5 each, two angle rows 4 each, thermal 2 each; balance rows
    # (vr, vi, generators, arcs); magnitude rows 2
    assert O.nnzj == 1 + 36 * nl + 6 * nb + 2 * ng
    # (vr, vr), (vi, vi) per bus; four cross entries per connected pair;
    # cost; thermal (p, p), (q, q)
    assert O.nnzh == 2 * nb + 4 * len(pairs) + ng + 4 * nl
    r, c = O.hess_pattern()
    assert np.all(np.diff(r * O.n + c) > 0) and np.all(r >= c)


@pytest.mark.parametrize("which", ["three", "case30", "case30g"])
def test_rect_newton_power_flow_zero_mismatch(oracle_mod, which):
    """At a Newton-converged power flow (dense Y_bus), written in rectangular
    voltages with flows from Yf V, Yt V, every flow and balance row vanishes,
    the reference row is Im V_ref = 0 and the magnitude rows are |V|^2."""
    g = CASES[which]()
    Pd, Qd = pins.bus_demand(g)
    V = pins.newton_pf(g, np.full(g.ngen, Pd.sum() / g.ngen))
    Y, Yf, Yt = pins.ybus(g)
    S = V * np.conj(Y @ V)
    G = pins.groups(g)
    x = np.zeros(G["q"].stop)
    x[G["va"]] = V.real
    x[G["vm"]] = V.imag
    Sg = S + Pd + 1j * Qd
    x[G["pg"]] = Sg.real[g.gen_bus]
    x[G["qg"]] = Sg.imag[g.gen_bus]
    Sf = V[g.br_f] * np.conj(Yf @ V)
    St = V[g.br_t] * np.conj(Yt @ V)
    x[G["p"]] = np.concatenate([Sf.real, St.real])
    x[G["q"]] = np.concatenate([Sf.imag, St.imag])
    c = oracle_mod.Oracle(g, form="rect").cons(x)
    R = rect_rows(g)
    for k in ("fpf", "fqf", "fpt", "fqt"):
        assert np.max(np.abs(c[R[k]])) < 1e-12, k
    assert np.max(np.abs(c[R["pb"]])) < 1e-10
    assert np.max(np.abs(c[R["qb"]])) < 1e-10
    assert abs(c[R["ref"]][0]) < 1e-15  # the slack angle is 0
    np.testing.assert_allclose(c[R["vm"]], np.abs(V) ** 2, rtol=1e-15)


@pytest.mark.parametrize("which", ["three", "case30g"])
def test_rect_equals_polar_at_same_point(oracle_mod, which):
    """Flow, balance and thermal rows and the objective are those of the
    polar model at the same physical point; the angle rows equal the closed
    form vm_f vm_t sin(d - limit) / cos(limit)."""
    g = CASES[which]()
    Op, Or = oracle_mod.Oracle(g), oracle_mod.Oracle(g, form="rect")
    x = point(g, 3)
    y = to_rect(g, x)
    cp, cr = Op.cons(x), Or.cons(y)
    Rp, Rr = pins.rows(g), rect_rows(g)
    for k in ("fpf", "fqf", "fpt", "fqt", "pb", "qb", "thf", "tht"):
        np.testing.assert_allclose(cr[Rr[k]], cp[Rp[k]], rtol=1e-12, atol=1e-12, err_msg=k)
    assert Or.obj(y) == Op.obj(x)
    G = pins.groups(g)
    va, vm = x[G["va"]], x[G["vm"]]
    d = va[g.br_f] - va[g.br_t]
    m = vm[g.br_f] * vm[g.br_t]
    np.testing.assert_allclose(cr[Rr["ang"]], m * np.sin(d - g.br_angmax) / np.cos(g.br_angmax),
                               rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(cr[Rr["anl"]], m * np.sin(d - g.br_angmin) / np.cos(g.br_angmin),
                               rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(cr[Rr["vm"]], vm ** 2, rtol=1e-14)
    assert cr[Rr["ref"]][0] == pytest.approx(vm[g.ref_bus] * math.sin(va[g.ref_bus]), rel=1e-15)


@pytest.mark.parametrize("which", ["three", "case30g"])
def test_rect_jacobian_chain_rule(oracle_mod, which):
    """J_polar = J_rect d(vr, vi)/d(va, vm) on the voltage columns of every
    row the two forms share (the polar Jacobian is pinned by differences and
    sympy); the other columns are equal."""
    g = CASES[which]()
    Op, Or = oracle_mod.Oracle(g), oracle_mod.Oracle(g, form="rect")
    x = point(g, 8)
    y = to_rect(g, x)

    def dense(O, z):
        r, c = O.jac_pattern()
        return sp.coo_matrix((O.jac(z), (r, c)), shape=(O.m, O.n)).toarray()

    Jp, Jr = dense(Op, x), dense(Or, y)
    G = pins.groups(g)
    va, vm = x[G["va"]], x[G["vm"]]
    nb = g.nbus
    T = np.eye(Op.n)  # d(rect variables)/d(polar variables)
    iva, ivm = np.arange(G["va"].start, G["va"].stop), np.arange(G["vm"].start, G["vm"].stop)
    T[iva, iva] = -vm * np.sin(va)   # dvr/dva
    T[iva, ivm] = np.cos(va)         # dvr/dvm
    T[ivm, iva] = vm * np.cos(va)    # dvi/dva
    T[ivm, ivm] = np.sin(va)         # dvi/dvm
    Rp, Rr = pins.rows(g), rect_rows(g)
    for k in ("fpf", "fqf", "fpt", "fqt", "pb", "qb", "thf", "tht"):
        np.testing.assert_allclose(Jr[Rr[k]] @ T, Jp[Rp[k]], rtol=1e-11, atol=1e-11, err_msg=k)
    assert nb == iva.size


@pytest.mark.parametrize("which", ["three", "case30g", "mp"])
def test_rect_jacobian_differences(oracle_mod, which):
    g = {**CASES, "mp": lambda: synth.multi_period(three_bus(True), 3, seed=4, ramp_ratio=0.2)}[which]()
    O = oracle_mod.Oracle(g, form="rect")
    x = synth.random_point(g, np.random.default_rng(5))
    r, c = O.jac_pattern()
    J = sp.coo_matrix((O.jac(x), (r, c)), shape=(O.m, O.n)).toarray()
    fd = pins.central_diff(O.cons, x)
    np.testing.assert_allclose(J, fd, rtol=1e-8, atol=1e-8)
    mask = np.zeros((O.m, O.n), bool)
    mask[r, c] = True
    assert np.max(np.abs(fd[~mask])) < 1e-9


@pytest.mark.parametrize("which,sigma", [("three", 1.0), ("case30g", 0.3), ("mp", 0.7)])
def test_rect_hessian_differences(oracle_mod, which, sigma):
    g = {**CASES, "mp": lambda: synth.multi_period(three_bus(True), 3, seed=4, ramp_ratio=0.2)}[which]()
    O = oracle_mod.Oracle(g, form="rect")
    rng = np.random.default_rng(23)
    x = synth.random_point(g, rng)
    lam = rng.standard_normal(O.m)
    jr, jc = O.jac_pattern()

    def grad_L(y):
        return sigma * O.grad(y) + sp.coo_matrix((O.jac(y), (jr, jc)), shape=(O.m, O.n)).T @ lam

    fd = pins.central_diff(grad_L, x)
    hr, hc = O.hess_pattern()
    H = dense_lower(hr, hc, O.hess(x, lam, sigma), O.n)
    np.testing.assert_allclose(H, 0.5 * (fd + fd.T), rtol=1e-8, atol=1e-8)
    mask = np.zeros((O.n, O.n), bool)
    mask[hr, hc] = True
    mask |= mask.T
    assert np.max(np.abs(fd[~mask])) < 1e-8


@pytest.mark.parametrize("which", ["three", "case30g"])
def test_rect_exact_second_order_expansion(oracle_mod, which):
    """Every rectangular row and the cost are quadratic, so for any step h
    L(x + h) = L(x) + grad L(x) h + h^T H h / 2 holds exactly (up to
    rounding), L = sigma f + lambda^T g: a dropped term, wrong sign or wrong
    index anywhere in cons, jac or hess breaks it at a step of order one."""
    g = CASES[which]()
    O = oracle_mod.Oracle(g, form="rect")
    rng = np.random.default_rng(31)
    x = rect_point(g, 4)
    jr, jc = O.jac_pattern()
    hr, hc = O.hess_pattern()
    for trial in range(4):
        lam = rng.standard_normal(O.m)
        sigma = float(rng.uniform(0.1, 2.0))
        h = rng.standard_normal(O.n) * 0.7

        def L(z):
            return sigma * O.obj(z) + lam @ O.cons(z)

        J = sp.coo_matrix((O.jac(x), (jr, jc)), shape=(O.m, O.n))
        gL = sigma * O.grad(x) + J.T @ lam
        H = dense_lower(hr, hc, O.hess(x, lam, sigma), O.n)
        pred = L(x) + gL @ h + 0.5 * h @ H @ h
        scale = abs(L(x)) + np.abs(gL) @ np.abs(h) + 0.5 * np.abs(h) @ np.abs(H) @ np.abs(h)
        assert abs(L(x + h) - pred) <= 1e-13 * scale, trial
        # single rows: each row alone (sigma = 0, lambda = e_i) on a few rows
        for i in rng.choice(O.m, 8, replace=False):
            e = np.zeros(O.m)
            e[i] = 1.0
            Hi = dense_lower(hr, hc, O.hess(x, e, 0.0), O.n)
            gi = np.asarray(J.getrow(i).todense()).ravel()
            pi = O.cons(x)[i] + gi @ h + 0.5 * h @ Hi @ h
            assert abs(O.cons(x + h)[i] - pi) <= 1e-12 * (1 + abs(pi)), (trial, i)


def test_rect_hessian_independent_of_point(oracle_mod):
    """The rectangular Lagrangian Hessian is constant in x (every row is
    quadratic): equal, bit for bit, at unrelated points."""
    g = synth.case30(general=True)
    O = oracle_mod.Oracle(g, form="rect")
    lam = np.random.default_rng(2).standard_normal(O.m)
    np.testing.assert_array_equal(O.hess(rect_point(g, 1), lam, 0.4), O.hess(rect_point(g, 9), lam, 0.4))


def test_rect_bounds(oracle_mod):
    g = three_bus(True)
    O = oracle_mod.Oracle(g, form="rect")
    xl, xu, gl, gu = O.bounds()
    G, R = pins.groups(g), rect_rows(g)
    for k in ("va", "vm"):  # vr and vi
        np.testing.assert_array_equal(xl[G[k]], -g.bus_vmax)
        np.testing.assert_array_equal(xu[G[k]], g.bus_vmax)
    np.testing.assert_array_equal(gl[R["vm"]], g.bus_vmin ** 2)
    np.testing.assert_array_equal(gu[R["vm"]], g.bus_vmax ** 2)
    assert np.all(np.isneginf(gl[R["ang"]])) and np.all(gu[R["ang"]] == 0)
    assert np.all(gl[R["anl"]] == 0) and np.all(np.isposinf(gu[R["anl"]]))
    for k in ("ref", "fpf", "fqf", "fpt", "fqt", "pb", "qb"):
        assert np.all(gl[R[k]] == 0) and np.all(gu[R[k]] == 0), k
    # feasibility of the angle rows is that of the polar angle limits
    x = point(g, 12)
    va = x[G["va"]]
    d = va[g.br_f] - va[g.br_t]
    c = O.cons(to_rect(g, x))
    ok_p = (d >= g.br_angmin) & (d <= g.br_angmax)
    ok_r = (c[R["ang"]] <= 0) & (c[R["anl"]] >= 0)
    np.testing.assert_array_equal(ok_p, ok_r)


def test_rect_rejects_wide_angle_limits(oracle_mod):
    g = three_bus(True)
    g = g.copy(br_angmax=np.array([math.pi / 6, math.pi / 2, math.pi / 6]))
    oracle_mod.Oracle(g)  # the polar form accepts it
    with pytest.raises(ValueError, match="angle limits"):
        oracle_mod.Oracle(g, form="rect")


def test_rect_batch_reserve_links(oracle_mod):
    """A rectangular batch with per-instance ratios and reserve rows: blocks
    equal the single-instance oracles, linking and reserve rows as in polar."""
    insts = synth.contingencies(synth.case30(), 2, seed=9)
    Ob = oracle_mod.Oracle(insts, link_ratios=[0.0, 0.1, 0.3], reserve=0.15, form="rect")
    Op = oracle_mod.Oracle(insts, link_ratios=[0.0, 0.1, 0.3], reserve=0.15)
    singles = [oracle_mod.Oracle(s, form="rect") for s in insts]
    assert Ob.n == sum(s.n for s in singles)
    assert Ob.m - sum(s.m for s in singles) == Op.m - sum(oracle_mod.Oracle(s).m for s in insts)
    x = np.concatenate([rect_point(s, 40 + k) for k, s in enumerate(insts)])
    c = Ob.cons(x)
    off_x = off_c = 0
    for s, O1 in zip(insts, singles):
        np.testing.assert_array_equal(c[off_c:off_c + O1.m], O1.cons(x[off_x:off_x + O1.n]))
        off_x += O1.n
        off_c += O1.m
    # the coupling rows only read pg, which both forms place alike
    xp = np.concatenate([point(s, 40 + k) for k, s in enumerate(insts)])
    np.testing.assert_array_equal(c[off_c:], Op.cons(xp)[Op.m - (Ob.m - off_c):])
