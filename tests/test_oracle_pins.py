"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's own formulas: they use textbook
closed forms, a dense admittance-matrix evaluation, a Newton power flow,
symbolic differentiation (sympy), finite differences, invariants and the
closed-form sizes of the model of Listing 3.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2510_12897_b300 import synth
from tests import pins


def tiny(nbus, branches, gens, loads, *, gs=None, bs=None, T=1, ramp=0.0, ref=None):
    """Hand-built grid. branches: (f, t, r, x, b, tap, shift, rate);
    gens: (bus, c2, c1, c0); loads: (bus, pd, qd) or per-period arrays."""
    br = np.array(branches, dtype=float).reshape(-1, 8)
    gn = np.array(gens, dtype=float).reshape(-1, 4)
    ld = list(loads)
    nl = br.shape[0]
    lb = np.array([l[0] for l in ld], dtype=np.int32)
    pd = np.array([np.broadcast_to(l[1], (T,)) for l in ld], dtype=float).T.reshape(T, len(ld))
    qd = np.array([np.broadcast_to(l[2], (T,)) for l in ld], dtype=float).T.reshape(T, len(ld))
    return synth.Grid(
        nbus=nbus, bus_vmin=np.full(nbus, 0.9), bus_vmax=np.full(nbus, 1.1),
        bus_gs=np.zeros(nbus) if gs is None else np.asarray(gs, float),
        bus_bs=np.zeros(nbus) if bs is None else np.asarray(bs, float),
        br_f=br[:, 0].astype(np.int32), br_t=br[:, 1].astype(np.int32),
        br_r=br[:, 2].copy(), br_x=br[:, 3].copy(), br_b=br[:, 4].copy(),
        br_tap=br[:, 5].copy(), br_shift=br[:, 6].copy(), br_rate_a=br[:, 7].copy(),
        br_angmin=np.full(nl, -math.pi / 6), br_angmax=np.full(nl, math.pi / 6),
        gen_bus=gn[:, 0].astype(np.int32), gen_pmin=np.zeros(len(gn)), gen_pmax=np.full(len(gn), 2.0),
        gen_qmin=np.full(len(gn), -1.0), gen_qmax=np.full(len(gn), 1.0),
        gen_c2=gn[:, 1].copy(), gen_c1=gn[:, 2].copy(), gen_c0=gn[:, 3].copy(),
        load_bus=lb, load_pd=pd, load_qd=qd,
        ref_bus=int(gn[0, 0]) if ref is None else ref, ramp_ratio=ramp)


def three_bus(general=True):
    return tiny(
        3,
        [(0, 1, 0.02, 0.10, 0.04, 1.05 if general else 1.0, 0.05 if general else 0.0, 2.0),
         (1, 2, 0.03, 0.15, 0.02, 1.0, 0.0, 1.5),
         (2, 0, 0.01, 0.08, 0.03, 0.97 if general else 1.0, -0.04 if general else 0.0, 1.0)],
        [(0, 0.05, 20.0, 1.0), (2, 0.02, 30.0, 0.0)],
        [(1, 0.9, 0.3), (2, 0.4, 0.1)],
        gs=[0.0, 0.03, 0.0] if general else None, bs=[0.02, 0.0, -0.01] if general else None)


def point(g, seed):
    return synth.random_point(g, np.random.default_rng(seed))


def dense_lower(rows, cols, vals, n):
    H = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).toarray()
    return H + np.tril(H, -1).T


# --------------------------------------------------------------- sizes --

@pytest.mark.parametrize("gen", [False, True])
def test_sizes_closed_form(oracle_mod, gen):
    g = synth.case30(general=gen)
    O = oracle_mod.Oracle(g)
    nb, nl, ng = g.nbus, g.nbranch, g.ngen
    pairs = {(min(a, b), max(a, b)) for a, b in zip(g.br_f, g.br_t)}
    with_branch = len(set(g.br_f) | set(g.br_t))
    assert O.n == 2 * nb + 2 * ng + 4 * nl
    assert O.m == 1 + 7 * nl + 2 * nb
    assert O.nnzj == 1 + 30 * nl + 2 * nb + 2 * ng
    assert O.nnzh == 2 * with_branch + nb + 4 * len(pairs) + ng + 4 * nl
    if not gen:  # the 30-bus workload's closed-form figures
        assert (O.n, O.m, O.nnzj, O.nnzh) == (236, 348, 1303, 424)


def test_sizes_multiperiod_and_batch(oracle_mod):
    g = synth.multi_period(synth.case30(), 4, seed=5, ramp_ratio=0.2)
    O = oracle_mod.Oracle(g)
    T, nb, nl, ng = 4, g.nbus, g.nbranch, g.ngen
    assert O.n == T * (2 * nb + 2 * ng + 4 * nl)
    assert O.m == T * (1 + 7 * nl + 2 * nb) + ng * (T - 1)
    assert O.nnzj == T * (1 + 30 * nl + 2 * nb + 2 * ng) + 2 * ng * (T - 1)
    b = synth.contingencies(synth.case30(), 3, seed=1)
    Ob = oracle_mod.Oracle(b, link_ratio=0.2)
    singles = [oracle_mod.Oracle(x) for x in b]
    assert Ob.n == sum(s.n for s in singles)
    assert Ob.m == sum(s.m for s in singles) + 3 * b[0].ngen
    assert Ob.nnzj == sum(s.nnzj for s in singles) + 2 * 3 * b[0].ngen
    assert Ob.nnzh == sum(s.nnzh for s in singles)


def test_pattern_order(oracle_mod):
    O = oracle_mod.Oracle(synth.case30(general=True))
    for r, c in (O.jac_pattern(), O.hess_pattern()):
        key = r * O.n + c
        assert np.all(np.diff(key) > 0)  # sorted row-major, no duplicates
    hr, hc = O.hess_pattern()
    assert np.all(hr >= hc)


# ------------------------------------------------------ textbook flows --

def flows(O, g, x):
    """Branch flows as the oracle's flow rows give them at p = q = 0."""
    G = pins.groups(g)
    R = pins.rows(g)
    x = x.copy()
    x[G["p"]] = 0.0
    x[G["q"]] = 0.0
    c = O.cons(x)
    return -c[R["fpf"]], -c[R["fqf"]], -c[R["fpt"]], -c[R["fqt"]]


@pytest.mark.parametrize("tap,shift", [(1.0, 0.0), (1.07, 0.0), (1.0, 0.13), (0.93, -0.2)])
def test_lossless_line_textbook(oracle_mod, tap, shift):
    """r = 0, b = 0: P_fr = vf vt sin(d - shift) / (tap x),
    Q_fr = vf^2 / (tap^2 x) - vf vt cos(d - shift) / (tap x)."""
    xk = 0.2
    g = tiny(2, [(0, 1, 0.0, xk, 0.0, tap, shift, 1.0)], [(0, 0.1, 10.0, 0.0)], [(1, 0.1, 0.0)])
    O = oracle_mod.Oracle(g)
    x = point(g, 3)
    G = pins.groups(g)
    vaf, vat = x[G["va"]]
    vf, vt = x[G["vm"]]
    d = vaf - vat - shift
    pf, qf, pt, qt = flows(O, g, x)
    assert pf[0] == pytest.approx(vf * vt * math.sin(d) / (tap * xk), rel=1e-14, abs=1e-15)
    assert qf[0] == pytest.approx(vf ** 2 / (tap ** 2 * xk) - vf * vt * math.cos(d) / (tap * xk),
                                  rel=1e-13, abs=1e-14)
    assert pt[0] == pytest.approx(-pf[0], rel=1e-13, abs=1e-15)  # lossless
    assert qt[0] == pytest.approx(vt ** 2 / xk - vf * vt * math.cos(d) / (tap * xk), rel=1e-13, abs=1e-14)


def test_no_load_charging(oracle_mod):
    """Flat voltages, tap 1, no shift: no active flow; each end injects b/2."""
    b = 0.06
    g = tiny(2, [(0, 1, 0.03, 0.2, b, 1.0, 0.0, 1.0)], [(0, 0.1, 10.0, 0.0)], [(1, 0.1, 0.0)])
    O = oracle_mod.Oracle(g)
    x = point(g, 1)
    G = pins.groups(g)
    x[G["va"]] = 0.0
    x[G["vm"]] = 1.0
    pf, qf, pt, qt = flows(O, g, x)
    assert abs(pf[0]) < 1e-15 and abs(pt[0]) < 1e-15
    assert qf[0] == pytest.approx(-b / 2, rel=1e-14)
    assert qt[0] == pytest.approx(-b / 2, rel=1e-14)


def test_dense_ybus_three_bus(oracle_mod):
    """Per-bus sums of the oracle's arc flows plus the shunt equal the
    injections of a dense Y_bus evaluation S = V conj(Y V)."""
    g = three_bus(general=True)
    O = oracle_mod.Oracle(g)
    Y, Yf, Yt = pins.ybus(g)
    for seed in range(5):
        x = point(g, seed)
        G = pins.groups(g)
        V = x[G["vm"]] * np.exp(1j * x[G["va"]])
        S = V * np.conj(Y @ V)
        pf, qf, pt, qt = flows(O, g, x)
        Sb = np.zeros(g.nbus, complex)
        np.add.at(Sb, g.br_f, pf + 1j * qf)
        np.add.at(Sb, g.br_t, pt + 1j * qt)
        Sb += np.abs(V) ** 2 * (g.bus_gs - 1j * g.bus_bs)
        np.testing.assert_allclose(Sb, S, rtol=0, atol=1e-14)
        # branch rows: S_f = V_f conj(Yf V), S_t = V_t conj(Yt V)
        np.testing.assert_allclose(pf + 1j * qf, V[g.br_f] * np.conj(Yf @ V), atol=1e-14)
        np.testing.assert_allclose(pt + 1j * qt, V[g.br_t] * np.conj(Yt @ V), atol=1e-14)
        # balance rows at p, q = flows: Pd - sum(pg) + Re S, Qd - sum(qg) + Im S
        x2 = x.copy()
        x2[G["p"]] = np.concatenate([pf, pt])
        x2[G["q"]] = np.concatenate([qf, qt])
        c = O.cons(x2)
        R = pins.rows(g)
        Pd, Qd = pins.bus_demand(g)
        pg = np.zeros(g.nbus)
        qg = np.zeros(g.nbus)
        np.add.at(pg, g.gen_bus, x[G["pg"]])
        np.add.at(qg, g.gen_bus, x[G["qg"]])
        np.testing.assert_allclose(c[R["pb"]], Pd - pg + S.real, atol=1e-14)
        np.testing.assert_allclose(c[R["qb"]], Qd - qg + S.imag, atol=1e-14)


@pytest.mark.parametrize("which", ["three", "case30", "case30g"])
def test_newton_power_flow_zero_mismatch(oracle_mod, which):
    """At a Newton-converged power-flow point (dense Y_bus, textbook polar
    Newton-Raphson) with branch flows from Yf V / Yt V and generator outputs
    from the injections, every flow and balance row of the oracle vanishes."""
    g = {"three": lambda: three_bus(True), "case30": lambda: synth.case30(),
         "case30g": lambda: synth.case30(general=True)}[which]()
    Pd, Qd = pins.bus_demand(g)
    ng = g.ngen
    pg_pv = np.full(ng, Pd.sum() / ng)
    V = pins.newton_pf(g, pg_pv)
    Y, Yf, Yt = pins.ybus(g)
    S = V * np.conj(Y @ V)
    G = pins.groups(g)
    x = np.zeros(pins.groups(g)["q"].stop)
    x[G["va"]] = np.angle(V)
    x[G["vm"]] = np.abs(V)
    Sg = S + Pd + 1j * Qd   # generation needed at each bus
    x[G["pg"]] = Sg.real[g.gen_bus]
    x[G["qg"]] = Sg.imag[g.gen_bus]
    Sf = V[g.br_f] * np.conj(Yf @ V)
    St = V[g.br_t] * np.conj(Yt @ V)
    x[G["p"]] = np.concatenate([Sf.real, St.real])
    x[G["q"]] = np.concatenate([Sf.imag, St.imag])
    O = oracle_mod.Oracle(g)
    c = O.cons(x)
    R = pins.rows(g)
    for k in ("fpf", "fqf", "fpt", "fqt"):
        assert np.max(np.abs(c[R[k]])) < 1e-12, k
    assert np.max(np.abs(c[R["pb"]])) < 1e-10
    assert np.max(np.abs(c[R["qb"]])) < 1e-10
    assert c[R["ref"]][0] == x[G["va"]][g.ref_bus]


# ------------------------------------------------------------ objective --

def test_objective_closed_form(oracle_mod):
    g = synth.multi_period(synth.case30(general=True), 3, seed=2, ramp_ratio=0.2)
    O = oracle_mod.Oracle(g)
    x = point(g, 7)
    ng, T, nb = g.ngen, 3, g.nbus
    pg = x[2 * nb * T: 2 * nb * T + ng * T].reshape(T, ng)
    f = np.sum(g.gen_c2 * pg ** 2 + g.gen_c1 * pg + g.gen_c0)
    assert O.obj(x) == pytest.approx(f, rel=1e-14)
    gr = O.grad(x)
    ref = np.zeros_like(x)
    ref[2 * nb * T: 2 * nb * T + ng * T] = (2 * g.gen_c2 * pg + g.gen_c1).ravel()
    np.testing.assert_array_equal(gr, ref)


def test_gradient_differences(oracle_mod):
    g = synth.case30(general=True)
    O = oracle_mod.Oracle(g)
    x = point(g, 11)
    fd = pins.central_diff(lambda y: np.array([O.obj(y)]), x)[0]
    np.testing.assert_allclose(O.grad(x), fd, rtol=1e-9, atol=1e-9)


# ----------------------------------------------------------- Jacobian --

@pytest.mark.parametrize("which", ["three", "case30g", "mp"])
def test_jacobian_differences(oracle_mod, which):
    """Every Jacobian value equals the central difference of cons; every
    structural nonzero found by differences lies in the pattern."""
    g = {"three": lambda: three_bus(True), "case30g": lambda: synth.case30(general=True),
         "mp": lambda: synth.multi_period(three_bus(True), 3, seed=4, ramp_ratio=0.2)}[which]()
    O = oracle_mod.Oracle(g)
    x = point(g, 5)
    r, c = O.jac_pattern()
    J = sp.coo_matrix((O.jac(x), (r, c)), shape=(O.m, O.n)).toarray()
    fd = pins.central_diff(O.cons, x)
    np.testing.assert_allclose(J, fd, rtol=1e-8, atol=1e-8)
    mask = np.zeros((O.m, O.n), bool)
    mask[r, c] = True
    assert np.max(np.abs(fd[~mask])) < 1e-9


@pytest.mark.parametrize("opts", [dict(link_ratio=0.2),
                                  dict(link_ratios=[0.0, 0.1, 0.3], reserve=0.15)])
def test_jacobian_batch_with_links(oracle_mod, opts):
    """Central differences of cons over sampled columns (every pg column
    included) for a batch with linking rows, and with per-instance ratios
    and reserve rows."""
    insts = synth.contingencies(synth.case30(), 2, seed=9)
    O = oracle_mod.Oracle(insts, **opts)
    x = np.concatenate([point(s, 20 + k) for k, s in enumerate(insts)])
    r, c = O.jac_pattern()
    J = sp.coo_matrix((O.jac(x), (r, c)), shape=(O.m, O.n)).toarray()
    # differences only over a subset of columns to keep it fast
    pgs = np.concatenate([np.arange(2 * s.nbus, 2 * s.nbus + s.ngen) + off for s, off in
                          zip(insts, np.cumsum([0] + [synth.n_vars(s) for s in insts[:-1]]))])
    cols = np.union1d(np.random.default_rng(0).choice(O.n, 120, replace=False), pgs)
    for j in cols:
        def fj(t):
            y = x.copy()
            y[j] = t
            return O.cons(y)
        h = 1e-4
        d1 = (fj(x[j] + h) - fj(x[j] - h)) / (2 * h)
        d2 = (fj(x[j] + h / 2) - fj(x[j] - h / 2)) / h
        np.testing.assert_allclose(J[:, j], (4 * d2 - d1) / 3, rtol=1e-8, atol=1e-8)


# ------------------------------------------------------------ Hessian --

@pytest.mark.parametrize("which,sigma", [("three", 1.0), ("case30g", 1.0), ("case30g", 0.0),
                                         ("mp", 0.7)])
def test_hessian_differences_and_symmetry(oracle_mod, which, sigma):
    """Hessian of the Lagrangian = central difference of
    sigma grad f + J^T lambda; the difference matrix is symmetric."""
    g = {"three": lambda: three_bus(True), "case30g": lambda: synth.case30(general=True),
         "mp": lambda: synth.multi_period(three_bus(True), 3, seed=4, ramp_ratio=0.2)}[which]()
    O = oracle_mod.Oracle(g)
    rng = np.random.default_rng(17)
    x = point(g, 6)
    lam = rng.standard_normal(O.m)
    jr, jc = O.jac_pattern()

    def grad_L(y):
        JT = sp.coo_matrix((O.jac(y), (jr, jc)), shape=(O.m, O.n)).T
        return sigma * O.grad(y) + JT @ lam

    fd = pins.central_diff(grad_L, x)
    np.testing.assert_allclose(fd, fd.T, rtol=1e-7, atol=1e-7)
    hr, hc = O.hess_pattern()
    H = dense_lower(hr, hc, O.hess(x, lam, sigma), O.n)
    np.testing.assert_allclose(H, 0.5 * (fd + fd.T), rtol=1e-8, atol=1e-8)
    mask = np.zeros((O.n, O.n), bool)
    mask[hr, hc] = True
    mask |= mask.T
    assert np.max(np.abs(fd[~mask])) < 1e-8


def test_hessian_single_row_isolated(oracle_mod):
    """sigma = 0 and lambda = e_i gives the Hessian of row i alone; for a
    thermal row that is 2 on (p, p) and (q, q) and nothing else."""
    g = three_bus(True)
    O = oracle_mod.Oracle(g)
    R = pins.rows(g)
    G = pins.groups(g)
    x = point(g, 2)
    lam = np.zeros(O.m)
    k = 1
    lam[R["thf"].start + k] = 1.0
    hr, hc = O.hess_pattern()
    H = dense_lower(hr, hc, O.hess(x, lam, 0.0), O.n)
    expect = np.zeros_like(H)
    expect[G["p"].start + k, G["p"].start + k] = 2.0
    expect[G["q"].start + k, G["q"].start + k] = 2.0
    np.testing.assert_array_equal(H, expect)


# ---------------------------------------------------- symbolic (sympy) --

def test_sympy_branch_derivatives(oracle_mod):
    """First and second derivatives of the four flows of one branch, from
    sympy's symbolic differentiation of S = V conj(Y V), at 30 digits."""
    sympy = pytest.importorskip("sympy")
    r_, x_, b_, tau, th = 0.02, 0.11, 0.05, 1.04, 0.09
    g = tiny(2, [(0, 1, r_, x_, b_, tau, th, 2.0)], [(0, 0.1, 10.0, 0.0)], [(1, 0.2, 0.1)])
    O = oracle_mod.Oracle(g)
    x = point(g, 9)
    G = pins.groups(g)
    R = pins.rows(g)
    vmf, vmt, vaf, vat = sympy.symbols("vmf vmt vaf vat", real=True)
    Rn = lambda v: sympy.Float(repr(float(v)), 40)
    ys = 1 / (Rn(r_) + sympy.I * Rn(x_))
    ratio = Rn(tau) * sympy.exp(sympy.I * Rn(th))
    Ytt = ys + sympy.I * Rn(b_) / 2
    Yff = Ytt / Rn(tau) ** 2
    Yft = -ys / sympy.conjugate(ratio)
    Ytf = -ys / ratio
    Vf = vmf * sympy.exp(sympy.I * vaf)
    Vt = vmt * sympy.exp(sympy.I * vat)
    Sf = sympy.expand_complex(Vf * sympy.conjugate(Yff * Vf + Yft * Vt))
    St = sympy.expand_complex(Vt * sympy.conjugate(Ytf * Vf + Ytt * Vt))
    funcs = {"fpf": sympy.re(Sf), "fqf": sympy.im(Sf), "fpt": sympy.re(St), "fqt": sympy.im(St)}
    u = [vmf, vmt, vaf, vat]
    uidx = [G["vm"].start + 0, G["vm"].start + 1, G["va"].start + 0, G["va"].start + 1]
    subs = {vmf: Rn(x[uidx[0]]), vmt: Rn(x[uidx[1]]), vaf: Rn(x[uidx[2]]), vat: Rn(x[uidx[3]])}
    jr, jc = O.jac_pattern()
    J = sp.coo_matrix((O.jac(x), (jr, jc)), shape=(O.m, O.n)).toarray()
    hr, hc = O.hess_pattern()
    for name, F in funcs.items():
        row = R[name].start
        for a in range(4):
            d = float(sympy.diff(F, u[a]).evalf(30, subs=subs))
            assert J[row, uidx[a]] == pytest.approx(-d, rel=1e-13, abs=1e-13), (name, a)
        lam = np.zeros(O.m)
        lam[row] = 1.0
        H = dense_lower(hr, hc, O.hess(x, lam, 0.0), O.n)
        for a in range(4):
            for b in range(4):
                d2 = float(sympy.diff(F, u[a], u[b]).evalf(30, subs=subs))
                assert H[uidx[a], uidx[b]] == pytest.approx(-d2, rel=1e-13, abs=1e-13), (name, a, b)


# ------------------------------------------------ layouts and batches --

def test_multiperiod_blocks_equal_static(oracle_mod):
    """Period t of the multi-period model is the static model with period t's
    demand, at the indices elem + count * t (Listing 10); ramp rows are
    pg_t - pg_{t-1}."""
    T = 3
    g = synth.multi_period(synth.case30(general=True), T, seed=3, ramp_ratio=0.2)
    O = oracle_mod.Oracle(g)
    x = point(g, 8)
    c = O.cons(x)
    nb, ng, na, nl = g.nbus, g.ngen, 2 * g.nbranch, g.nbranch
    cnt_x = [nb, nb, ng, ng, na, na]
    cnt_c = [1, nl, nl, nl, nl, nl, nb, nb, nl, nl]
    for t in range(T):
        gt = g.copy(load_pd=g.load_pd[t:t + 1], load_qd=g.load_qd[t:t + 1], ramp_ratio=0.0)
        Ot = oracle_mod.Oracle(gt)
        xt, off = [], 0
        for k in cnt_x:
            xt.append(x[off + k * t: off + k * (t + 1)])
            off += k * T
        ct, off = [], 0
        for k in cnt_c:
            ct.append(c[off + k * t: off + k * (t + 1)])
            off += k * T
        np.testing.assert_array_equal(np.concatenate(ct), Ot.cons(np.concatenate(xt)))
    pg = x[2 * nb * T: 2 * nb * T + ng * T].reshape(T, ng)
    ramp = c[sum(cnt_c) * T:]
    np.testing.assert_array_equal(ramp, (pg[1:] - pg[:-1]).ravel())
    xl, xu, gl, gu = O.bounds()
    np.testing.assert_array_equal(gu[sum(cnt_c) * T:], np.tile(0.2 * g.gen_pmax, T - 1))


def test_batch_blocks_and_links(oracle_mod):
    insts = synth.contingencies(synth.case30(), 3, seed=12)
    O = oracle_mod.Oracle(insts, link_ratio=0.25)
    singles = [oracle_mod.Oracle(s) for s in insts]
    xs = [point(s, 30 + k) for k, s in enumerate(insts)]
    x = np.concatenate(xs)
    c = O.cons(x)
    off = 0
    for s, xi in zip(singles, xs):
        np.testing.assert_array_equal(c[off: off + s.m], s.cons(xi))
        off += s.m
    ng = insts[0].ngen
    nb = insts[0].nbus
    pg0 = xs[0][2 * nb: 2 * nb + ng]
    link = np.concatenate([xi[2 * nb: 2 * nb + ng] - pg0 for xi in xs[1:]])
    np.testing.assert_array_equal(c[off:], link)
    lam = np.random.default_rng(1).standard_normal(O.m)
    H = O.hess(x, lam, 0.5)
    o = 0
    lo = 0
    for s, xi in zip(singles, xs):
        np.testing.assert_allclose(H[o: o + s.nnzh], s.hess(xi, lam[lo: lo + s.m], 0.5), rtol=0, atol=0)
        o += s.nnzh
        lo += s.m


# ----------------------------------------------------------------- Cvio --

def test_cvio_closed_form(oracle_mod):
    g = three_bus(False)
    O = oracle_mod.Oracle(g)
    xl, xu, gl, gu = O.bounds()
    G = pins.groups(g)
    R = pins.rows(g)
    x = point(g, 4)
    c = O.cons(x)
    expect = max(np.max(np.maximum(gl - c, 0)), np.max(np.maximum(c - gu, 0)))
    cv, vv = O.cvio(x)
    assert cv == expect and vv == 0.0
    y = x.copy()
    y[G["vm"].start] = 1.3  # 0.2 above vmax
    assert O.cvio(y)[1] == pytest.approx(0.2, rel=1e-14)
    # bounds of Listing 3
    assert np.all(np.isinf(xl[G["va"]])) and np.all(xu[G["vm"]] == 1.1)
    np.testing.assert_array_equal(xu[G["p"]], np.concatenate([g.br_rate_a, g.br_rate_a]))
    assert np.all(np.isneginf(gl[R["thf"]])) and np.all(gu[R["thf"]] == 0)
    np.testing.assert_array_equal(gl[R["ang"]], g.br_angmin)


def test_invalid_networks_rejected(oracle_mod):
    g = three_bus(False)
    bad = g.copy(br_t=np.array([1, 2, 2], np.int32))  # branch 2 becomes a self-loop
    with pytest.raises(ValueError):
        oracle_mod.Oracle(bad)
    bad = g.copy(br_r=np.array([0.0, 0.03, 0.01]), br_x=np.array([0.0, 0.15, 0.08]))
    with pytest.raises(ValueError):
        oracle_mod.Oracle(bad)
    bad = g.copy(gen_bus=np.array([0, 5], np.int32))
    with pytest.raises(ValueError):
        oracle_mod.Oracle(bad)


def test_reserve_rows_value_and_bounds(oracle_mod):
    """A reserve row holds the instance-period's total generation and its
    upper bound leaves the requested share of the period's demand as spare
    capacity (both checked on hand-set outputs: every generator at the same
    value)."""
    g = synth.multi_period(synth.case30(), 3, seed=2, ramp_ratio=0.0)
    O = oracle_mod.Oracle(g, reserve=0.25)
    plain = oracle_mod.Oracle(g)
    x = np.zeros(O.n)
    nb, ng, T = g.nbus, g.ngen, 3
    x[2 * nb * T:2 * nb * T + ng * T] = 0.75  # every pg, every period
    c = O.cons(x)
    np.testing.assert_allclose(c[plain.m:], np.full(T, 0.75 * ng), rtol=1e-15)
    _, _, gl, gu = O.bounds()
    assert np.all(np.isneginf(gl[plain.m:]))
    demand = g.load_pd.sum(axis=1)
    np.testing.assert_allclose(gu[plain.m:], g.gen_pmax.sum() - 0.25 * demand, rtol=1e-14)
