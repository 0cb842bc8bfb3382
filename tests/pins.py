"""Independent references used to pin the oracle (test code, not the oracle).

Everything here is written from textbook definitions, independently of
oracle/oracle.c: a dense bus admittance matrix and branch admittance rows
(MATPOWER's makeYbus construction), complex power injections
S = V conj(Y V), a polar Newton-Raphson power flow, and Richardson-extrapolated
central differences.
"""
from __future__ import annotations

import numpy as np


def ybus(g):
    """Dense Y_bus (nbus x nbus) and branch rows Yf, Yt (nbranch x nbus)."""
    nb, nl = g.nbus, len(g.br_f)
    Y = np.zeros((nb, nb), complex)
    Yf = np.zeros((nl, nb), complex)
    Yt = np.zeros((nl, nb), complex)
    for k in range(nl):
        f, t = int(g.br_f[k]), int(g.br_t[k])
        ys = 1.0 / complex(g.br_r[k], g.br_x[k])
        tau = g.br_tap[k] if g.br_tap[k] != 0 else 1.0
        ratio = tau * np.exp(1j * g.br_shift[k])
        y_tt = ys + 0.5j * g.br_b[k]
        y_ff = y_tt / (tau * tau)
        y_ft = -ys / np.conj(ratio)
        y_tf = -ys / ratio
        Y[f, f] += y_ff
        Y[f, t] += y_ft
        Y[t, f] += y_tf
        Y[t, t] += y_tt
        Yf[k, f] += y_ff
        Yf[k, t] += y_ft
        Yt[k, f] += y_tf
        Yt[k, t] += y_tt
    Y[np.arange(nb), np.arange(nb)] += g.bus_gs + 1j * g.bus_bs
    return Y, Yf, Yt


def bus_demand(g, period=0):
    Pd = np.zeros(g.nbus)
    Qd = np.zeros(g.nbus)
    np.add.at(Pd, g.load_bus, g.load_pd[period])
    np.add.at(Qd, g.load_bus, g.load_qd[period])
    return Pd, Qd


def newton_pf(g, pg_pv, vm_set=1.0, tol=1e-13, maxit=30):
    """Polar Newton-Raphson: slack = ref bus, PV = other generator buses (one
    generator each), PQ = the rest. Returns complex bus voltages."""
    nb = g.nbus
    Y, _, _ = ybus(g)
    Pd, Qd = bus_demand(g)
    gen_bus = np.asarray(g.gen_bus)
    ref = g.ref_bus
    pv = np.array([b for b in gen_bus if b != ref], dtype=int)
    pq = np.array([b for b in range(nb) if b != ref and b not in set(pv)], dtype=int)
    Pspec = -Pd.copy()
    Qspec = -Qd.copy()
    for gi, b in enumerate(gen_bus):
        if b != ref:
            Pspec[b] += pg_pv[gi]
    vm = np.ones(nb)
    vm[pv] = vm_set
    vm[ref] = vm_set
    va = np.zeros(nb)
    nonslack = np.concatenate([pv, pq])
    for _ in range(maxit):
        V = vm * np.exp(1j * va)
        S = V * np.conj(Y @ V)
        F = np.concatenate([S.real[nonslack] - Pspec[nonslack], S.imag[pq] - Qspec[pq]])
        if np.max(np.abs(F)) < tol:
            return V
        # dS/dva and dS/dvm (MATPOWER dSbus_dV, polar)
        Ibus = Y @ V
        dVa = 1j * np.diag(V) @ np.conj(np.diag(Ibus) - Y @ np.diag(V))
        En = V / np.abs(V)
        dVm = np.diag(V) @ np.conj(Y @ np.diag(En)) + np.conj(np.diag(Ibus)) @ np.diag(En)
        J = np.block([
            [dVa.real[np.ix_(nonslack, nonslack)], dVm.real[np.ix_(nonslack, pq)]],
            [dVa.imag[np.ix_(pq, nonslack)], dVm.imag[np.ix_(pq, pq)]],
        ])
        dx = np.linalg.solve(J, -F)
        va[nonslack] += dx[: len(nonslack)]
        vm[pq] += dx[len(nonslack):]
    raise RuntimeError("power flow did not converge")


def central_diff(fun, x, h=1e-4):
    """Jacobian of fun at x by Richardson-extrapolated central differences:
    D(h) = (f(x+h) - f(x-h)) / 2h,  R = (4 D(h/2) - D(h)) / 3  (error O(h^4))."""
    x = np.asarray(x, float)
    f0 = np.asarray(fun(x))
    out = np.zeros((f0.size, x.size))
    for j in range(x.size):
        def d(hh):
            xp = x.copy()
            xm = x.copy()
            xp[j] += hh
            xm[j] -= hh
            return (np.asarray(fun(xp)) - np.asarray(fun(xm))) / (2 * hh)
        out[:, j] = (4 * d(h / 2) - d(h)) / 3
    return out


def groups(g):
    """Slices of the variable groups of one single-period instance."""
    nb, ng, na = g.nbus, len(g.gen_bus), 2 * len(g.br_f)
    o = np.cumsum([0, nb, nb, ng, ng, na, na])
    names = ["va", "vm", "pg", "qg", "p", "q"]
    return {k: slice(o[i], o[i + 1]) for i, k in enumerate(names)}


def rows(g):
    """Slices of the constraint groups of one single-period instance."""
    nl, nb = len(g.br_f), g.nbus
    sizes = [("ref", 1), ("fpf", nl), ("fqf", nl), ("fpt", nl), ("fqt", nl), ("ang", nl),
             ("pb", nb), ("qb", nb), ("thf", nl), ("tht", nl)]
    out, o = {}, 0
    for k, s in sizes:
        out[k] = slice(o, o + s)
        o += s
    return out
