"""Seeded synthetic power grids and evaluation points.

This module is the one place where inputs are drawn. It serves both the CUDA
path and the FP64 oracle and holds none of the method's arithmetic: it draws
network parameters, loads and points from fixed distributions and nothing
else (no power-flow formula, no derivative, no layout of the NLP).

The networks stand in for the pglib-opf cases the paper benchmarks (Sec. IV-A,
IV-B, IV-C), which are not available here. Recipe:

* buses at uniform positions in the unit square; a random spanning tree in
  which each bus, in random order, attaches to its nearest already placed bus;
  then ``nbranch - (nbus - 1)`` extra edges, each from a random bus to a random
  one of its 8 nearest non-adjacent buses, never parallel to an existing edge;
* r ~ U(0.01, 0.1), x ~ U(0.05, 0.3), b ~ U(0, 0.05) p.u., tap 1, shift 0,
  rate_a ~ U(0.5, 2), angle-difference limits +-30 degrees;
* generators at distinct random buses, c2 ~ U(0.01, 0.1), c1 ~ U(10, 40),
  c0 = 0, Pg in [0, 2], Qg in [-1, 1]; the reference bus is generator 0's bus;
* loads at round(0.7 nbus) distinct random buses, Pd ~ U(0, 0.5), Qd = 0.3 Pd;
* V in [0.9, 1.1], no shunts.

``general=True`` additionally draws shunts, off-nominal taps and phase shifts
and a few parallel branches, so that parity tests reach every term of the
formulation (the paper's cases contain all of them).

The draw above does not make an OPF instance feasible: on the 2,000-bus
grid no dispatch keeps every line within rate_a even in the lossless DC
approximation. The paper's cases are feasible instances, and the learned
warm start is judged by its constraint violation, so its grid goes through
``secure_ratings``: a linear program (DC flows on the series susceptances,
HiGHS) finds the dispatch at 1.2 times the base load that overloads the
lines least (in L1), and each line's rating becomes max(rate_a, 1.3 |flow|)
for that dispatch. Only lines the dispatch needs are lifted; the draw is
unchanged elsewhere. This DC dispatch is a data-generation step that neither
side of the evaluation computes.

Multi-period loads follow the paper's demand-curve interface (Sec. III-C-2,
``mpopf_model`` with a curve): every load is scaled per period by one daily
curve, here a seeded sinusoid, times lognormal(0, 0.05) noise per load.

Storage follows the paper's multi-period-with-storage cases (Sec. IV-B):
units at the buses with the largest 10% of active load, energy rating 1.5
times the bus's (base) demand; the paper takes the ratio of energy to
charge and discharge rating from its storage reference without printing it,
here 2 hours; thermal rating 1.1 times the larger rating, reactive limits
half of it either way, efficiencies 0.95, series resistance 0.02 p.u., no
standby loss, initial energy half the rating, periods spanning one day.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np
from scipy.spatial import cKDTree

DEG = math.pi / 180.0


@dataclass
class Storage:
    """Storage units of one network (multi-period model with storage)."""

    bus: np.ndarray
    energy_rating: np.ndarray
    charge_rating: np.ndarray
    discharge_rating: np.ndarray
    thermal_rating: np.ndarray
    eta_c: np.ndarray
    eta_d: np.ndarray
    r: np.ndarray
    p_loss: np.ndarray
    qmin: np.ndarray
    qmax: np.ndarray
    e_init: np.ndarray
    dt: float

    @property
    def nstor(self) -> int:
        return int(self.bus.shape[0])


@dataclass
class Grid:
    """A network as structure-of-arrays (0-based indices, per-unit values)."""

    nbus: int
    bus_vmin: np.ndarray
    bus_vmax: np.ndarray
    bus_gs: np.ndarray
    bus_bs: np.ndarray
    br_f: np.ndarray
    br_t: np.ndarray
    br_r: np.ndarray
    br_x: np.ndarray
    br_b: np.ndarray
    br_tap: np.ndarray
    br_shift: np.ndarray
    br_rate_a: np.ndarray
    br_angmin: np.ndarray
    br_angmax: np.ndarray
    gen_bus: np.ndarray
    gen_pmin: np.ndarray
    gen_pmax: np.ndarray
    gen_qmin: np.ndarray
    gen_qmax: np.ndarray
    gen_c2: np.ndarray
    gen_c1: np.ndarray
    gen_c0: np.ndarray
    load_bus: np.ndarray
    load_pd: np.ndarray  # [nperiod, nload]
    load_qd: np.ndarray  # [nperiod, nload]
    ref_bus: int
    ramp_ratio: float = 0.0
    xy: np.ndarray | None = field(default=None, repr=False)
    storage: Storage | None = field(default=None, repr=False)

    @property
    def nbranch(self) -> int:
        return int(self.br_f.shape[0])

    @property
    def ngen(self) -> int:
        return int(self.gen_bus.shape[0])

    @property
    def nload(self) -> int:
        return int(self.load_bus.shape[0])

    @property
    def nperiod(self) -> int:
        return int(self.load_pd.shape[0])

    def copy(self, **changes) -> "Grid":
        return replace(self, **changes)


def _spanning_tree(xy: np.ndarray, rng: np.random.Generator) -> list[tuple[int, int]]:
    nb = xy.shape[0]
    order = rng.permutation(nb)
    edges = []
    # distance from every bus to the nearest placed bus, and which one it is
    best_d = np.full(nb, np.inf)
    best_j = np.full(nb, -1, dtype=np.int64)
    placed = np.zeros(nb, dtype=bool)
    for step, i in enumerate(order):
        if step > 0:
            edges.append((int(i), int(best_j[i])))
        placed[i] = True
        d = np.sum((xy - xy[i]) ** 2, axis=1)
        upd = (d < best_d) & ~placed
        best_d[upd] = d[upd]
        best_j[upd] = i
    return edges


def _extra_edges(xy, edges, n_extra, rng, allow_parallel=0):
    nb = xy.shape[0]
    adj = [set() for _ in range(nb)]
    for f, t in edges:
        adj[f].add(t)
        adj[t].add(f)
    tree = cKDTree(xy)
    out = []
    guard = 0
    while len(out) < n_extra:
        guard += 1
        if guard > 100 * (n_extra + 10):
            raise RuntimeError("could not place extra edges")
        i = int(rng.integers(nb))
        k = min(nb, 9 + len(adj[i]))
        _, idx = tree.query(xy[i], k=k)
        cand = [int(j) for j in np.atleast_1d(idx) if j != i and j not in adj[i]][:8]
        if not cand:
            continue
        j = cand[int(rng.integers(len(cand)))]
        adj[i].add(j)
        adj[j].add(i)
        out.append((i, j))
    # a few parallel branches (general grids only): duplicate existing edges
    all_edges = edges + out
    for _ in range(allow_parallel):
        e = all_edges[int(rng.integers(len(all_edges)))]
        out.append(e)
    return out


def make_grid(nbus: int, nbranch: int, ngen: int, seed: int, nload: int | None = None,
              general: bool = False) -> Grid:
    """One seeded synthetic network (single period)."""
    if nbranch < nbus - 1:
        raise ValueError("need at least a spanning tree")
    rng = np.random.default_rng(seed)
    xy = rng.random((nbus, 2))
    tree = _spanning_tree(xy, rng)
    npar = 0
    if general:
        npar = max(1, (nbranch - (nbus - 1)) // 8)
    n_extra = nbranch - (nbus - 1) - npar
    if n_extra < 0:
        npar, n_extra = nbranch - (nbus - 1), 0
    extra = _extra_edges(xy, tree, n_extra, rng, allow_parallel=npar)
    edges = tree + extra
    perm = rng.permutation(len(edges))
    edges = [edges[p] for p in perm]
    # random orientation of each branch
    fl, tl = [], []
    for (a, b) in edges:
        if rng.random() < 0.5:
            a, b = b, a
        fl.append(a)
        tl.append(b)
    nl = len(edges)
    br_f = np.asarray(fl, dtype=np.int32)
    br_t = np.asarray(tl, dtype=np.int32)
    br_r = rng.uniform(0.01, 0.1, nl)
    br_x = rng.uniform(0.05, 0.3, nl)
    br_b = rng.uniform(0.0, 0.05, nl)
    br_tap = np.ones(nl)
    br_shift = np.zeros(nl)
    if general:
        sel = rng.random(nl) < 0.3
        br_tap[sel] = rng.uniform(0.9, 1.1, int(sel.sum()))
        sel = rng.random(nl) < 0.2
        br_shift[sel] = rng.uniform(-10 * DEG, 10 * DEG, int(sel.sum()))
    br_rate_a = rng.uniform(0.5, 2.0, nl)
    br_angmin = np.full(nl, -30 * DEG)
    br_angmax = np.full(nl, 30 * DEG)

    gen_bus = rng.choice(nbus, size=ngen, replace=False).astype(np.int32)
    gen_c2 = rng.uniform(0.01, 0.1, ngen)
    gen_c1 = rng.uniform(10.0, 40.0, ngen)
    gen_c0 = np.zeros(ngen)
    if general:
        gen_c0 = rng.uniform(0.0, 5.0, ngen)
    gen_pmin = np.zeros(ngen)
    gen_pmax = np.full(ngen, 2.0)
    gen_qmin = np.full(ngen, -1.0)
    gen_qmax = np.full(ngen, 1.0)

    if nload is None:
        nload = int(round(0.7 * nbus))
    load_bus = rng.choice(nbus, size=nload, replace=False).astype(np.int32)
    pd = rng.uniform(0.0, 0.5, nload)
    qd = 0.3 * pd

    bus_gs = np.zeros(nbus)
    bus_bs = np.zeros(nbus)
    if general:
        sel = rng.random(nbus) < 0.3
        bus_gs[sel] = rng.uniform(0.0, 0.05, int(sel.sum()))
        sel = rng.random(nbus) < 0.3
        bus_bs[sel] = rng.uniform(-0.05, 0.05, int(sel.sum()))

    return Grid(
        nbus=nbus,
        bus_vmin=np.full(nbus, 0.9), bus_vmax=np.full(nbus, 1.1),
        bus_gs=bus_gs, bus_bs=bus_bs,
        br_f=br_f, br_t=br_t, br_r=br_r, br_x=br_x, br_b=br_b,
        br_tap=br_tap, br_shift=br_shift, br_rate_a=br_rate_a,
        br_angmin=br_angmin, br_angmax=br_angmax,
        gen_bus=gen_bus, gen_pmin=gen_pmin, gen_pmax=gen_pmax,
        gen_qmin=gen_qmin, gen_qmax=gen_qmax,
        gen_c2=gen_c2, gen_c1=gen_c1, gen_c0=gen_c0,
        load_bus=load_bus, load_pd=pd[None, :].copy(), load_qd=qd[None, :].copy(),
        ref_bus=int(gen_bus[0]), xy=xy,
    )


def daily_curve(nperiod: int, seed: int, amplitude: float = 0.2) -> np.ndarray:
    """One seeded daily demand curve: 1 + a sin(2 pi t / T + phi)."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    t = np.arange(nperiod)
    return 1.0 + amplitude * np.sin(2.0 * math.pi * t / nperiod + phi)


def multi_period(g: Grid, nperiod: int, seed: int, ramp_ratio: float = 0.2,
                 noise_sigma: float = 0.05) -> Grid:
    """Multi-period copy of ``g``: loads scaled per period by a daily curve
    times per-load lognormal(0, noise_sigma) noise; ramp ratio recorded."""
    rng = np.random.default_rng(seed + 7919)
    curve = daily_curve(nperiod, seed)
    noise = np.exp(rng.normal(0.0, noise_sigma, (nperiod, g.nload)))
    scale = curve[:, None] * noise
    pd = g.load_pd[0][None, :] * scale
    qd = g.load_qd[0][None, :] * scale
    return g.copy(load_pd=pd, load_qd=qd, ramp_ratio=float(ramp_ratio))


def scenarios(g: Grid, count: int, seed: int, low: float = 0.8, high: float = 1.2) -> Grid:
    """``count`` load scenarios of ``g`` as the periods of one model without
    ramp rows: scenario s scales every load by its own U(low, high) factor."""
    rng = np.random.default_rng(seed + 31337)
    scale = rng.uniform(low, high, count)[:, None]
    return g.copy(load_pd=g.load_pd[0][None, :] * scale, load_qd=g.load_qd[0][None, :] * scale,
                  ramp_ratio=0.0)


def load_samples(g: Grid, count: int, seed: int, rank: int = 8, share: float = 0.7):
    """``count`` load profiles of ``g`` for the learned warm start: every
    load's Pd and Qd scaled by factors that are U(0.8, 1.2) marginally and
    correlated across loads through ``rank`` seeded common factors (a normal
    copula: z = sqrt(share) F w + sqrt(1 - share) e, factor = 0.8 + 0.4 Phi(z),
    each row of F of unit norm). Returns (pd, qd), each [count][nload]."""
    from scipy.special import ndtr
    rng = np.random.default_rng(seed + 4242)
    nload = g.nload
    F = rng.standard_normal((nload, rank))
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    w = rng.standard_normal((count, rank))
    common = w @ F.T
    zp = math.sqrt(share) * common + math.sqrt(1.0 - share) * rng.standard_normal((count, nload))
    zq = math.sqrt(share) * common + math.sqrt(1.0 - share) * rng.standard_normal((count, nload))
    a = 0.8 + 0.4 * ndtr(zp)
    b = 0.8 + 0.4 * ndtr(zq)
    return g.load_pd[0][None, :] * a, g.load_qd[0][None, :] * b


def secure_ratings(g: Grid, load_scale: float = 1.2, margin: float = 1.3,
                   angle_frac: float = 0.8) -> Grid:
    """Copy of single-period ``g`` with line ratings lifted so that the DC
    dispatch of ``load_scale`` times the base load that minimises the total
    overload stays within them, with ``margin`` (recipe in the module
    docstring). Angle differences of that dispatch are held within
    ``angle_frac`` of the limits."""
    import scipy.sparse as sp
    from scipy.optimize import linprog
    nb, nl, ng = g.nbus, g.nbranch, g.ngen
    f, t = g.br_f.astype(np.int64), g.br_t.astype(np.int64)
    bser = g.br_x / (g.br_r ** 2 + g.br_x ** 2)
    k = np.arange(nl)
    # variables: theta [nb], pg [ng], overload s [nl] >= 0
    nv = nb + ng + nl
    # DC flow of branch k: bser_k (theta_f - theta_t), as a row over theta
    D = sp.csr_matrix((np.concatenate([bser, -bser]), (np.concatenate([k, k]), np.concatenate([f, t]))),
                      shape=(nl, nb))
    inc = sp.csr_matrix((np.concatenate([np.ones(nl), -np.ones(nl)]),
                         (np.concatenate([f, t]), np.concatenate([k, k]))), shape=(nb, nl))
    G = sp.csr_matrix((np.ones(ng), (g.gen_bus.astype(np.int64), np.arange(ng))), shape=(nb, ng))
    pd = np.zeros(nb)
    np.add.at(pd, g.load_bus, load_scale * g.load_pd[0])
    ref = sp.csr_matrix(([1.0], ([0], [int(g.ref_bus)])), shape=(1, nb))
    A_eq = sp.vstack([sp.hstack([inc @ D, -G, sp.csr_matrix((nb, nl))]),
                      sp.hstack([ref, sp.csr_matrix((1, ng + nl))])]).tocsr()
    b_eq = np.concatenate([-pd, [0.0]])
    S = -sp.identity(nl, format="csr")
    Z = sp.csr_matrix((nl, ng))
    A = sp.csr_matrix((np.concatenate([np.ones(nl), -np.ones(nl)]), (np.concatenate([k, k]),
                       np.concatenate([f, t]))), shape=(nl, nb))
    A_ub = sp.vstack([sp.hstack([D, Z, S]), sp.hstack([-D, Z, S]),
                      sp.hstack([A, Z, sp.csr_matrix((nl, nl))]),
                      sp.hstack([-A, Z, sp.csr_matrix((nl, nl))])]).tocsr()
    b_ub = np.concatenate([g.br_rate_a, g.br_rate_a, angle_frac * g.br_angmax, -angle_frac * g.br_angmin])
    c = np.concatenate([np.zeros(nb + ng), np.ones(nl)])
    bounds = [(None, None)] * nb + list(zip(g.gen_pmin, g.gen_pmax)) + [(0.0, None)] * nl
    res = linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=A_eq, b_eq=b_eq, bounds=bounds, method="highs")
    if res.status != 0:
        raise RuntimeError("secure_ratings: " + res.message)
    flow = D @ res.x[:nb]
    return g.copy(br_rate_a=np.maximum(g.br_rate_a, margin * np.abs(flow)))


def bridges(nbus: int, f: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Boolean mask of bridge branches (iterative Tarjan low-link)."""
    nl = len(f)
    adj = [[] for _ in range(nbus)]
    for k in range(nl):
        adj[int(f[k])].append((int(t[k]), k))
        adj[int(t[k])].append((int(f[k]), k))
    disc = [-1] * nbus
    low = [0] * nbus
    is_bridge = np.zeros(nl, dtype=bool)
    timer = 0
    for root in range(nbus):
        if disc[root] >= 0:
            continue
        disc[root] = low[root] = timer
        timer += 1
        stack = [(root, -1, iter(adj[root]))]
        while stack:
            v, pe, it = stack[-1]
            advanced = False
            for (w, k) in it:
                if k == pe:
                    continue
                if disc[w] < 0:
                    disc[w] = low[w] = timer
                    timer += 1
                    stack.append((w, k, iter(adj[w])))
                    advanced = True
                    break
                low[v] = min(low[v], disc[w])
            if not advanced:
                stack.pop()
                if stack:
                    u = stack[-1][0]
                    low[u] = min(low[u], low[v])
                    if low[v] > disc[u]:
                        is_bridge[pe] = True
    return is_bridge


def drop_branch(g: Grid, k: int) -> Grid:
    """The N-1 contingency network without branch ``k``."""
    keep = np.ones(g.nbranch, dtype=bool)
    keep[k] = False
    kw = {name: getattr(g, name)[keep] for name in (
        "br_f", "br_t", "br_r", "br_x", "br_b", "br_tap", "br_shift",
        "br_rate_a", "br_angmin", "br_angmax")}
    return g.copy(**kw)


def contingencies(g: Grid, count: int, seed: int) -> list[Grid]:
    """Base case followed by ``count`` N-1 networks, each without one seeded
    non-bridge branch (so every instance stays connected)."""
    rng = np.random.default_rng(seed + 104729)
    cand = np.flatnonzero(~bridges(g.nbus, g.br_f, g.br_t))
    if len(cand) < count:
        raise ValueError("not enough non-bridge branches")
    drop = rng.choice(cand, size=count, replace=False)
    return [g] + [drop_branch(g, int(k)) for k in drop]


# ----------------------------------------------------------------------------
# evaluation points
# ----------------------------------------------------------------------------

def n_vars(g: Grid) -> int:
    T = g.nperiod
    ns = g.storage.nstor if g.storage is not None else 0
    return T * (2 * g.nbus + 2 * g.ngen + 4 * g.nbranch + 5 * ns)


def with_storage(g: Grid, share: float = 0.1, energy_factor: float = 1.5, hours: float = 2.0) -> Grid:
    """Copy of multi-period ``g`` with storage units at the buses carrying the
    largest ``share`` of base active load (recipe in the module docstring)."""
    pd = np.zeros(g.nbus)
    np.add.at(pd, g.load_bus, g.load_pd[0])
    count = max(1, int(round(share * np.count_nonzero(pd))))
    bus = np.sort(np.argsort(-pd, kind="stable")[:count]).astype(np.int32)
    E = energy_factor * pd[bus]
    rate = E / hours
    S = 1.1 * rate
    k = bus.shape[0]
    st = Storage(bus=bus, energy_rating=E, charge_rating=rate.copy(), discharge_rating=rate.copy(),
                 thermal_rating=S, eta_c=np.full(k, 0.95), eta_d=np.full(k, 0.95), r=np.full(k, 0.02),
                 p_loss=np.zeros(k), qmin=-0.5 * S, qmax=0.5 * S, e_init=0.5 * E, dt=24.0 / g.nperiod)
    return g.copy(storage=st)


def random_point(g: Grid, rng: np.random.Generator, form: str = "polar") -> np.ndarray:
    """x = [va, vm, pg, qg, p, q], each group ``elem + count * period``:
    va ~ U(-pi/6, pi/6), vm ~ U(vmin, vmax), pg and qg uniform in their
    bounds, p, q ~ U(-rate_a, rate_a) of the arc's branch. ``form="rect"``
    gives the same draw in rectangular voltages, vr = vm cos va and
    vi = vm sin va in the places of va and vm."""
    T, nb, ng, nl = g.nperiod, g.nbus, g.ngen, g.nbranch
    na = 2 * nl
    va = rng.uniform(-math.pi / 6, math.pi / 6, (T, nb))
    vm = rng.uniform(g.bus_vmin, g.bus_vmax, (T, nb))
    pg = rng.uniform(g.gen_pmin, g.gen_pmax, (T, ng))
    qg = rng.uniform(g.gen_qmin, g.gen_qmax, (T, ng))
    rate = np.concatenate([g.br_rate_a, g.br_rate_a])
    p = rng.uniform(-rate, rate, (T, na))
    q = rng.uniform(-rate, rate, (T, na))
    if form == "rect":
        va, vm = vm * np.cos(va), vm * np.sin(va)
    parts = [va, vm, pg, qg, p, q]
    st = g.storage
    if st is not None:  # ps, qs, sc, sd, se uniform in their bounds
        parts += [rng.uniform(-st.thermal_rating, st.thermal_rating, (T, st.nstor)),
                  rng.uniform(st.qmin, st.qmax, (T, st.nstor)),
                  rng.uniform(0.0, st.charge_rating, (T, st.nstor)),
                  rng.uniform(0.0, st.discharge_rating, (T, st.nstor)),
                  rng.uniform(0.0, st.energy_rating, (T, st.nstor))]
    return np.concatenate([a.ravel() for a in parts])


def random_multipliers(m: int, rng: np.random.Generator) -> np.ndarray:
    return rng.standard_normal(m)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def case30(seed: int = 30, general: bool = False) -> Grid:
    """30 buses, 41 branches, 6 generators, 21 loads."""
    return make_grid(30, 41, 6, seed, general=general)


def case10k(seed: int = 10000) -> Grid:
    """10,000 buses, 13,000 branches, 2,500 generators, 7,000 loads."""
    return make_grid(10000, 13000, 2500, seed)


def case2k(seed: int = 2000) -> Grid:
    """2,000 buses, 2,600 branches, 500 generators, 1,400 loads."""
    return make_grid(2000, 2600, 500, seed)


def case1k(seed: int = 1000) -> Grid:
    """1,000 buses, 1,300 branches, 250 generators, 700 loads."""
    return make_grid(1000, 1300, 250, seed)


def case2k_secure(seed: int = 2000) -> Grid:
    """The 2,000-bus grid with ratings lifted by ``secure_ratings`` (the
    learned warm start's grid)."""
    return secure_ratings(case2k(seed))


def mp2k(nperiod: int = 96, seed: int = 2000) -> Grid:
    """The 2,000-bus grid over ``nperiod`` periods, ramp 0.2 Pmax."""
    return multi_period(case2k(seed), nperiod, seed, ramp_ratio=0.2)


def mp2k_storage(nperiod: int = 96, seed: int = 2000) -> Grid:
    """The 2,000-bus grid over ``nperiod`` periods with storage units."""
    return with_storage(mp2k(nperiod, seed))


def sc1k(ncont: int = 500, seed: int = 1000) -> list[Grid]:
    """The 1,000-bus grid plus ``ncont`` N-1 contingencies."""
    return contingencies(case1k(seed), ncont, seed)
