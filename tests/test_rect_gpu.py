"""Parity of the rectangular form's CUDA path (form = :rect, Sec. III-C-1)
with the FP64 oracle, through the C ABI; the same bar as the polar
parity tests (patterns bit for bit, values to 1e-12 of the oracle's entry
scale)."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2510_12897_b300 import opf, synth
from tests.test_parity_gpu import both, check_against_oracle, close, dev, host, run_all, torch  # noqa: F401

pytestmark = pytest.mark.gpu


def rpoints(g, m, count, seed):
    rng = np.random.default_rng(seed)
    gl = g if isinstance(g, list) else [g]
    for _ in range(count):
        x = np.concatenate([synth.random_point(h, rng, form="rect") for h in gl])
        yield x, rng.standard_normal(m)


def jtprod_check(torch, M, O, x, v):
    out = torch.full((M.n,), np.nan, dtype=torch.float64, device="cuda")
    M.eval_jtprod(dev(torch, x), dev(torch, v), out)
    torch.cuda.synchronize()
    r, c = O.jac_pattern()
    jv, js = O.jac(x, with_scale=True)
    ref = sp.coo_matrix((jv, (r, c)), shape=(O.m, O.n)).T @ v
    scale = sp.coo_matrix((js, (r, c)), shape=(O.m, O.n)).T @ np.abs(v)
    close("jtprod", host(out), ref, scale)


@pytest.mark.parametrize("seed", [30, 31])
def test_rect_general_terms(torch, oracle_mod, seed):
    """Shunts, taps, phase shifters, parallel branches; several launch shapes."""
    g = synth.case30(seed=seed, general=True)
    M, O = both(torch, oracle_mod, g, form="rect")
    for k, (x, lam) in enumerate(rpoints(g, M.m, 6, seed)):
        launch = [None, dict(branch_block=64, bus_block=32), dict(branch_ctas_per_sm=1, bus_ctas_per_sm=1),
                  dict(bus_order=1), dict(branch_block=512, bus_block=256), None][k]
        sigma = 0.0 if k == 3 else 0.8
        check_against_oracle(O, run_all(torch, M, x, lam, sigma, launch), x, lam, sigma, f"pt{k} ")
        jtprod_check(torch, M, O, x, lam)


def test_rect_isolated_bus(torch, oracle_mod):
    """A bus with no branch keeps its two diagonal Hessian entries and its
    magnitude row."""
    from tests.test_oracle_pins import tiny
    g = tiny(4, [(0, 1, 0.02, 0.1, 0.03, 1.0, 0.0, 2.0), (1, 2, 0.01, 0.07, 0.0, 1.02, 0.1, 1.0)],
             [(0, 0.05, 20.0, 1.0), (3, 0.02, 30.0, 0.0)], [(1, 0.9, 0.3), (3, 0.2, 0.1)],
             gs=[0.0, 0.03, 0.0, 0.01], bs=[0.02, 0.0, -0.01, 0.05])
    M, O = both(torch, oracle_mod, g, form="rect")
    for x, lam in rpoints(g, M.m, 3, seed=2):
        check_against_oracle(O, run_all(torch, M, x, lam, 1.0), x, lam, 1.0)


def test_rect_multiperiod_reserve(torch, oracle_mod):
    g = synth.multi_period(synth.case30(general=True), 5, seed=6, ramp_ratio=0.2)
    M, O = both(torch, oracle_mod, g, form="rect", reserve=0.2)
    for x, lam in rpoints(g, M.m, 3, seed=6):
        check_against_oracle(O, run_all(torch, M, x, lam, 1.0), x, lam, 1.0)
        jtprod_check(torch, M, O, x, lam)


def test_rect_batch_links_reserve(torch, oracle_mod):
    insts = synth.contingencies(synth.case30(general=True), 9, seed=7)
    M, O = both(torch, oracle_mod, insts, form="rect", link_ratios=[0.0] + [0.05 * k for k in range(1, 10)],
                reserve=0.1)
    for x, lam in rpoints(insts, M.m, 2, seed=8):
        check_against_oracle(O, run_all(torch, M, x, lam, 1.0), x, lam, 1.0)
        jtprod_check(torch, M, O, x, lam)


def test_rect_flat_start_and_flows(torch, oracle_mod):
    """Flat start: vr = 1 (inside [vmin, vmax]), vi = 0, p and q the flows;
    opf_eval_flows makes every flow row vanish at a random point."""
    g = synth.multi_period(synth.case30(general=True), 3, seed=4, ramp_ratio=0.2)
    M, O = both(torch, oracle_mod, g, form="rect")
    x = torch.full((M.n,), np.nan, dtype=torch.float64, device="cuda")
    M.flat_start(x)
    x = host(x)
    nbT, nl, T = g.nbus * 3, g.nbranch, 3
    assert np.all(x[:nbT] == 1.0) and np.all(x[nbT:2 * nbT] == 0.0)
    c, s = O.cons(x, with_scale=True)
    fl = slice(T, T + 4 * nl * T)
    close("flat flows", c[fl], np.zeros(4 * nl * T), s[fl])
    y0, _ = next(rpoints(g, M.m, 1, seed=14))
    dy = dev(torch, y0)
    M.eval_flows(dy)
    torch.cuda.synchronize()
    y = host(dy)
    c, s = O.cons(y, with_scale=True)
    close("flow rows", c[fl], np.zeros(4 * nl * T), s[fl])


def test_rect_case10k_full(torch, oracle_mod):
    """The 10,000-bus grid in rectangular form, every entry, default and
    autotuned launch shapes; J^T v."""
    g = synth.case10k()
    M, O = both(torch, oracle_mod, g, form="rect")
    x, lam = next(rpoints(g, M.m, 1, seed=10))
    check_against_oracle(O, run_all(torch, M, x, lam, 1.0), x, lam, 1.0, "default ")
    best, _ = M.autotune(dev(torch, x), dev(torch, lam), reps=3)
    check_against_oracle(O, run_all(torch, M, x, lam, 1.0, best), x, lam, 1.0, "tuned ")
    jtprod_check(torch, M, O, x, lam)


@pytest.mark.parametrize("which", ["case30g", "batch_links", "case10k", "hub"])
def test_rect_split_bus_phase(torch, oracle_mod, which):
    """The split bus phase in rectangular form (buses with more than six arc
    slots a warp each, groups of parallel arcs summed by a segmented scan of
    their aR and aI terms): every output against the oracle, one thread per
    item and persistent grids; a hub beyond 32 slots stays per thread."""
    from tests.test_hub_gpu import hub_grid
    g = {"case30g": lambda: synth.case30(general=True),
         "batch_links": lambda: synth.contingencies(synth.case30(general=True), 6, seed=3),
         "case10k": lambda: synth.case10k(),
         "hub": hub_grid}[which]()
    link = 0.2 if which == "batch_links" else 0.0
    M, O = both(torch, oracle_mod, g, link=link, form="rect")
    for k, (x, lam) in enumerate(rpoints(g, M.m, 2, seed=37)):
        for bu, cu in ((32, 0), (128, 2)):
            launch = dict(branch_block=64, bus_block=bu, branch_ctas_per_sm=0, bus_ctas_per_sm=cu, bus_order=2)
            sigma = 0.0 if k else 1.0
            check_against_oracle(O, run_all(torch, M, x, lam, sigma, launch), x, lam, sigma, f"pt{k} bu{bu} ")


@pytest.mark.parametrize("which", ["case30g", "batch_links", "case10k", "mp30"])
def test_rect_two_threads_per_branch(torch, oracle_mod, which):
    """branch_occupancy 2 in rectangular form: each branch item by two lanes,
    each evaluating its end's rows on (own, far) voltages and one angle row,
    exchanging the Hessian's aR and aI by shuffles; every output against the
    oracle, one thread per item and persistent grids, with the split bus
    phase and without."""
    g = {"case30g": lambda: synth.case30(general=True),
         "batch_links": lambda: synth.contingencies(synth.case30(general=True), 6, seed=3),
         "case10k": lambda: synth.case10k(),
         "mp30": lambda: synth.multi_period(synth.case30(general=True), 4, seed=8, ramp_ratio=0.2)}[which]()
    link = 0.2 if which == "batch_links" else 0.0
    M, O = both(torch, oracle_mod, g, link=link, form="rect")
    for k, (x, lam) in enumerate(rpoints(g, M.m, 2, seed=38)):
        for bb, cb, order in ((32, 0, 0), (256, 1, 2), (64, 0, 2)):
            launch = dict(branch_block=bb, bus_block=64, branch_ctas_per_sm=cb, bus_ctas_per_sm=0, bus_order=order,
                          branch_occupancy=2)
            sigma = 0.0 if k else 1.0
            check_against_oracle(O, run_all(torch, M, x, lam, sigma, launch), x, lam, sigma, f"pt{k} bb{bb} ")


@pytest.mark.parametrize("which", ["case30g", "isolated", "batch_links", "case10k", "mp30", "hub"])
def test_rect_fused_evaluation(torch, oracle_mod, which):
    """bus_order 3 in rectangular form: the one-kernel evaluation (whole buses
    packed into warps, each slot lane one lane of the rectangular two-lane
    kernel with the far end's aR and aI parts formed in place, per-bus sums
    of the diagonal parts and per-group sums of aR and aI by segmented
    scans); every output against the oracle, one or two warps per packed
    warp; a hub beyond 32 slots runs the split bus phase instead."""
    from tests.test_hub_gpu import hub_grid
    from tests.test_parity_gpu import isolated_bus_grid
    g = {"case30g": lambda: synth.case30(general=True),
         "isolated": isolated_bus_grid,
         "batch_links": lambda: synth.contingencies(synth.case30(general=True), 6, seed=3),
         "case10k": lambda: synth.case10k(),
         "mp30": lambda: synth.multi_period(synth.case30(general=True), 4, seed=8, ramp_ratio=0.2),
         "hub": hub_grid}[which]()
    link = 0.2 if which == "batch_links" else 0.0
    M, O = both(torch, oracle_mod, g, link=link, form="rect")
    for k, (x, lam) in enumerate(rpoints(g, M.m, 2, seed=41)):
        for bu, cu, occ in ((32, 0, 0), (128, 2, 0), (64, 0, 2)):
            launch = dict(branch_block=128, bus_block=bu, branch_ctas_per_sm=0, bus_ctas_per_sm=cu, bus_order=3,
                          branch_occupancy=occ)
            sigma = 0.0 if k else 0.9
            check_against_oracle(O, run_all(torch, M, x, lam, sigma, launch), x, lam, sigma,
                                 f"pt{k} bu{bu} occ{occ} ")


def test_rect_rejects_wide_angle_limits(torch):
    g = synth.case30()
    g = g.copy(br_angmax=np.where(np.arange(g.nbranch) == 3, np.pi / 2, g.br_angmax))
    opf.Model(g)  # polar accepts it
    with pytest.raises(opf.OpfError):
        opf.Model(g, form="rect")
