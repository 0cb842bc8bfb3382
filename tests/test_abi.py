"""Host-side checks of libopf (no GPU needed): the library loads and exports
every entry point include/opf.h declares; the layout-generated sparsity
patterns and bounds equal the oracle's bit for bit; invalid input is
rejected with the documented codes before any device work."""
import ctypes
import os

import numpy as np
import pytest

from paper_2510_12897_b300 import opf, synth


@pytest.fixture(scope="module")
def L():
    from paper_2510_12897_b300 import build
    build.build()
    return opf.lib()


def test_exports_every_declared_symbol(L):
    inc = os.path.dirname(opf.HEADER)
    names = (opf.declared_symbols() + opf.declared_symbols(os.path.join(inc, "opf_warm.h"))
             + opf.declared_symbols(os.path.join(inc, "opf_al.h")))
    assert "opf_warm_train_step" in names and "opf_eval_all" in names and "opf_al_iterate" in names
    assert "opf_eval_jac_hess" in names and "opf_model_create" in names
    for name in names:
        assert hasattr(L, name), name


def _grids():
    g30 = synth.case30()
    g30g = synth.case30(general=True)
    return {
        "case30": g30,
        "case30_general": g30g,
        "mp30x5": synth.multi_period(g30g, 5, seed=3, ramp_ratio=0.2),
        "batch30": synth.contingencies(g30, 6, seed=4),
    }


@pytest.mark.parametrize("name", ["case30", "case30_general", "mp30x5", "batch30"])
def test_patterns_and_bounds_equal_oracle(L, oracle_mod, name):
    g = _grids()[name]
    link = 0.2 if isinstance(g, list) else 0.0
    M = opf.Model(g, link_ratio=link, structure_only=True)
    O = oracle_mod.Oracle(g, link_ratio=link)
    assert (M.n, M.m, M.nnzj, M.nnzh) == (O.n, O.m, O.nnzj, O.nnzh)
    for a, b in zip(M.jac_pattern(), O.jac_pattern()):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(M.hess_pattern(), O.hess_pattern()):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(M.bounds(), O.bounds()):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("name,opts", [
    ("batch30", dict(link_ratios=[0.0, 0.1, 0.3, 0.05, 0.2, 0.15, 0.25], reserve=0.1)),
    ("mp30x5", dict(reserve=0.2)),
    ("case30_general", dict(reserve=0.05)),
])
def test_reserve_and_corrective_patterns_equal_oracle(L, oracle_mod, name, opts):
    """Reserve rows (one per instance and period, after the linking rows) and
    per-instance corrective ratios: sizes, patterns and bounds equal the
    oracle's bit for bit."""
    g = _grids()[name]
    M = opf.Model(g, structure_only=True, **opts)
    O = oracle_mod.Oracle(g, **opts)
    assert (M.n, M.m, M.nnzj, M.nnzh) == (O.n, O.m, O.nnzj, O.nnzh)
    for a, b in zip(M.jac_pattern() + M.hess_pattern(), O.jac_pattern() + O.hess_pattern()):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(M.bounds(), O.bounds()):
        np.testing.assert_array_equal(a, b)
    # one reserve row per instance and period on top of the plain model
    nres = sum(x.nperiod for x in (g if isinstance(g, list) else [g]))
    plain = oracle_mod.Oracle(g, link_ratio=max(opts.get("link_ratios") or [0.0]))
    assert O.m == plain.m + nres


def test_reserve_options_rejected(L):
    g = synth.contingencies(synth.case30(), 2, seed=4)
    _expect(opf.OPF_EINVAL, opf.Model, g, structure_only=True, reserve=-0.1)
    _expect(opf.OPF_EINVAL, opf.Model, g, structure_only=True, link_ratios=[0.0, float("nan"), 0.1])


@pytest.mark.slow
def test_patterns_10k_equal_oracle(L, oracle_mod):
    g = synth.case10k()
    M = opf.Model(g, structure_only=True)
    O = oracle_mod.Oracle(g)
    assert (M.n, M.m, M.nnzj, M.nnzh) == (77000, 111001, 415001, 136500)
    for a, b in zip(M.jac_pattern() + M.hess_pattern(), O.jac_pattern() + O.hess_pattern()):
        np.testing.assert_array_equal(a, b)


def test_isolated_bus_and_empty_parts(L, oracle_mod):
    """A bus with no branch keeps only (vm, vm) in the Hessian; zero loads
    and a generator-free bus are fine."""
    g = synth.case30(general=True)
    nb = g.nbus + 1  # one extra isolated bus
    g2 = g.copy(nbus=nb, bus_vmin=np.append(g.bus_vmin, 0.95), bus_vmax=np.append(g.bus_vmax, 1.05),
                bus_gs=np.append(g.bus_gs, 0.01), bus_bs=np.append(g.bus_bs, 0.02))
    M = opf.Model(g2, structure_only=True)
    O = oracle_mod.Oracle(g2)
    for a, b in zip(M.jac_pattern() + M.hess_pattern(), O.jac_pattern() + O.hess_pattern()):
        np.testing.assert_array_equal(a, b)
    single = g.copy(nbus=1, bus_vmin=g.bus_vmin[:1], bus_vmax=g.bus_vmax[:1], bus_gs=g.bus_gs[:1],
                    bus_bs=g.bus_bs[:1], br_f=g.br_f[:0], br_t=g.br_t[:0], br_r=g.br_r[:0],
                    br_x=g.br_x[:0], br_b=g.br_b[:0], br_tap=g.br_tap[:0], br_shift=g.br_shift[:0],
                    br_rate_a=g.br_rate_a[:0], br_angmin=g.br_angmin[:0], br_angmax=g.br_angmax[:0],
                    gen_bus=np.zeros(1, np.int32), gen_pmin=g.gen_pmin[:1], gen_pmax=g.gen_pmax[:1],
                    gen_qmin=g.gen_qmin[:1], gen_qmax=g.gen_qmax[:1], gen_c2=g.gen_c2[:1],
                    gen_c1=g.gen_c1[:1], gen_c0=g.gen_c0[:1], load_bus=np.zeros(0, np.int32),
                    load_pd=np.zeros((1, 0)), load_qd=np.zeros((1, 0)), ref_bus=0)
    M = opf.Model(single, structure_only=True)
    O = oracle_mod.Oracle(single)
    assert (M.n, M.m, M.nnzj, M.nnzh) == (O.n, O.m, O.nnzj, O.nnzh) == (4, 3, 5, 2)
    for a, b in zip(M.jac_pattern() + M.hess_pattern(), O.jac_pattern() + O.hess_pattern()):
        np.testing.assert_array_equal(a, b)


def _expect(code, fn, *a, **k):
    with pytest.raises(opf.OpfError) as e:
        fn(*a, **k)
    assert e.value.code == code, str(e.value)


def test_invalid_networks_rejected(L):
    g = synth.case30()
    f = g.br_f.copy()
    f[3] = g.br_t[3]
    _expect(opf.OPF_EINVAL, opf.Model, g.copy(br_f=f), structure_only=True)  # self-loop
    f = g.br_f.copy()
    f[0] = g.nbus
    _expect(opf.OPF_EINVAL, opf.Model, g.copy(br_f=f), structure_only=True)  # out of range
    r, x = g.br_r.copy(), g.br_x.copy()
    r[2] = x[2] = 0.0
    _expect(opf.OPF_EINVAL, opf.Model, g.copy(br_r=r, br_x=x), structure_only=True)
    tap = g.br_tap.copy()
    tap[1] = -1.0
    _expect(opf.OPF_EINVAL, opf.Model, g.copy(br_tap=tap), structure_only=True)
    gb = g.gen_bus.copy()
    gb[0] = -1
    _expect(opf.OPF_EINVAL, opf.Model, g.copy(gen_bus=gb), structure_only=True)
    lb = g.load_bus.copy()
    lb[0] = 999
    _expect(opf.OPF_EINVAL, opf.Model, g.copy(load_bus=lb), structure_only=True)
    c2 = g.gen_c2.copy()
    c2[0] = np.nan
    _expect(opf.OPF_EINVAL, opf.Model, g.copy(gen_c2=c2), structure_only=True)
    _expect(opf.OPF_EINVAL, opf.Model, g.copy(ref_bus=g.nbus), structure_only=True)
    _expect(opf.OPF_EINVAL, opf.Model, g.copy(load_pd=np.zeros((0, g.nload)),
                                              load_qd=np.zeros((0, g.nload))), structure_only=True)
    # linking rows need equal generator counts
    g2 = g.copy(gen_bus=g.gen_bus[:-1], gen_pmin=g.gen_pmin[:-1], gen_pmax=g.gen_pmax[:-1],
                gen_qmin=g.gen_qmin[:-1], gen_qmax=g.gen_qmax[:-1], gen_c2=g.gen_c2[:-1],
                gen_c1=g.gen_c1[:-1], gen_c0=g.gen_c0[:-1])
    _expect(opf.OPF_ESTATE, opf.Model, [g, g2], link_ratio=0.2, structure_only=True)


def test_null_and_state_errors(L):
    _expect(opf.OPF_EINVAL, opf._check, L.opf_dims(None, None, None, None, None))
    _expect(opf.OPF_EINVAL, opf._check, L.opf_model_create(None, ctypes.byref(ctypes.c_void_p())))
    M = opf.Model(synth.case30(), structure_only=True)
    # a structure-only model refuses evaluation without touching a device
    _expect(opf.OPF_ESTATE, opf._check, L.opf_eval_cons(M.h, ctypes.c_void_p(16), ctypes.c_void_p(16), None))
    _expect(opf.OPF_ESTATE, opf._check, L.opf_flat_start(M.h, ctypes.c_void_p(16), None))
    _expect(opf.OPF_EINVAL, opf._check, L.opf_sparsity(M.h, 7, ctypes.cast(None, opf._i64p),
                                                       ctypes.cast(None, opf._i64p)))
    cfg = opf.OpfLaunch(100, 128, 0, 0)
    _expect(opf.OPF_EINVAL, opf._check, L.opf_set_launch(M.h, ctypes.byref(cfg)))
    assert b"multiple of 32" in L.opf_last_error()
    for bad in (opf.OpfLaunch(512, 128, 0, 0, 0, 1), opf.OpfLaunch(1024, 128, 0, 0, 0, 0),
                opf.OpfLaunch(128, 128, 0, 0, 4, 0), opf.OpfLaunch(128, 128, 0, 0, 0, -1),
                opf.OpfLaunch(128, 128, 0, 0, 0, 3)):
        _expect(opf.OPF_EINVAL, opf._check, L.opf_set_launch(M.h, ctypes.byref(bad)))
    ok = opf.OpfLaunch(256, 64, 0, 0, 1, 1)
    opf._check(L.opf_set_launch(M.h, ctypes.byref(ok)))
    assert M.get_launch() == ok.as_dict()
    # the fused evaluation (bus_order 3), with one or two warps per packed warp
    for occ in (0, 2):
        fused = opf.OpfLaunch(128, 32, 0, 4, 3, occ)
        opf._check(L.opf_set_launch(M.h, ctypes.byref(fused)))
        assert M.get_launch() == fused.as_dict()


def test_warm_create_rejects_bad_options(L):
    """opf_warm_create validates its options on the host before any device
    work (batch and hidden multiples of 128, one period, positive rates)."""
    from paper_2510_12897_b300 import warm
    g = synth.case30()
    keep = []
    net = opf._net_struct(g, keep)
    wl = warm._lib()
    bad = [warm.WarmOpts(100, 128, 1e3, 1e-4, 1e-2, 1.0, 0), warm.WarmOpts(128, 96, 1e3, 1e-4, 1e-2, 1.0, 0),
           warm.WarmOpts(128, 128, -1.0, 1e-4, 1e-2, 1.0, 0), warm.WarmOpts(128, 128, 1e3, 0.0, 1e-2, 1.0, 0),
           warm.WarmOpts(128, 128, 1e3, 1e-4, -1.0, 1.0, 0),
           warm.WarmOpts(128, 128, 1e3, 1e-4, 1e-2, float("nan"), 0)]
    for opts in bad:
        h = ctypes.c_void_p()
        _expect(opf.OPF_EINVAL, opf._check, wl.opf_warm_create(ctypes.byref(net), ctypes.byref(opts), ctypes.byref(h)))
        assert not h.value
    mp = synth.multi_period(g, 3, seed=1)
    net2 = opf._net_struct(mp, keep)
    h = ctypes.c_void_p()
    _expect(opf.OPF_EINVAL, opf._check, wl.opf_warm_create(ctypes.byref(net2), ctypes.byref(warm.WarmOpts(128, 128, 1e3, 1e-4, 1e-2, 1.0, 0)), ctypes.byref(h)))
    _expect(opf.OPF_EINVAL, opf._check, wl.opf_warm_create(None, None, ctypes.byref(h)))


def test_rect_structure_matches_oracle(oracle_mod):
    """Rectangular form (host-only model, no GPU): dims, both patterns and
    all bounds equal the oracle's bit for bit, for a single grid, a
    multi-period grid with ramps and reserve, and an N-1 batch with
    per-instance ratios."""
    from paper_2510_12897_b300 import opf, synth
    cases = [(synth.case30(general=True), {}),
             (synth.multi_period(synth.case30(), 3, seed=2, ramp_ratio=0.2), dict(reserve=0.1)),
             (synth.contingencies(synth.case30(), 3, seed=1), dict(link_ratios=[0, .1, .2, .3], reserve=0.1))]
    for g, opts in cases:
        M = opf.Model(g, structure_only=True, form="rect", **opts)
        O = oracle_mod.Oracle(g, form="rect", **opts)
        assert (M.n, M.m, M.nnzj, M.nnzh) == (O.n, O.m, O.nnzj, O.nnzh)
        for a, b in zip(M.jac_pattern() + M.hess_pattern(), O.jac_pattern() + O.hess_pattern()):
            np.testing.assert_array_equal(a, b)
        for a, b in zip(M.bounds(), O.bounds()):
            np.testing.assert_array_equal(a, b)


def test_rect_form_validation():
    from paper_2510_12897_b300 import opf, synth
    g = synth.case30()
    wide = g.copy(br_angmax=np.where(np.arange(g.nbranch) == 2, np.pi / 2, g.br_angmax))
    opf.Model(wide, structure_only=True)
    with pytest.raises(opf.OpfError, match="angle limits"):
        opf.Model(wide, structure_only=True, form="rect")
    with pytest.raises(ValueError):
        opf.Model(g, structure_only=True, form="cartesian")


def test_storage_structure_matches_oracle(oracle_mod):
    """Multi-period model with storage (host-only model): dims, patterns and
    bounds equal the oracle's bit for bit, with and without complementarity
    rows, alone and in a batch with reserve rows; invalid descriptions are
    rejected before any device work."""
    from paper_2510_12897_b300 import opf, synth
    g = synth.with_storage(synth.multi_period(synth.case30(general=True), 4, seed=3, ramp_ratio=0.2))
    batch = [synth.with_storage(synth.multi_period(synth.case30(), 2, seed=1)),
             synth.multi_period(synth.case30(seed=31), 2, seed=2)]
    for grids, opts in ((g, {}), (g, dict(compl=True)), (batch, dict(compl=True, reserve=0.1))):
        M = opf.Model(grids, structure_only=True, **opts)
        O = oracle_mod.Oracle(grids, **opts)
        assert (M.n, M.m, M.nnzj, M.nnzh) == (O.n, O.m, O.nnzj, O.nnzh)
        for a, b in zip(M.jac_pattern() + M.hess_pattern(), O.jac_pattern() + O.hess_pattern()):
            np.testing.assert_array_equal(a, b)
        for a, b in zip(M.bounds(), O.bounds()):
            np.testing.assert_array_equal(a, b)
    for change, msg in ((dict(bus=np.array([0, g.nbus], np.int32)), "bus"),
                        (dict(eta_d=np.zeros(g.storage.nstor)), "efficienc"), (dict(dt=-1.0), "dt")):
        bad = g.copy(storage=synth.replace(g.storage, **change))
        with pytest.raises(opf.OpfError, match=msg):
            opf.Model(bad, structure_only=True)
    with pytest.raises(opf.OpfError, match="polar"):
        opf.Model(g, structure_only=True, form="rect")


def test_hub_bus_structure_matches_oracle(oracle_mod):
    """A bus with 45 arc slots (more than the 32 the per-bus bitmask covers):
    patterns equal the oracle's bit for bit in every form."""
    from paper_2510_12897_b300 import opf, synth
    from tests.test_hub_gpu import hub_grid
    g = hub_grid()
    for opts, gg in (({}, g), (dict(form="rect"), g),
                     (dict(compl=True), synth.with_storage(synth.multi_period(g, 3, seed=5, ramp_ratio=0.2)))):
        M = opf.Model(gg, structure_only=True, **opts)
        O = oracle_mod.Oracle(gg, **opts)
        assert (M.n, M.m, M.nnzj, M.nnzh) == (O.n, O.m, O.nnzj, O.nnzh)
        for a, b in zip(M.jac_pattern() + M.hess_pattern(), O.jac_pattern() + O.hess_pattern()):
            np.testing.assert_array_equal(a, b)
