"""Parity of the multi-period model with storage (Sec. III-C-2) on the GPU
with the FP64 oracle, through the C ABI: patterns bit for bit, every value
to 1e-12 of the oracle's entry scale, J^T v, the flat start."""
import numpy as np
import pytest

from paper_2510_12897_b300 import opf, synth
from tests.test_parity_gpu import both, check_against_oracle, dev, host, points, run_all, torch  # noqa: F401
from tests.test_rect_gpu import jtprod_check

pytestmark = pytest.mark.gpu


def stor(T=4, seed=3, general=True):
    return synth.with_storage(synth.multi_period(synth.case30(general=general), T, seed=seed, ramp_ratio=0.2))


@pytest.mark.parametrize("compl", [False, True])
def test_storage_case30(torch, oracle_mod, compl):
    g = stor()
    M, O = both(torch, oracle_mod, g, compl=compl)
    for k, (x, lam) in enumerate(points(g, M.m, 5, seed=21)):
        launch = [None, dict(bus_block=32), dict(bus_ctas_per_sm=1), dict(bus_order=1), None][k]
        sigma = 0.0 if k == 4 else 0.9
        check_against_oracle(O, run_all(torch, M, x, lam, sigma, launch), x, lam, sigma, f"pt{k} ")
        jtprod_check(torch, M, O, x, lam)


def test_storage_batch_with_reserve(torch, oracle_mod):
    """Instances with and without storage in one batch, reserve rows."""
    insts = [stor(T=3, seed=1), synth.multi_period(synth.case30(seed=31, general=True), 3, seed=2, ramp_ratio=0.2),
             stor(T=2, seed=5, general=False)]
    M, O = both(torch, oracle_mod, insts, reserve=0.1, compl=True)
    for x, lam in points(insts, M.m, 3, seed=22):
        check_against_oracle(O, run_all(torch, M, x, lam, 1.0), x, lam, 1.0)
        jtprod_check(torch, M, O, x, lam)


def test_storage_flat_start(torch, oracle_mod):
    """Units idle (ps = qs = sc = sd = 0) at their initial energy: every
    state-of-charge and loss row of the oracle sits at its bound."""
    g = stor(T=5)
    M, O = both(torch, oracle_mod, g)
    x = torch.full((M.n,), np.nan, dtype=torch.float64, device="cuda")
    M.flat_start(x)
    x = host(x)
    assert not np.isnan(x).any()
    ns, T = g.storage.nstor, 5
    base = synth.n_vars(g) - 5 * ns * T
    assert np.all(x[base:base + 4 * ns * T] == 0)
    np.testing.assert_array_equal(x[base + 4 * ns * T:], np.tile(g.storage.e_init, T))
    c = O.cons(x)
    gl = O.bounds()[2]
    rows = slice(O.m - 3 * ns * T, O.m - ns * T)
    np.testing.assert_allclose(c[rows], gl[rows], atol=1e-15)


def test_storage_mp2k_24(torch, oracle_mod):
    """The 2,000-bus grid over 24 periods with storage and complementarity
    rows, every entry, default and autotuned launch shapes."""
    g = synth.with_storage(synth.multi_period(synth.case2k(), 24, seed=2000, ramp_ratio=0.2))
    M, O = both(torch, oracle_mod, g, compl=True)
    x, lam = next(points(g, M.m, 1, seed=23))
    check_against_oracle(O, run_all(torch, M, x, lam, 1.0), x, lam, 1.0, "default ")
    best, _ = M.autotune(dev(torch, x), dev(torch, lam), reps=3)
    check_against_oracle(O, run_all(torch, M, x, lam, 1.0, best), x, lam, 1.0, "tuned ")
    jtprod_check(torch, M, O, x, lam)


def test_storage_rejections(torch):
    g = stor(T=2)
    with pytest.raises(opf.OpfError, match="polar"):
        opf.Model(g, form="rect")
    bad = g.copy(storage=synth.replace(g.storage, dt=0.0))
    with pytest.raises(opf.OpfError, match="dt"):
        opf.Model(bad)


def test_storage_single_period(torch, oracle_mod):
    """One period: every state-of-charge row has its first-period form
    (no previous energy)."""
    g = synth.with_storage(synth.case30(general=True))
    M, O = both(torch, oracle_mod, g, compl=True)
    for x, lam in points(g, M.m, 3, seed=24):
        check_against_oracle(O, run_all(torch, M, x, lam, 1.0), x, lam, 1.0)
        jtprod_check(torch, M, O, x, lam)
