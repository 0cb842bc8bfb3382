"""A hub bus with more than 32 arc slots (45: 40 neighbours, five of them
over two parallel branches) in the middle of the id range: the bus phase
reads its slot codes from memory instead of the per-bus bitmask, and its
Hessian rows hold groups on both sides of the diagonal. Every output of the
polar form, the rectangular form and the storage model against the oracle."""
import numpy as np
import pytest

from paper_2510_12897_b300 import synth
from tests.test_oracle_pins import tiny
from tests.test_parity_gpu import both, check_against_oracle, points, run_all, torch  # noqa: F401
from tests.test_rect_gpu import jtprod_check, rpoints

pytestmark = pytest.mark.gpu

HUB = 20


def hub_grid():
    rng = np.random.default_rng(42)
    nb = 41
    br = []
    for j in range(nb):
        if j == HUB:
            continue
        br.append((HUB, j) if j % 3 else (j, HUB))  # both orientations
    for j in (1, 7, 25, 33, 40):  # parallel branches
        br.append((j, HUB))
    for j in range(0, nb - 1, 4):  # a few leaf-to-leaf branches
        if j != HUB and j + 1 != HUB:
            br.append((j, j + 1))
    rows = [(f, t, rng.uniform(0.01, 0.1), rng.uniform(0.05, 0.3), rng.uniform(0, 0.05),
             rng.choice([1.0, 1.03]), rng.choice([0.0, 0.05]), rng.uniform(0.5, 2)) for f, t in br]
    gens = [(HUB, 0.05, 20.0, 1.0), (3, 0.02, 30.0, 0.0), (HUB, 0.03, 25.0, 0.5)]
    loads = [(j, rng.uniform(0, 0.5), rng.uniform(0, 0.15)) for j in range(nb) if j % 2]
    return tiny(nb, rows, gens, loads, gs=rng.uniform(0, 0.02, nb), bs=rng.uniform(-0.02, 0.02, nb))


def test_hub_polar(torch, oracle_mod):
    g = hub_grid()
    deg = np.bincount(np.concatenate([g.br_f, g.br_t]), minlength=g.nbus)
    assert deg[HUB] > 32
    M, O = both(torch, oracle_mod, g)
    for k, (x, lam) in enumerate(points(g, M.m, 4, seed=3)):
        launch = [None, dict(bus_block=32, bus_order=1), dict(bus_ctas_per_sm=1, branch_ctas_per_sm=1), None][k]
        check_against_oracle(O, run_all(torch, M, x, lam, 1.0, launch), x, lam, 1.0, f"pt{k} ")
        jtprod_check(torch, M, O, x, lam)


def test_hub_rect(torch, oracle_mod):
    g = hub_grid()
    M, O = both(torch, oracle_mod, g, form="rect")
    for x, lam in rpoints(g, M.m, 3, seed=4):
        check_against_oracle(O, run_all(torch, M, x, lam, 0.7), x, lam, 0.7)
        jtprod_check(torch, M, O, x, lam)


def test_hub_storage_multiperiod(torch, oracle_mod):
    g = synth.with_storage(synth.multi_period(hub_grid(), 3, seed=5, ramp_ratio=0.2))
    M, O = both(torch, oracle_mod, g, compl=True)
    for x, lam in points(g, M.m, 3, seed=5):
        check_against_oracle(O, run_all(torch, M, x, lam, 1.0), x, lam, 1.0)
        jtprod_check(torch, M, O, x, lam)
