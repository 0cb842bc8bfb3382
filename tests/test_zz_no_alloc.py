"""The allocation-free evaluation entry point (opf_eval_all_noalloc).

It exists for callers that cannot allocate device memory while they run (a
solver embedded in a process whose device memory belongs to another runtime,
or a loop that must keep cudaMalloc/cudaFree out of its iterations). These
tests call it through the C ABI and compare its outputs with those of
opf_eval_all and with the FP64 oracle's on the same model, point and
multipliers, on two calls in a row; this file is collected last so that a failure here stops a ``-x`` run
only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2510_12897_b300 import opf, synth

pytestmark = pytest.mark.gpu
RTOL = 1e-12


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2510_12897_b300 import build
    build.build()
    return t


def _close(name, got, ref, scale):
    bound = RTOL * np.maximum(np.abs(ref), scale)
    bad = np.abs(got - ref) > bound
    assert not bad.any(), f"{name}: {int(bad.sum())} entries differ beyond the tolerance"


@pytest.mark.parametrize("which", ["case30_general", "case10k", "mp30x6", "rect30", "storage30x4",
                                   "case10k_fused", "rect30_fused"])
def test_noalloc_matches_eval_all_twice(torch, oracle_mod, which):
    g = {"case30_general": lambda: synth.case30(general=True),
         "case10k": lambda: synth.case10k(),
         "mp30x6": lambda: synth.multi_period(synth.case30(general=True), 6, seed=4, ramp_ratio=0.2),
         "rect30": lambda: synth.case30(general=True),
         "storage30x4": lambda: synth.with_storage(synth.multi_period(synth.case30(general=True), 4, seed=4,
                                                                      ramp_ratio=0.2)),
         "case10k_fused": lambda: synth.case10k(),
         "rect30_fused": lambda: synth.case30(general=True),
         }[which]()
    opts = dict(form="rect") if which.startswith("rect30") else dict(compl=True) if which == "storage30x4" else {}
    M = opf.Model(g, **opts)
    if which.endswith("_fused"):  # the one-kernel evaluation needs no arc scratch
        M.set_launch(branch_block=128, bus_block=32, branch_ctas_per_sm=0, bus_ctas_per_sm=0, bus_order=3)
    O = oracle_mod.Oracle(g, **opts)
    rng = np.random.default_rng(21)
    x = synth.random_point(g, rng, form=opts.get("form", "polar"))
    lam = rng.standard_normal(M.m)
    dev = torch.device("cuda")
    dx = torch.tensor(x, device=dev)
    dl = torch.tensor(lam, device=dev)

    def bufs():
        return [torch.full((k,), np.nan, dtype=torch.float64, device=dev)
                for k in (1, M.n, M.m, M.nnzj, M.nnzh)]

    ref = bufs()
    M.eval_all(dx, dl, 0.8, *ref)
    torch.cuda.synchronize()
    ref = [t.cpu().numpy() for t in ref]
    # the oracle's values and per-entry magnitude scales, as in the parity tests
    f, fs = O.obj(x, with_scale=True)
    gr = O.grad(x)
    ora = [(np.array([f]), np.array([fs])), (gr, np.abs(gr)), O.cons(x, with_scale=True),
           O.jac(x, with_scale=True), O.hess(x, lam, 0.8, with_scale=True)]
    scales = [s for _, s in ora]
    names = ["obj", "grad", "cons", "jac", "hess"]
    for call in range(2):  # two calls in a row share the static scratch
        out = bufs()
        free_before = torch.cuda.mem_get_info()[0] if call == 1 else None
        opf._check(opf.lib().opf_eval_all_noalloc(
            M.h, ctypes.c_void_p(dx.data_ptr()), ctypes.c_void_p(dl.data_ptr()), ctypes.c_double(0.8),
            *(ctypes.c_void_p(t.data_ptr()) for t in out), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
        torch.cuda.synchronize()
        if free_before is not None:
            assert torch.cuda.mem_get_info()[0] == free_before
        for name, got, r, s, (o, _) in zip(names, out, ref, scales, ora):
            got = got.cpu().numpy()
            _close(f"call {call} {name} vs opf_eval_all", got, r, s)
            _close(f"call {call} {name} vs the oracle", got, o, s)


def test_noalloc_rejects_models_beyond_the_static_scratch(torch):
    g = synth.multi_period(synth.case1k(), 70, seed=3, ramp_ratio=0.2)  # 182,000 arc slots
    M = opf.Model(g)
    M.set_launch(branch_block=128, bus_block=128, branch_ctas_per_sm=0, bus_ctas_per_sm=0, bus_order=2)
    dev = torch.device("cuda")
    x = torch.zeros(M.n, dtype=torch.float64, device=dev)
    c = torch.zeros(M.m, dtype=torch.float64, device=dev)
    with pytest.raises(opf.OpfError) as e:
        M.eval_all_noalloc(x, c=c)
    assert e.value.code == opf.OPF_EINVAL
    assert "arc scratch slots" in str(e.value)
    # the fused one-kernel evaluation writes no arc slots: the same model is
    # accepted under it, with the rows of opf_eval_all
    M.set_launch(branch_block=128, bus_block=32, branch_ctas_per_sm=0, bus_ctas_per_sm=0, bus_order=3)
    xr = torch.tensor(synth.random_point(g, np.random.default_rng(5)), device=dev)
    M.eval_all_noalloc(xr, c=c)
    c2 = torch.zeros_like(c)
    M.eval_all(xr, None, 1.0, None, None, c2)
    torch.cuda.synchronize()
    assert torch.equal(c, c2)


def test_noalloc_rejects_a_model_of_another_device(torch):
    """With another device current the call returns OPF_EINVAL before any
    launch (needs a second visible device)."""
    g = synth.case30(general=True)
    M = opf.Model(g)
    dev = torch.device("cuda")
    x = torch.tensor(synth.random_point(g, np.random.default_rng(6)), device=dev)
    c = torch.zeros(M.m, dtype=torch.float64, device=dev)
    if torch.cuda.device_count() < 2:
        pytest.skip("one visible device: the device mismatch needs a second one")
    with torch.cuda.device(1):
        with pytest.raises(opf.OpfError) as e:
            M.eval_all_noalloc(x, c=c)
    assert e.value.code == opf.OPF_EINVAL and "device" in str(e.value)
