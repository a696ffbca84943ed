"""The allocation-free Euler step against the regular one.

mxe_diffuse_step_noalloc serves callers that cannot call cudaMalloc (a host
framework whose allocator already holds the card, a fixed memory budget, or a
latency-critical loop that must not synchronise the device through an
allocation).  It keeps its scratch in one fixed device array shared by every
call, so this test calls it twice in a row through the C ABI -- the second
call runs on whatever the first left in that array -- and checks each result
against mxe_diffuse_step from the same inputs.  This file is collected last
on purpose, and it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1910_01235_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_01235_gb300 import mxe as M  # noqa: E402

# the same tolerance as the FP64 Euler-step parity tests
TOL = 1e-12


def _cases():
    single = W.random_fractions(W.perturb(W.config_vacancy_lattice(), 0.05, 0.02), vac_min=0.02, seed=21)
    binary = W.perturb(W.config_binary_alloy(cells=6), 0.05, 0.02, seed=22)
    return {"single": single, "binary": binary}


@pytest.mark.parametrize("case", ["single", "binary"])
def test_noalloc_step_matches_regular_step_twice(case):
    s = _cases()[case]
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    g.free_energy_grad()
    boff, bidx = g.export_bonds()
    mu = g.mu_ex.clone()
    x0 = g.x.clone()
    # a small, stable step: the largest rate times dt stays well below 1
    dt = s.dt_default() * 1e-3
    stream = g.stream
    # reference: two regular steps from x0 with fixed mu
    ref = []
    for _ in range(2):
        g.diffuse_step(dt, mu_ex=mu)
        ref.append(g.x.clone())
    # allocation-free: two calls in a row on a separate copy of x0
    x = x0.clone()
    T = g.T.contiguous()
    for k in range(2):
        st = M.mxe_diffuse_step_noalloc(s.n, s.S, M._ptr(x), M._ptr(T), M._ptr(mu), M._ptr(boff), M._ptr(bidx),
                                        dt, s.nu0, s.Qm, stream.cuda_stream)
        assert st == M.OK, M.mxe_status_string(st)
        diff = (x - ref[k]).abs().max().item()
        assert diff <= TOL, (k, diff)
    assert (ref[1] - x0).abs().max().item() > 1e-8   # the steps moved mass
    g.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    for S in (1, 2):
        n = M.noalloc_max_sites(S) + 1
        st = M.mxe_diffuse_step_noalloc(n, S, 0, 0, 0, 0, 0, 1e-12, 1e13, 0.69, 0)
        assert st == M.ERR_ARG
    st = M.mxe_diffuse_step_noalloc(10, 3, 0, 0, 0, 0, 0, 1e-12, 1e13, 0.69, 0)
    assert st == M.ERR_ARG


def test_noalloc_x_range_keeps_x():
    s = _cases()["single"]
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    g.free_energy_grad()
    boff, bidx = g.export_bonds()
    x = g.x.clone()
    x0 = x.clone()
    st = M.mxe_diffuse_step_noalloc(s.n, s.S, M._ptr(x), M._ptr(g.T), M._ptr(g.mu_ex), M._ptr(boff), M._ptr(bidx),
                                    s.dt_default() * 1e6, s.nu0, s.Qm, g.stream.cuda_stream)
    assert st == M.ERR_X_RANGE
    assert torch.equal(x, x0)
    g.close()
