"""The Krylov sweeps captured as CUDA graphs (options.graphs, on by default) give
the results of direct launches bit for bit: the first call with a shape runs
directly, the second is captured, the third and later replay (also on new
source data), and a change of mu starts over; for FP64 and FP32 fields and
several sources."""
import numpy as np
import pytest
import torch

from paper_1604_08057_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _run(u, b, xbar, mu, k, prec, reb, passes):
    du, dmu, x = binding.tsl_sign_vjp(u, mu, -2.0, b, k, xbar, precision=prec, rebiorth=reb, passes=passes)
    xs = binding.tsl_sign(u, mu, -2.0, b, k, precision=prec, rebiorth=reb, passes=passes)
    return du, dmu, x, xs


@pytest.mark.parametrize("dims,nsrc,k,prec,reb,passes", [((4, 4, 4, 4), 1, 200, "fp64", 20, 1),
                                                          ((3, 5, 2, 4), 2, 60, "mixed", 1, 2)])
def test_graph_replay_equals_direct_launches(dims, nsrc, k, prec, reb, passes):
    rng = np.random.default_rng(91)
    u = torch.tensor(inputs.su3_links(dims, 0.3, rng), device="cuda")
    b1, b2, xbar = (torch.tensor(inputs.gaussian_spinors(dims, nsrc, rng), device="cuda") for _ in range(3))
    out = {}
    for graphs in (False, True):
        binding.sweep_graphs(graphs, prec, reb, passes)
        try:
            ctx = binding.context(prec, reb, passes)
            l0 = binding.launch_count(ctx)
            first = _run(u, b1, xbar, 0.3, k, prec, reb, passes)
            l1 = binding.launch_count(ctx)
            second = _run(u, b1, xbar, 0.3, k, prec, reb, passes)
            third = _run(u, b1, xbar, 0.3, k, prec, reb, passes)
            l3 = binding.launch_count(ctx)
            other_b = _run(u, b2, xbar, 0.3, k, prec, reb, passes)
            other_mu = _run(u, b1, xbar, 0.25, k, prec, reb, passes)
            other_mu2 = _run(u, b1, xbar, 0.25, k, prec, reb, passes)
            other_mu3 = _run(u, b1, xbar, 0.25, k, prec, reb, passes)
        finally:
            binding.sweep_graphs(True, prec, reb, passes)
        out[graphs] = (first, second, third, other_b, other_mu, other_mu2, other_mu3)
        # captures and replays launch (and count) the same kernels as direct launches
        assert l3 - l1 == 2 * (l1 - l0)
    for a, b in zip(out[False], out[True]):
        du0, dmu0, x0, xs0 = a
        du1, dmu1, x1, xs1 = b
        assert torch.equal(du0, du1) and dmu0 == dmu1 and torch.equal(x0, x1) and torch.equal(xs0, xs1)
