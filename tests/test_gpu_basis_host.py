"""Krylov bases in pinned host memory (options.basis_memory = 1): the kernels
read and write them through their device alias over the CPU-GPU link.  The
same kernels run on the same data, so every result equals the device-memory
run bit for bit, with re-biorthogonalisation (which reads the whole basis at
every projection step) and in the reverse sweep."""
import numpy as np
import pytest
import torch

from paper_1604_08057_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,nsrc,k,reb", [((4, 4, 4, 4), 1, 200, 20), ((6, 5, 4, 7), 2, 90, 1)])
def test_host_basis_equals_device_basis(dims, nsrc, k, reb):
    rng = np.random.default_rng(81)
    u = torch.tensor(inputs.su3_links(dims, 0.3, rng), device="cuda")
    b = torch.tensor(inputs.gaussian_spinors(dims, nsrc, rng), device="cuda")
    xbar = torch.tensor(inputs.gaussian_spinors(dims, nsrc, rng), device="cuda")
    out = {}
    for where in ("device", "host"):
        binding.basis_memory(where, rebiorth=reb, passes=1)
        try:
            du, dmu, x = binding.tsl_sign_vjp(u, 0.3, -2.0, b, k, xbar, rebiorth=reb, passes=1)
            xs = binding.tsl_sign(u, 0.3, -2.0, b, k, rebiorth=reb, passes=1)
        finally:
            binding.basis_memory("device", rebiorth=reb, passes=1)
        out[where] = (du, dmu, x, xs)
    (du0, dmu0, x0, xs0), (du1, dmu1, x1, xs1) = out["device"], out["host"]
    assert torch.equal(du0, du1) and dmu0 == dmu1 and torch.equal(x0, x1) and torch.equal(xs0, xs1)
