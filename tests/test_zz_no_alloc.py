"""ov_apply_H_noalloc: the allocation-free H(mu) psi, for callers that must not
allocate device memory when they apply the operator (a framework allocator
that owns the device memory, an inner loop that cannot pay for the device
synchronisation of cudaMalloc/cudaFree, a plug-in whose host forbids
allocations).  Called through the C ABI and compared with ov_apply_H, twice
in a row (the fixed scratch array keeps the previous call's contents).

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1604_08057_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
SCRATCH_LIMIT = -7


def _noalloc(lib):
    f = lib.ov_apply_H_noalloc
    f.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _call(f, u, mu, m_w, psi, dagger):
    nt, nz, ny, nx = u.shape[:4]
    dims = (ctypes.c_int32 * 4)(nx, ny, nz, nt)
    out = torch.empty_like(psi)
    stream = torch.cuda.current_stream().cuda_stream
    st = f(dims, ctypes.c_void_p(u.data_ptr()), mu, m_w, psi.shape[0], ctypes.c_void_p(psi.data_ptr()),
           ctypes.c_void_p(out.data_ptr()), dagger, ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return st, out


def test_noalloc_matches_apply_h_on_consecutive_calls():
    lib = binding.load()
    f = _noalloc(lib)
    dims, mu, m_w = (6, 5, 4, 7), 0.3, -2.0
    rng = np.random.default_rng(77)
    u = torch.tensor(inputs.su3_links(dims, 0.3, rng), device="cuda")
    for call, (nsrc, dagger) in enumerate([(3, 0), (2, 1)]):
        psi = torch.tensor(inputs.gaussian_spinors(dims, nsrc, rng), device="cuda")
        st, got = _call(f, u, mu, m_w, psi, dagger)
        assert st == 0, (call, lib.ov_strerror(st))
        want = binding.apply_H(u, mu, m_w, psi, dagger=bool(dagger), precision="fp64")
        rel = float(torch.linalg.vector_norm(got - want) / torch.linalg.vector_norm(want))
        assert rel <= 1e-13, (call, rel)


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = binding.load()
    f = _noalloc(lib)
    dims = (16, 16, 16, 16)     # 65536 sites: (72 + 48) * 8 B per site > 32 MiB
    u = torch.zeros(dims[::-1] + (4, 3, 3), dtype=torch.complex128, device="cuda")
    psi = torch.zeros((1,) + dims[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
    st, _ = _call(f, u, 0.1, -1.0, psi, 0)
    assert st == SCRATCH_LIMIT
    assert b"scratch" in lib.ov_strerror(st)
    # more sources than any call accepts: rejected before the scratch bound is computed
    # (the arrays are never read: the check comes first)
    small = torch.zeros((2, 2, 2, 2, 4, 3, 3), dtype=torch.complex128, device="cuda")
    one = torch.zeros((1, 2, 2, 2, 2, 4, 3), dtype=torch.complex128, device="cuda")
    dims4 = (ctypes.c_int32 * 4)(2, 2, 2, 2)
    st = f(dims4, ctypes.c_void_p(small.data_ptr()), 0.1, -1.0, 4097, ctypes.c_void_p(one.data_ptr()),
           ctypes.c_void_p(one.data_ptr()), 0, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -1
