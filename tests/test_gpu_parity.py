"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances.  FP64 stencil: 1e-13 relative (a few roundings of a 9-term sum).
FP32 stencil: 2e-6 relative.  The k-step TSL map itself amplifies rounding: at
the 4x4^3 workload point (m_w = -2, mu = 0.3, k = 200) a relative perturbation
of b by 1e-16 moves x by 1e-10 and dU by 9e-8 (full re-biorthogonalisation),
so FP64 parity there is required to 10x those floors.  On the well-conditioned
m_w = -1 points the floors are ~1e-14, and 1e-11 is required.
"""
import ctypes
import functools

import numpy as np
import pytest
import torch

from oracle import dirac, tsl, vjp
from paper_1604_08057_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@functools.lru_cache(maxsize=None)
def case(dims, eps, seed, nsrc=1):
    rng = np.random.default_rng(seed)
    u = inputs.su3_links(dims, eps, rng)
    b = inputs.gaussian_spinors(dims, nsrc, rng)
    xbar = inputs.gaussian_spinors(dims, nsrc, rng)
    return u, b, xbar


@functools.lru_cache(maxsize=None)
def oracle_fwd(dims, eps, seed, mu, m_w, k, rebiorth=1, passes=2, src=0):
    u, b, _ = case(dims, eps, seed, max(src + 1, 1))
    return tsl.tsl_forward(u, b[src], mu, m_w, k, rebiorth=rebiorth, passes=passes)


@functools.lru_cache(maxsize=None)
def oracle_vjp(dims, eps, seed, mu, m_w, k, rebiorth=1, passes=2):
    u, b, xbar = case(dims, eps, seed)
    du, dmu, fwd = vjp.tsl_vjp(u, b[0], mu, m_w, k, xbar[0], rebiorth=rebiorth, passes=passes,
                               fwd=oracle_fwd(dims, eps, seed, mu, m_w, k, rebiorth, passes))
    return du, dmu


def T(a):
    return torch.tensor(a, device=DEV)


# ---------------------------------------------------------------------------
# H and H^dagger
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (3, 5, 2, 4), (4, 4, 4, 4), (8, 8, 8, 8), (14, 14, 14, 14)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 2e-6)])
def test_apply_h_parity(dims, precision, tol):
    u, b, _ = case(dims, 0.3, 1, 2)
    mu, m_w = 0.3, -2.0
    ut, bt = T(u), T(b)
    for dagger in (False, True):
        got = binding.apply_H(ut, mu, m_w, bt, dagger=dagger, precision=precision).cpu().numpy()
        for s in range(2):
            want = (dirac.apply_h_dagger if dagger else dirac.apply_h)(u, b[s], mu, m_w)
            assert rel(got[s], want) <= tol, (dims, precision, dagger, s, rel(got[s], want))


def test_apply_h_single_source_shape():
    u, b, _ = case((3, 3, 3, 3), 0.3, 2)
    got = binding.apply_H(T(u), 0.1, -1.0, T(b[0])).cpu().numpy()
    assert got.shape == b[0].shape
    assert rel(got, dirac.apply_h(u, b[0], 0.1, -1.0)) <= 1e-13


@pytest.mark.parametrize("dims", [(3, 5, 2, 4), (12, 6, 2, 3)])   # the second has 72-site x-y planes
@pytest.mark.parametrize("precision,tol_h,tol_x", [("fp64", 1e-13, 1e-11), ("mixed", 2e-6, None)])
def test_every_stencil_variant(dims, precision, tol_h, tol_x):
    """Each compiled launch variant of both stencil kernels gives the oracle's result."""
    mu, m_w, k = 0.3, -1.0, 20
    u, b, _ = case(dims, 0.3, 8, 5)
    ut, bt = T(u), T(b)
    rep = binding.autotune(ut, mu, m_w, nsrc=5, precision=precision)
    assert len(rep["apply_us"]) >= 9 and len(rep["pair_us"]) >= 7
    refs = [tsl.tsl_forward(u, b[s], mu, m_w, k) for s in range(2)]
    for v in range(len(rep["apply_us"])):
        binding.set_stencil_variants(v, 0, precision)
        got = binding.apply_H(ut, mu, m_w, bt, precision=precision).cpu().numpy()
        for s in range(5):
            assert rel(got[s], dirac.apply_h(u, b[s], mu, m_w)) <= tol_h, (v, s)
    for v in range(len(rep["pair_us"])):
        binding.set_stencil_variants(0, v, precision)
        x = binding.tsl_sign(ut, mu, m_w, bt[:2], k, precision=precision).cpu().numpy()
        for s in range(2):
            err = rel(x[s], refs[s].x)
            assert err <= (tol_x if tol_x else 1e-4), (v, s, err)
    binding.set_stencil_variants(rep["apply_variant"], rep["pair_variant"], precision)


@pytest.mark.parametrize("nsrc", [32, 33, 1])
def test_sources_interleaved_variant_equals_variant_0(nsrc):
    """The FP32 variant with the sources interleaved innermost (13) runs the same
    per-site arithmetic as variant 0 on its own field layout: bitwise equal results,
    for a full warp of sources per site, a source count that makes warps straddle
    sites, and a lone source."""
    dims, mu, m_w = (4, 4, 6, 8), 0.3, -2.0
    u, b, _ = case(dims, 0.3, 23, nsrc)
    ut, bt = T(u), T(b)
    out = {}
    try:
        for v in (0, 13):
            binding.set_stencil_variants(v, 0, "mixed")
            out[v] = [binding.apply_H(ut, mu, m_w, bt, dagger=d, precision="mixed") for d in (False, True)]
    finally:
        binding.set_stencil_variants(0, 0, "mixed")
    for d in range(2):
        assert torch.equal(out[13][d], out[0][d]), d
    want = dirac.apply_h(u, b[0], mu, m_w)
    assert rel(out[13][0].cpu().numpy()[0], want) <= 2e-6


@pytest.mark.parametrize("variant", [9, 10, 11, 12, 13])
def test_shared_memory_stencil_variants_long_runs(variant):
    """The FP32 variants that stage the input in shared memory, on a lattice whose
    per-block runs of z-planes are long enough that the sweep variant (12) refills
    its ring of four plane slots (runs of 4-5 planes: 6-7 staged planes), with
    periodic wrap in z and t, against the oracle's operator."""
    dims, mu, m_w = (3, 4, 9, 40), 0.3, -2.0
    u, b, _ = case(dims, 0.3, 17, 6)
    ut, bt = T(u), T(b)
    binding.set_stencil_variants(variant, 0, "mixed")
    try:
        for dagger in (False, True):
            got = binding.apply_H(ut, mu, m_w, bt, dagger=dagger, precision="mixed").cpu().numpy()
            for s in range(6):
                want = (dirac.apply_h_dagger if dagger else dirac.apply_h)(u, b[s], mu, m_w)
                assert rel(got[s], want) <= 2e-6, (variant, dagger, s, rel(got[s], want))
    finally:
        binding.set_stencil_variants(0, 0, "mixed")


# ---------------------------------------------------------------------------
# forward TSL
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,mu,m_w,k,reb,passes,tol", [
    ((3, 3, 3, 3), 0.3, -1.0, 60, 1, 2, 1e-11),
    ((3, 5, 2, 4), 0.4, -1.0, 45, 10, 2, 1e-11),     # ragged lattice, pair-periodic
    ((4, 4, 4, 4), 0.3, -2.0, 200, 1, 2, 1e-9),      # the 4x4^3 workload: floor 1e-10
    ((4, 4, 4, 4), 0.3, -2.0, 200, 20, 1, 1e-9),     # P = 20, one pass
    ((4, 4, 4, 4), 0.3, -2.0, 200, 20, 2, 1e-9),     # benchmark schedule: P = 20, two passes
])
def test_tsl_forward_fp64(dims, mu, m_w, k, reb, passes, tol):
    u, b, _ = case(dims, 0.3, 3)
    ref = oracle_fwd(dims, 0.3, 3, mu, m_w, k, reb, passes)
    x = binding.tsl_sign(T(u), mu, m_w, T(b[0]), k, rebiorth=reb, passes=passes).cpu().numpy()
    a, bt, d = binding.tsl_coefficients(k, rebiorth=reb, passes=passes)
    # the first coefficients agree to rounding before the map's amplification sets in
    assert np.abs(a[:10] - ref.alpha[:10]).max() <= 1e-12 * np.abs(ref.alpha[:10]).max()
    assert np.abs(d[1:10] - ref.delta[1:10]).max() <= 1e-12 * np.abs(ref.delta[1:10]).max()
    assert np.abs(bt[1:10] - ref.beta[1:10]).max() <= 1e-12 * np.abs(ref.beta[1:10]).max()
    assert rel(x, ref.x) <= tol, rel(x, ref.x)


def test_tsl_forward_batched_sources_and_k2():
    dims, mu, m_w = (3, 3, 2, 3), 0.2, -1.0
    u, b, _ = case(dims, 0.3, 4, 3)
    for k in (2, 30):
        x = binding.tsl_sign(T(u), mu, m_w, T(b), k).cpu().numpy()
        for s in range(3):
            ref = tsl.tsl_forward(u, b[s], mu, m_w, k)
            assert rel(x[s], ref.x) <= 1e-11, (k, s, rel(x[s], ref.x))


def test_growing_source_count_on_one_context():
    """A call with more sources than the context has seen reuses workspace buffers
    whose capacity already covers it: their unused part must start at zero (ticket
    counters).  Device memory is dirtied first so that stale bytes would show."""
    junk = torch.full((64 << 20,), -1, dtype=torch.int32, device=DEV)
    del junk
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    dims, mu, m_w = (3, 5, 2, 4), 0.3, -1.0
    u, b, _ = case(dims, 0.3, 12, 3)
    reb, passes = 7, 1                     # options no other test uses: a fresh context
    for nsrc, k in ((1, 24), (3, 24), (2, 30)):
        x = binding.tsl_sign(T(u), mu, m_w, T(b[:nsrc]), k, rebiorth=reb, passes=passes).cpu().numpy()
        for s in range(nsrc):
            ref = tsl.tsl_forward(u, b[s], mu, m_w, k, rebiorth=reb, passes=passes)
            assert rel(x[s], ref.x) <= 1e-11, (nsrc, s, rel(x[s], ref.x))


def test_tsl_forward_mixed_precision():
    """FP32 vectors: compared with the FP64 oracle to 2x the error of the oracle's own FP32 emulation."""
    dims, mu, m_w, k = (3, 3, 3, 3), 0.3, -1.0, 60
    u, b, _ = case(dims, 0.3, 3)
    ref = oracle_fwd(dims, 0.3, 3, mu, m_w, k)
    emu = tsl.tsl_forward(u, b[0], mu, m_w, k, emulate_fp32=True)
    bar = max(2.0 * rel(emu.x, ref.x), 1e-6)
    x = binding.tsl_sign(T(u), mu, m_w, T(b[0]), k, precision="mixed").cpu().numpy()
    assert rel(x, ref.x) <= bar, (rel(x, ref.x), bar)


# ---------------------------------------------------------------------------
# VJP
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,mu,m_w,k,reb,passes,tol", [
    ((3, 3, 3, 3), 0.3, -1.0, 40, 1, 2, 1e-9),
    ((3, 5, 2, 4), 0.3, -1.0, 50, 10, 2, 1e-8),
    ((4, 4, 4, 4), 0.3, -2.0, 200, 1, 2, 1e-6),      # the 4x4^3 workload: dU floor 9e-8
    ((4, 4, 4, 4), 0.3, -2.0, 200, 20, 1, 5e-6),     # P = 20, one pass: dU floor 7.4e-7
    ((4, 4, 4, 4), 0.3, -2.0, 200, 20, 2, 5e-6),     # benchmark schedule: dU floor 3.7e-7
])
def test_vjp_fp64(dims, mu, m_w, k, reb, passes, tol):
    u, b, xbar = case(dims, 0.3, 3)
    du_o, dmu_o = oracle_vjp(dims, 0.3, 3, mu, m_w, k, reb, passes)
    du, dmu, x = binding.tsl_sign_vjp(T(u), mu, m_w, T(b[0]), k, T(xbar[0]), rebiorth=reb, passes=passes)
    assert rel(du.cpu().numpy(), du_o) <= tol, rel(du.cpu().numpy(), du_o)
    assert abs(dmu - dmu_o) <= tol * max(1.0, abs(dmu_o)), (dmu, dmu_o)
    ref = oracle_fwd(dims, 0.3, 3, mu, m_w, k, reb, passes)
    assert rel(x.cpu().numpy(), ref.x) <= max(tol, 1e-11)


def test_vjp_mixed_precision_well_conditioned():
    dims, mu, m_w, k = (3, 3, 3, 3), 0.3, -1.0, 40
    u, b, xbar = case(dims, 0.3, 3)
    du_o, dmu_o = oracle_vjp(dims, 0.3, 3, mu, m_w, k)
    du, dmu, _ = binding.tsl_sign_vjp(T(u), mu, m_w, T(b[0]), k, T(xbar[0]), precision="mixed")
    assert rel(du.cpu().numpy(), du_o) <= 1e-4
    assert abs(dmu - dmu_o) <= 1e-4 * abs(dmu_o)


def test_vjp_batched_sources_sum():
    """With several sources the VJP is the sum of the per-source VJPs."""
    dims, mu, m_w, k = (2, 3, 2, 3), 0.25, -1.0, 25
    u, b, xbar = case(dims, 0.3, 5, 2)
    du, dmu, _ = binding.tsl_sign_vjp(T(u), mu, m_w, T(b), k, T(xbar))
    du_o = np.zeros_like(u)
    dmu_o = 0.0
    for s in range(2):
        d, m, _ = vjp.tsl_vjp(u, b[s], mu, m_w, k, xbar[s])
        du_o += d
        dmu_o += m
    assert rel(du.cpu().numpy(), du_o) <= 1e-9
    assert abs(dmu - dmu_o) <= 1e-9 * abs(dmu_o)


def test_autograd_function_matches_vjp():
    from paper_1604_08057_gb300.autograd import tsl_sign as tsl_fn
    dims, mu, m_w, k = (3, 3, 3, 3), 0.3, -1.0, 30
    u, b, xbar = case(dims, 0.3, 3)
    ut = T(u).requires_grad_(True)
    mut = torch.tensor(mu, dtype=torch.float64, device=DEV, requires_grad=True)
    x = tsl_fn(ut, mut, T(b[0]), k, m_w)
    loss = torch.real(torch.vdot(T(xbar[0]).flatten(), x.flatten()))
    loss.backward()
    du_o, dmu_o, _ = vjp.tsl_vjp(u, b[0], mu, m_w, k, xbar[0])
    assert rel(ut.grad.cpu().numpy(), du_o) <= 1e-9
    assert abs(mut.grad.item() - dmu_o) <= 1e-9 * abs(dmu_o)


# ---------------------------------------------------------------------------
# errors
# ---------------------------------------------------------------------------
def test_invalid_arguments_and_breakdown():
    u, b, _ = case((2, 2, 2, 2), 0.3, 6)
    with pytest.raises(binding.OVError) as e:
        binding.tsl_sign(T(u), 0.3, -1.0, T(b[0]), 1)
    assert e.value.status == -1
    # the chiral constant spinor on the free field at mu = 0 is an eigenvector of H: breakdown
    shape = inputs.lattice_shape((2, 2, 2, 2))
    uf = np.zeros(shape + (4, 3, 3), dtype=complex)
    uf[...] = np.eye(3)
    bf = np.zeros(shape + (4, 3), dtype=complex)
    bf[..., 0, 0] = 1.0
    with pytest.raises(binding.OVError) as e:
        binding.tsl_sign(T(uf), 0.0, -1.0, T(bf), 5, rebiorth=0)
    assert e.value.status == -3


# ---------------------------------------------------------------------------
# Theorem 1: TSL on the block matrix [[H, dH], [0, H]]
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,m_w,k,reb,with_e,m_dir,tol", [
    ((3, 3, 3, 3), -1.0, 60, 1, True, 0.7, 1e-10),
    ((3, 5, 2, 4), -1.0, 50, 10, True, 0.0, 1e-10),
    ((3, 3, 2, 3), -1.0, 40, 1, False, 1.0, 1e-10),     # mu direction only
    ((4, 4, 4, 4), -2.0, 120, 1, True, 0.3, 1e-7),      # the 4x4^3 physics point
])
def test_block_tsl_jvp_fp64(dims, m_w, k, reb, with_e, m_dir, tol):
    rng = np.random.default_rng(71)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 2, rng)
    e = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape) if with_e else None
    mu = 0.3
    dx, x = binding.tsl_sign_jvp(T(u), mu, m_w, T(b), k, T(e) if with_e else None, m_dir, rebiorth=reb)
    dx, x = dx.cpu().numpy(), x.cpu().numpy()
    for s in range(2):
        rdx, rx, _ = tsl.block_tsl(u, b[s], mu, m_w, k, e, m_dir, rebiorth=reb)
        assert rel(dx[s], rdx) <= tol, (s, rel(dx[s], rdx))
        assert rel(x[s], rx) <= tol, (s, rel(x[s], rx))


@pytest.mark.parametrize("dims,k,reb", [((3, 5, 2, 4), 50, 10), ((3, 3, 3, 3), 60, 1)])
def test_block_tsl_from_general_start_fp64(dims, k, reb):
    rng = np.random.default_rng(73)
    u = inputs.su3_links(dims, 0.3, rng)
    top = inputs.gaussian_spinors(dims, 2, rng)
    bot = inputs.gaussian_spinors(dims, 2, rng)
    e = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    mu, m_w, m = 0.3, -1.0, 0.4
    zt, zb = binding.block_tsl_sign(T(u), mu, m_w, T(top), T(bot), k, T(e), m, rebiorth=reb)
    zt, zb = zt.cpu().numpy(), zb.cpu().numpy()
    for s in range(2):
        rt, rb, _ = tsl.block_tsl_start(u, top[s], bot[s], mu, m_w, k, e, m, rebiorth=reb)
        assert rel(zt[s], rt) <= 1e-10, (s, rel(zt[s], rt))
        assert rel(zb[s], rb) <= 1e-10, (s, rel(zb[s], rb))


@pytest.mark.parametrize("dims,m_w,k,reb,passes,tol", [
    ((3, 3, 3, 3), -1.0, 40, 1, 2, 1e-6),
    ((4, 4, 4, 4), -2.0, 200, 1, 2, 1e-3),      # the 4x4^3 physics point: agreement to 1e-3
])
def test_eps_a_matches_oracle(dims, m_w, k, reb, passes, tol):
    u, b, _ = case(dims, 0.3, 14, 2)
    mu = 0.3
    got = binding.tsl_eps(T(u), mu, m_w, T(b), k, rebiorth=reb, passes=passes)
    for s in range(2):
        want = tsl.eps_a(u, b[s], mu, m_w, k, rebiorth=reb, passes=passes)
        assert abs(got[s] - want) <= tol * want, (s, got[s], want)


def test_eps_b_matches_oracle():
    dims, mu, m_w, k, m = (3, 3, 2, 3), 0.3, -1.0, 40, 0.5
    rng = np.random.default_rng(74)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 2, rng)
    e = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    got = binding.block_tsl_eps(T(u), mu, m_w, T(b), k, T(e), m)
    for s in range(2):
        want = tsl.eps_b(u, b[s], mu, m_w, k, e, m)
        assert abs(got[s] - want) <= 1e-6 * want, (s, got[s], want)


def test_eps_b_without_direction_equals_eps_a():
    """dH = 0: the block estimate reduces to eps_A (the same closed form the oracle is pinned by)."""
    dims, mu, m_w, k = (3, 5, 2, 4), 0.3, -1.0, 50
    u, b, _ = case(dims, 0.3, 15, 2)
    ea = binding.tsl_eps(T(u), mu, m_w, T(b), k)
    eb = binding.block_tsl_eps(T(u), mu, m_w, T(b), k, None, 0.0)
    assert np.all(ea > 1e-6)
    assert np.all(np.abs(eb - ea) <= 1e-9 * ea), (ea, eb)


def test_block_tsl_jvp_mixed_well_conditioned():
    dims, m_w, k, mu = (3, 3, 3, 3), -1.0, 60, 0.3
    rng = np.random.default_rng(72)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    e = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    dx, x = binding.tsl_sign_jvp(T(u), mu, m_w, T(b), k, T(e), 0.5, precision="mixed")
    rdx, rx, _ = tsl.block_tsl(u, b, mu, m_w, k, e, 0.5)
    assert rel(dx.cpu().numpy(), rdx) <= 1e-4
    assert rel(x.cpu().numpy(), rx) <= 1e-4


# ---------------------------------------------------------------------------
# uneven batch
# ---------------------------------------------------------------------------
def test_uneven_batch_equals_single_calls():
    specs = [((3, 3, 3, 3), 0.3, 40, False, 1), ((3, 5, 2, 4), 0.1, 50, True, 2), ((4, 4, 4, 4), 0.5, 60, True, 1)]
    probs = []
    for n, (dims, mu, k, vjp_, nsrc) in enumerate(specs):
        u, b, xbar = case(dims, 0.3, 20 + n, nsrc)
        bb = b if nsrc > 1 else b[0]
        xb = (xbar if nsrc > 1 else xbar[0]) if vjp_ else None
        probs.append(dict(u=T(u), mu=mu, m_w=-1.0, b=T(bb), k=k, xbar=T(xb) if xb is not None else None))
    res = binding.tsl_batch(probs, nworkers=3, rebiorth=10, passes=2)
    for pr, r in zip(probs, res):
        assert r["status"] == 0
        if pr["xbar"] is None:
            x = binding.tsl_sign(pr["u"], pr["mu"], pr["m_w"], pr["b"], pr["k"], rebiorth=10, passes=2)
            assert torch.equal(r["x"], x)
        else:
            du, dmu, x = binding.tsl_sign_vjp(pr["u"], pr["mu"], pr["m_w"], pr["b"], pr["k"], pr["xbar"],
                                              rebiorth=10, passes=2)
            assert torch.equal(r["x"], x) and torch.equal(r["dU"], du) and r["dmu"] == dmu


def test_uneven_batch_against_the_oracle():
    """An uneven batch at the workloads' mass (m_w = -2): three lattices, three values
    of mu, different k and source counts, forward + VJP each, on four workers, every
    problem against the FP64 oracle (x per source, dU and dmu of the summed loss)
    within 10x the largest rounding floor the oracle measures for these maps (b
    perturbed by 1e-16: x 1.7e-11, dU 2.1e-9, dmu 3.3e-9, on the 2x3x4x5 problem)."""
    specs = [((4, 4, 4, 4), 0.1, 120, 1), ((3, 5, 2, 4), 0.3, 90, 2), ((2, 3, 4, 5), 0.5, 150, 1)]
    probs, refs = [], []
    for n, (dims, mu, k, nsrc) in enumerate(specs):
        u, b, xbar = case(dims, 0.2, 40 + n, nsrc)
        probs.append(dict(u=T(u), mu=mu, m_w=-2.0, b=T(b), k=k, xbar=T(xbar)))
        xs, du, dmu = [], np.zeros_like(u), 0.0
        for s in range(nsrc):
            f = tsl.tsl_forward(u, b[s], mu, -2.0, k, rebiorth=20, passes=1)
            d, m, _ = vjp.tsl_vjp(u, b[s], mu, -2.0, k, xbar[s], rebiorth=20, passes=1, fwd=f)
            xs.append(f.x)
            du += d
            dmu += m
        refs.append((xs, du, dmu))
    res = binding.tsl_batch(probs, nworkers=4, rebiorth=20, passes=1)
    for (xs, du, dmu), r in zip(refs, res):
        assert r["status"] == 0
        for s, xo in enumerate(xs):
            assert rel(r["x"][s].cpu().numpy(), xo) <= 2e-10
        assert rel(r["dU"].cpu().numpy(), du) <= 3e-8
        assert abs(r["dmu"] - dmu) <= 3e-8 * abs(dmu)


def test_uneven_batch_reports_each_problem_status():
    u, b, _ = case((3, 3, 3, 3), 0.3, 23, 1)
    good = dict(u=T(u), mu=0.3, m_w=-1.0, b=T(b[0]), k=30)
    bad = dict(u=T(u), mu=0.3, m_w=-1.0, b=T(b[0]), k=1)      # k < 2: invalid
    res = binding.tsl_batch([good, bad, good], nworkers=2, check=False)
    assert [r["status"] for r in res] == [0, -1, 0]
    assert torch.equal(res[0]["x"], res[2]["x"])
    assert torch.equal(res[0]["x"], binding.tsl_sign(good["u"], 0.3, -1.0, good["b"], 30))


# ---------------------------------------------------------------------------
# two-pass TSL with segment replay (no re-biorthogonalisation)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("S", [7, 16, 49])
def test_segment_replay_forward_matches_stored_basis(S):
    dims, mu, m_w, k = (3, 5, 2, 4), 0.3, -1.0, 50
    u, b, _ = case(dims, 0.3, 30, 2)
    xs = binding.tsl_sign(T(u), mu, m_w, T(b), k, rebiorth=0)
    co = [binding.tsl_coefficients(k, src=s, rebiorth=0) for s in range(2)]
    xg = binding.tsl_sign(T(u), mu, m_w, T(b), k, rebiorth=0, segment=S)
    cg = [binding.tsl_coefficients(k, src=s, rebiorth=0, segment=S) for s in range(2)]
    for s in range(2):
        for a, c in zip(co[s], cg[s]):
            assert np.array_equal(a, c)                  # the replayed recurrence is bit for bit
        assert rel(xg[s].cpu().numpy(), xs[s].cpu().numpy()) <= 1e-13
        ref = tsl.tsl_forward(u, b[s], mu, m_w, k, rebiorth=0)
        assert rel(xg[s].cpu().numpy(), ref.x) <= 1e-11


@pytest.mark.parametrize("S", [7, 10, 25])
def test_segment_replay_vjp_matches_stored_basis(S):
    dims, mu, m_w, k = (3, 5, 2, 4), 0.3, -1.0, 50
    u, b, xbar = case(dims, 0.3, 31, 2)
    du, dmu, x = binding.tsl_sign_vjp(T(u), mu, m_w, T(b), k, T(xbar), rebiorth=0)
    dug, dmug, xg = binding.tsl_sign_vjp(T(u), mu, m_w, T(b), k, T(xbar), rebiorth=0, segment=S)
    assert rel(dug.cpu().numpy(), du.cpu().numpy()) <= 1e-12
    assert abs(dmug - dmu) <= 1e-12 * abs(dmu)
    assert rel(xg.cpu().numpy(), x.cpu().numpy()) <= 1e-13
    du_o = np.zeros_like(u)
    dmu_o = 0.0
    for s in range(2):
        d, m_, _ = vjp.tsl_vjp(u, b[s], mu, m_w, k, xbar[s], rebiorth=0)
        du_o += d
        dmu_o += m_
    assert rel(dug.cpu().numpy(), du_o) <= 1e-9
    assert abs(dmug - dmu_o) <= 1e-9 * abs(dmu_o)


def test_segment_option_constraints():
    u, b, _ = case((3, 3, 3, 3), 0.3, 32, 1)
    with pytest.raises(binding.OVError) as e:       # segments need rebiorth = 0
        binding.tsl_sign(T(u), 0.3, -1.0, T(b[0]), 20, rebiorth=1, segment=5)
    assert e.value.status == -1
    with pytest.raises(binding.OVError) as e:       # not for the block TSL
        ctx = binding.context("fp64", 0, 2, segment=5)
        dx = torch.empty_like(T(b[0]))
        x = torch.empty_like(dx)
        dims = (ctypes.c_int32 * 4)(3, 3, 3, 3)
        binding._check(binding.load().ov_tsl_sign_jvp(ctx, dims, binding._ptr(T(u)), 0.3, -1.0, 1,
                                                      binding._ptr(T(b[0])), 20, None, 1.0, binding._ptr(dx),
                                                      binding._ptr(x), None), "ov_tsl_sign_jvp")
    assert e.value.status == -1
    # eps_A through the two-pass path equals the stored-basis one
    ea = binding.tsl_eps(T(u), 0.3, -1.0, T(b[0]), 30, rebiorth=0)
    eg = binding.tsl_eps(T(u), 0.3, -1.0, T(b[0]), 30, rebiorth=0, segment=8)
    assert abs(eg - ea) <= 1e-10 * ea


# ---------------------------------------------------------------------------
# reverse mode from a tape (forward kept on the device)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,reb,passes,segment", [("fp64", 10, 2, 0), ("fp64", 0, 2, 7), ("mixed", 1, 2, 0)])
def test_tape_vjp_equals_direct_vjp(precision, reb, passes, segment):
    dims, mu, m_w, k = (3, 5, 2, 4), 0.3, -1.0, 50
    u, b, xbar = case(dims, 0.3, 40, 2)
    xbar2 = inputs.gaussian_spinors(dims, 2, np.random.default_rng(41))
    opts = dict(precision=precision, rebiorth=reb, passes=passes, segment=segment)
    x, tape = binding.tsl_sign_fwd(T(u), mu, m_w, T(b), k, **opts)
    assert torch.equal(x, binding.tsl_sign(T(u), mu, m_w, T(b), k, **opts))
    for xb in (xbar, xbar2):                          # one tape, two cotangents
        du_t, dmu_t = tape.vjp(T(xb))
        du, dmu, _ = binding.tsl_sign_vjp(T(u), mu, m_w, T(b), k, T(xb), **opts)
        assert torch.equal(du_t, du) and dmu_t == dmu
    tape.free()


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(1, 2, 3, 2), (2, 1, 1, 5), (1, 1, 1, 3)])
def test_degenerate_lattice_extents(dims):
    """Extents 1 and 2: a hop wraps onto the site itself or onto the same neighbour both ways."""
    u, b, _ = case(dims, 0.3, 50, 2)
    for dagger in (False, True):
        got = binding.apply_H(T(u), 0.3, -1.0, T(b), dagger=dagger).cpu().numpy()
        for s in range(2):
            want = (dirac.apply_h_dagger if dagger else dirac.apply_h)(u, b[s], 0.3, -1.0)
            assert rel(got[s], want) <= 1e-13
    k = min(12, 12 * int(np.prod(dims)) - 1)
    x = binding.tsl_sign(T(u), 0.3, -1.0, T(b), k).cpu().numpy()
    for s in range(2):
        assert rel(x[s], tsl.tsl_forward(u, b[s], 0.3, -1.0, k).x) <= 1e-11


def test_hermitian_limit_mu_zero():
    """At mu = 0, H is Hermitian: the left and right Lanczos vectors coincide, so the
    coefficients are real and beta = delta, as in the oracle."""
    dims, k = (3, 3, 2, 3), 40
    u, b, _ = case(dims, 0.3, 51, 1)
    x = binding.tsl_sign(T(u), 0.0, -1.0, T(b[0]), k).cpu().numpy()
    a, bt, d = binding.tsl_coefficients(k)
    assert np.abs(a.imag).max() <= 1e-12 * np.abs(a.real).max()
    assert np.abs(bt[1:] - d[1:]).max() <= 1e-12 * np.abs(d[1:]).max()
    assert rel(x, tsl.tsl_forward(u, b[0], 0.0, -1.0, k).x) <= 1e-11


def test_out_of_range_arguments():
    u, b, _ = case((2, 2, 2, 2), 0.3, 52, 1)
    for k in (1, 4097):
        with pytest.raises(binding.OVError) as e:
            binding.tsl_sign(T(u), 0.3, -1.0, T(b[0]), k)
        assert e.value.status == -1
    with pytest.raises(binding.OVError) as e:          # kappa = 1/(2 m_w + 8) undefined
        binding.apply_H(T(u), 0.3, -4.0, T(b[0]))
    assert e.value.status == -1
    # a zero direction: the derivative vanishes and x is still sgn(H) b
    dx, x = binding.tsl_sign_jvp(T(u), 0.3, -1.0, T(b[0]), 20, None, 0.0)
    assert float(dx.abs().max()) == 0.0
    assert rel(x.cpu().numpy(), tsl.tsl_forward(u, b[0], 0.3, -1.0, 20).x) <= 1e-10



def test_profile_select_times_only_selected_kinds():
    """The kind mask leaves results and launch counts alone and times only the selected kinds."""
    u, b, _ = case((4, 4, 4, 4), 0.3, 1)
    ut, bt = (torch.tensor(a, device=DEV) for a in (u, b))
    ctx = binding.context("fp64", 1, 2)
    binding.profile_enable(ctx, True)
    binding.profile_read(ctx, reset=True)
    x_all = binding.tsl_sign(ut, 0.3, -2.0, bt, 40, "fp64", 1, 2)
    all_kinds = binding.profile_read(ctx, reset=True)
    binding.profile_select(ctx, ["stencil_pair", "proj_dots"])
    l0 = binding.launch_count(ctx)
    x_sel = binding.tsl_sign(ut, 0.3, -2.0, bt, 40, "fp64", 1, 2)
    nl = binding.launch_count(ctx) - l0
    sel = binding.profile_read(ctx, reset=True)
    binding.profile_select(ctx, None)
    binding.profile_enable(ctx, False)
    assert torch.equal(x_all, x_sel)
    assert nl > 0
    for kd in binding.KINDS:
        if kd in ("stencil_pair", "proj_dots"):
            assert sel[kd][0] == all_kinds[kd][0] > 0
            assert sel[kd][1] > 0.0
        else:
            assert sel[kd] == (0, 0.0)
    assert sum(v[0] for v in all_kinds.values()) > sel["stencil_pair"][0] + sel["proj_dots"][0]


@pytest.mark.parametrize("rules", ["norm", "det"])
@pytest.mark.parametrize("dims,nsrc,k", [((4, 4, 4, 4), 1, 200), ((4, 4, 4, 4), 4, 120), ((4, 4, 4, 4), 1, 700),
                                         ((4, 4, 4, 4), 1, 1100), ((2, 2, 2, 2), 1, 37)])
def test_dense_modes_identical(dims, nsrc, k, rules):
    """The cooperative k x k inversion and the per-step form give bitwise equal results
    (sign and VJP), with either Newton rule (the determinant rule also sums log|det|
    in both forms; the norm rule skips it)."""
    u, b, xbar = case(dims, 0.3, 21, nsrc)
    ut, bt, xt = (torch.tensor(a, device=DEV) for a in (u, b, xbar))
    out = {}
    for mode in (1, 0):
        binding.newton_rules(rules, "fp64", 1, 2)
        binding.dense_mode(mode, "fp64", 1, 2)
        try:
            x, info = binding.tsl_sign(ut, 0.3, -2.0, bt, k, "fp64", 1, 2, return_info=True)
            du, dmu, _ = binding.tsl_sign_vjp(ut, 0.3, -2.0, bt, k, xt, "fp64", 1, 2)
        finally:
            binding.dense_mode(0, "fp64", 1, 2)
            binding.newton_rules("norm", "fp64", 1, 2)
        out[mode] = (x, info["newton_iters"], du, dmu)
    dx = float((out[0][0] - out[1][0]).abs().max() / out[1][0].abs().max())
    ddu = float((out[0][2] - out[1][2]).abs().max() / out[1][2].abs().max())
    assert torch.equal(out[0][0], out[1][0]), f"x differs by {dx:.3e} (iters {out[0][1]} vs {out[1][1]})"
    assert out[0][1] == out[1][1]
    assert torch.equal(out[0][2], out[1][2]), f"dU differs by {ddu:.3e}"
    assert out[0][3] == out[1][3]


def test_bounded_wait_gives_up():
    """The inter-block wait of the cooperative inversion returns an error status when nothing arrives."""
    status, ms = binding.selftest_wait(1_000_000)
    assert status == -8
    assert 0.5 < ms < 50.0
    # the context is still usable afterwards
    u, b, _ = case((2, 2, 2, 2), 0.3, 3)
    x = binding.tsl_sign(torch.tensor(u, device=DEV), 0.3, -2.0, torch.tensor(b, device=DEV), 20, "fp64", 1, 2)
    assert torch.isfinite(torch.view_as_real(x)).all()
