"""The k x k products of the Frechet adjoint's iteration (Theorem 1) on the BF16
tensor cores by exact digit splitting (Ozaki scheme; options.gemm), through
ov_kk_gemm, against exact and extended-precision products on the host, and the
TSL VJP with those products against the same call with FP64 products."""
import numpy as np
import pytest
import torch

from paper_1604_08057_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def op(m, h):
    return m.conj().T if h else m


def cmat(rng, k, scale_rows=0, scale_cols=0, ints=False):
    if ints:
        m = rng.integers(-(1 << 20), 1 << 20, (k, k)) + 1j * rng.integers(-(1 << 20), 1 << 20, (k, k))
    else:
        m = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    if scale_rows:
        m = m * np.exp2(rng.integers(-scale_rows, scale_rows + 1, k))[:, None]
    if scale_cols:
        m = m * np.exp2(rng.integers(-scale_cols, scale_cols + 1, k))[None, :]
    return m.astype(np.complex128)


def gpu(a, b, ha, hb, mode):
    c = binding.kk_gemm(torch.tensor(a, device=DEV), torch.tensor(b, device=DEV), ha, hb, mode)
    torch.cuda.synchronize()
    return c.cpu().numpy()


@pytest.mark.parametrize("k", [1, 7, 128, 257, 800])
@pytest.mark.parametrize("ha,hb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_split_product_is_exact_on_integer_matrices(k, ha, hb):
    """Complex integer entries below 2^20: every partial sum of the product is an
    integer below 2^53, so the host's FP64 product is exact, and so must be the
    split product (the digits hold the entries exactly and their products are
    summed exactly)."""
    rng = np.random.default_rng(1000 + k + 10 * ha + 20 * hb)
    a, b = cmat(rng, k, ints=True), cmat(rng, k, ints=True)
    exact = op(a, ha) @ op(b, hb)
    assert np.array_equal(gpu(a, b, ha, hb, "split"), exact)
    assert np.array_equal(gpu(a, b, ha, hb, "fp64"), exact)


def _extended(a, b):
    """op(A) op(B) in extended precision (long double: 64- or 113-bit significand)."""
    ar, ai = a.real.astype(np.longdouble), a.imag.astype(np.longdouble)
    br, bi = b.real.astype(np.longdouble), b.imag.astype(np.longdouble)
    return ar @ br - ai @ bi, ar @ bi + ai @ br


@pytest.mark.parametrize("k,ha,hb", [(256, 1, 0), (256, 0, 1), (600, 0, 0)])
def test_split_product_within_fp64_rounding(k, ha, hb):
    """Gaussian entries with row and column scales spread over 2^-12 .. 2^12: the
    split product's error against an extended-precision product stays within
    4u (|L||R|)_ij (the final FP64 roundings) + 12 k 2^-70 rowmax|L| colmax|R|
    (truncated digits, dropped digit products; scales up to twice the line
    maximum), and its size is that of FP64 rounding."""
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip("long double is not wider than double here")
    rng = np.random.default_rng(77 + k)
    a, b = cmat(rng, k, 12, 12), cmat(rng, k, 12, 12)
    L, R = op(a, ha), op(b, hb)
    ref_re, ref_im = _extended(L, R)
    bound = (4 * 2.0**-53 * (np.abs(L) @ np.abs(R))
             + 12 * k * 2.0**-70 * 4 * np.outer(np.abs(L).max(axis=1), np.abs(R).max(axis=0)))
    for mode in ("split", "fp64"):
        c = gpu(a, b, ha, hb, mode)
        err = np.maximum(np.abs((c.real - ref_re).astype(np.float64)), np.abs((c.imag - ref_im).astype(np.float64)))
        if mode == "split":
            assert np.all(err <= bound)
            split_err = np.linalg.norm(err)
        else:
            fp64_err = np.linalg.norm(err)
    assert split_err <= 2 * fp64_err


def test_split_product_propagates_non_finite_entries():
    k = 160
    rng = np.random.default_rng(5)
    a, b = cmat(rng, k), cmat(rng, k)
    a[3, 5] = np.nan
    b[7, 11] = np.inf
    c = gpu(a, b, 0, 0, "split")
    assert np.all(np.isnan(c[3]))        # row 3 of A holds the NaN
    assert np.all(np.isnan(c[:, 11]))    # column 11 of B holds the Inf
    rows = [i for i in range(k) if i != 3]
    cols = [j for j in range(k) if j != 11]
    ref = a @ b
    assert np.allclose(c[np.ix_(rows, cols)], ref[np.ix_(rows, cols)], rtol=1e-12, atol=1e-12)


def test_kk_gemm_argument_checks():
    z = torch.zeros((1025, 1025), dtype=torch.complex128, device=DEV)
    with pytest.raises(binding.OVError):
        binding.kk_gemm(z, z, mode="split")          # beyond the exact-accumulation limit
    c = binding.kk_gemm(z, z, mode="fp64")             # FP64 has no limit
    assert float(c.abs().max()) == 0.0


def test_vjp_with_split_products_matches_fp64_products():
    """The 4x4^3, k = 200 workload's VJP with tensor-core products in the Frechet
    adjoint against FP64 products: the same x bit for bit (the forward pass forms
    no products), and dU, dmu within the bar of this schedule's parity against the
    oracle (10x the map's rounding floor: dU 7.4e-7, dmu 2.7e-7), since the two
    product forms differ only by rounding."""
    wl = inputs.WORKLOADS["4x4^3"]
    u, b, xbar = inputs.make_inputs(wl)
    reb, passes = 20, 1
    out = {}
    try:
        for mode in ("fp64", "split"):
            binding.kk_products(mode, rebiorth=reb, passes=passes)
            du, dmu, x = binding.tsl_sign_vjp(torch.tensor(u, device=DEV), wl.mu, wl.m_w,
                                              torch.tensor(b[0], device=DEV), wl.k,
                                              torch.tensor(xbar[0], device=DEV), rebiorth=reb, passes=passes)
            out[mode] = (x.cpu().numpy(), du.cpu().numpy(), dmu)
    finally:
        binding.kk_products("auto", rebiorth=reb, passes=passes)
    (x64, du64, dmu64), (xs, dus, dmus) = out["fp64"], out["split"]
    assert np.array_equal(xs, x64)   # the forward pass has no products
    r_du = np.linalg.norm(dus - du64) / np.linalg.norm(du64)
    r_dmu = abs(complex(dmus) - complex(dmu64)) / abs(complex(dmu64))
    assert r_du <= 5e-6 and r_dmu <= 5e-6, (r_du, r_dmu)
