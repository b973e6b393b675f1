"""CUDA path against the FP64 oracle at sizes that reach the code paths of the
full-size workloads, element by element through the C ABI.

* 12x12^3 (20 736 sites, two sources, k = 130, re-biorthogonalisation every
  60 steps with one pass): lattices of at least 152 blocks of 128 sites run
  the force contraction in its single-pass branch (each block a site range,
  accumulating into the force directly), which is the branch the 14x14^3 and
  6x18^3 workloads take; the projection steps 59, 60, 119 and 120 are inside
  the run, as in the benchmark's schedule (period 60, one pass).
* 4x4^3 at k = 800 (period 20, one pass): the k x k stage at the benchmark's k
  (the cooperative Gauss-Jordan inversion over 25 row blocks and the Frechet
  adjoint past its low-rank start).  At n = 3072 and k = 800 a period of 60
  leaves the k-step map chaotic (oracle rounding floor of dU ~1), so this case
  uses 20 (floors x 1.8e-13, dU 5.0e-10, dmu 3.4e-10).
* 8x8^3 with four sources at k = 400 (the four-source workload's own lattice,
  couplings and k; period 20, one pass).  This map is ill-conditioned at any
  period: the oracle's rounding floor of dU is 0.3 at period 60, 4.2e-4 at 20
  and 1.6e-4 at 10.

Bars (relative 2-norm for x and dU, relative for dmu).  At m_w = -1 the map is
well conditioned (oracle rounding floors 6e-15 for x, 2e-12 for dU, 2e-11 for
dmu at 12x12^3) and the bars are 1e-11 (x) and 1e-9 (dU, dmu).  At m_w = -2 the
floor was measured with the oracle itself, by perturbing b by 1e-16 relative
(which any change of summation order does); the bar is 10x that floor:
  12x12^3, k = 130: floor x 8.2e-12, dU 3.8e-8, dmu 9.1e-8 -> 1e-10, 4e-7, 1e-6
  8x8^3,   k = 400: floor x 1.8e-8, dU 4.2e-4, dmu 1.3e-3 -> 2e-7, 5e-3, 1.5e-2

The oracle references run in background processes (tests/oracle_jobs.py),
started when the session's tests have been collected.
"""
import numpy as np
import pytest
import torch

import oracle_jobs
from oracle import tsl, vjp
from paper_1604_08057_gb300 import binding

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def T(a):
    return torch.tensor(a, device=DEV)


def gpu_vs_oracle(name, bars):
    """Run the case's sources in one GPU call and compare with the per-source oracle:
    x per source, dU and dmu of the summed loss."""
    case = oracle_jobs.CASES[name]
    u, b, xbar = oracle_jobs.case_inputs(case)
    du, dmu, x = binding.tsl_sign_vjp(T(u), case.mu, case.m_w, T(b), case.k, T(xbar), rebiorth=case.rebiorth,
                                      passes=case.passes)
    x = x.cpu().numpy()
    du = du.cpu().numpy()
    du_o = np.zeros_like(du)
    dmu_o = 0.0
    errs = {}
    for s in range(case.nsrc):
        x_o, d_o, m_o = oracle_jobs.result(name, s)
        errs[f"x{s}"] = rel(x[s], x_o)
        du_o += d_o
        dmu_o += m_o
    errs["dU"] = rel(du, du_o)
    errs["dmu"] = abs(dmu - dmu_o) / abs(dmu_o)
    bx, bdu, bdmu = bars
    bad = {key: e for key, e in errs.items()
           if e > (bx if key.startswith("x") else bdu if key == "dU" else bdmu)}
    assert not bad, (name, errs)
    return errs


@pytest.mark.oracle_cases("w12_mw1")
def test_single_pass_force_branch_well_conditioned():
    gpu_vs_oracle("w12_mw1", (1e-11, 1e-9, 1e-9))


@pytest.mark.oracle_cases("w12_mw2")
def test_single_pass_force_branch_at_the_workload_mass():
    gpu_vs_oracle("w12_mw2", (1e-10, 4e-7, 1e-6))


@pytest.mark.oracle_cases("k800_mw1")
@pytest.mark.parametrize("dense", [0, 1])
def test_k800_sign_and_frechet_stage(dense):
    """dense = 0: the cooperative inversion (rows on chip, 25 row blocks at k = 800);
    dense = 1: one launch per elimination step.  Both against the oracle."""
    binding.dense_mode(dense, rebiorth=20, passes=1)
    try:
        gpu_vs_oracle("k800_mw1", (1e-11, 5e-9, 5e-9))
    finally:
        binding.dense_mode(0, rebiorth=20, passes=1)


@pytest.mark.oracle_cases("c1_8")
def test_four_sources_8x8x8x8_k400():
    gpu_vs_oracle("c1_8", (2e-7, 5e-3, 1.5e-2))


# ---------------------------------------------------------------------------
# mixed precision at the 4x4^3 workload point (m_w = -2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k", [40, 80])
def test_mixed_path_at_the_workload_point(k):
    """FP32 vectors, FP64 scalars, projections at every step with two passes, on
    the 4x4^3 workload's lattice, links and physics point.  The oracle's own FP32
    emulation differs from FP64 by 3.7e-7 (x) and 6.8e-5 (dU) at k = 40 and by
    1.2e-5 and 1.9e-4 at k = 80; the GPU mixed path must stay within twice the
    emulation's error (and within the stated bars 1e-5 / 1e-4 where those are
    larger).  Beyond k ~ 120 the FP32 emulation's gradient departs from the FP64
    one by O(1) at this point, so no FP32-vector path can hold a bar there."""
    from paper_1604_08057_gb300 import inputs
    wl = inputs.WORKLOADS["4x4^3"]
    u, b, xbar = inputs.make_inputs(wl)
    f64 = tsl.tsl_forward(u, b[0], wl.mu, wl.m_w, k, rebiorth=1, passes=2)
    du64, dmu64, _ = vjp.tsl_vjp(u, b[0], wl.mu, wl.m_w, k, xbar[0], rebiorth=1, passes=2, fwd=f64)
    du32, dmu32, f32 = vjp.tsl_vjp(u, b[0], wl.mu, wl.m_w, k, xbar[0], rebiorth=1, passes=2, emulate_fp32=True)
    bar_x = max(2 * rel(f32.x, f64.x), 1e-5)
    bar_du = max(2 * rel(du32, du64), 1e-4)
    bar_dmu = max(2 * abs(dmu32 - dmu64) / abs(dmu64), 1e-4)
    du, dmu, x = binding.tsl_sign_vjp(T(u), wl.mu, wl.m_w, T(b[0]), k, T(xbar[0]), precision="mixed",
                                      rebiorth=1, passes=2)
    errs = (rel(x.cpu().numpy(), f64.x), rel(du.cpu().numpy(), du64), abs(dmu - dmu64) / abs(dmu64))
    assert errs[0] <= bar_x and errs[1] <= bar_du and errs[2] <= bar_dmu, (errs, (bar_x, bar_du, bar_dmu))
