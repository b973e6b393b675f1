"""Thin Python binding of the C ABI in ``include/ov.h`` (argument marshalling only).

Every numerical step runs in the CUDA library; this module checks shapes and
dtypes of torch tensors, passes their device pointers and the current CUDA
stream, and turns status codes into exceptions.  There is no CPU path: if the
library has not been built, ``load()`` raises.

Tensor conventions (complex128, contiguous, on a CUDA device):
    U    (Nt, Nz, Ny, Nx, 4, 3, 3)    links, direction order x, y, z, t
    psi  (nsrc, Nt, Nz, Ny, Nx, 4, 3) or (Nt, Nz, Ny, Nx, 4, 3) for one source
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libov.so")

OV_FP64, OV_MIXED = 0, 1
_PREC = {"fp64": OV_FP64, "mixed": OV_MIXED}

_lib = None
_contexts = {}


class OVError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_lib.ov_strerror(status).decode()} (status {status})")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("rebiorth", ctypes.c_int32),
                ("passes", ctypes.c_int32), ("segment", ctypes.c_int32), ("dense", ctypes.c_int32),
                ("diagnostics", ctypes.c_int32), ("newton", ctypes.c_int32),
                ("basis_memory", ctypes.c_int32), ("graphs", ctypes.c_int32), ("gemm", ctypes.c_int32),
                ("nested", ctypes.c_int32)]


class TuneReport(ctypes.Structure):
    _fields_ = [("apply_variant", ctypes.c_int32), ("pair_variant", ctypes.c_int32),
                ("n_apply", ctypes.c_int32), ("n_pair", ctypes.c_int32),
                ("apply_us", ctypes.c_float * 16), ("pair_us", ctypes.c_float * 16)]


class Info(ctypes.Structure):
    _fields_ = [("k_reached", ctypes.c_int32), ("newton_iters", ctypes.c_int32),
                ("newton_iters_adj", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("min_abs_re_ritz", ctypes.c_double), ("t_ms", ctypes.c_double * 8),
                ("biorth_loss", ctypes.c_double), ("t_norm", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {"k_reached": self.k_reached, "newton_iters": self.newton_iters,
                "newton_iters_adj": self.newton_iters_adj, "t_ms": list(self.t_ms),
                "min_abs_re_ritz": self.min_abs_re_ritz, "biorth_loss": self.biorth_loss,
                "t_norm": self.t_norm}


class Problem(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("U", ctypes.c_void_p), ("mu", ctypes.c_double),
                ("m_w", ctypes.c_double), ("nsrc", ctypes.c_int32), ("b", ctypes.c_void_p), ("k", ctypes.c_int32),
                ("xbar", ctypes.c_void_p), ("x", ctypes.c_void_p), ("dU", ctypes.c_void_p),
                ("dmu", ctypes.c_void_p), ("info", Info), ("status", ctypes.c_int32)]


EXPORTS = ["ov_context_create", "ov_context_destroy", "ov_context_set_options", "ov_apply_H",
           "ov_tsl_sign", "ov_tsl_sign_vjp", "ov_tsl_coefficients", "ov_profile_enable", "ov_profile_read",
           "ov_launch_count", "ov_apply_H_noalloc", "ov_autotune", "ov_set_stencil_variants",
           "ov_tsl_sign_jvp", "ov_block_tsl_sign", "ov_tsl_eps", "ov_block_tsl_eps", "ov_tsl_batch", "ov_profile_select", "ov_selftest_wait", "ov_tsl_sign_fwd", "ov_tsl_sign_vjp_tape", "ov_tape_destroy", "ov_tridiag_eigenvalues", "ov_debug_inject", "ov_overlap_apply", "ov_overlap_solve", "ov_u1_current",
           "ov_kk_gemm", "ov_tsl_sign_deflated", "ov_tsl_sign_jvp_deflated",
           "ov_tridiag_eigenvector", "ov_tsl_ritz_triples",
           "ov_eigen_derivatives",
           "ov_hessenberg_eigen", "ov_eigen_smallest", "ov_tridiag_sign_nested", "ov_strerror"]

KINDS = ["stencil_pair", "update", "proj_dots", "proj_update", "combine", "dense", "rev_scalar",
         "rev_stencil", "force", "apply_h", "layout", "dense_gemm"]


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I32, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    dims_t = ctypes.POINTER(ctypes.c_int32)
    lib.ov_context_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Options), P]
    lib.ov_context_destroy.argtypes = [P]
    lib.ov_context_set_options.argtypes = [P, ctypes.POINTER(Options)]
    lib.ov_apply_H.argtypes = [P, dims_t, P, D, D, I32, P, P, I32]
    lib.ov_tsl_sign.argtypes = [P, dims_t, P, D, D, I32, P, I32, P, ctypes.POINTER(Info)]
    lib.ov_tsl_sign_vjp.argtypes = [P, dims_t, P, D, D, I32, P, I32, P, P, P,
                                    ctypes.POINTER(D), ctypes.POINTER(Info)]
    lib.ov_tsl_coefficients.argtypes = [P, I32, I32, P, P, P]
    lib.ov_tsl_sign_jvp.argtypes = [P, dims_t, P, D, D, I32, P, I32, P, D, P, P, ctypes.POINTER(Info)]
    lib.ov_block_tsl_sign.argtypes = [P, dims_t, P, D, D, I32, P, P, I32, P, D, P, P, ctypes.POINTER(Info)]
    lib.ov_tsl_batch.argtypes = [P, I32, ctypes.POINTER(Problem), I32]
    lib.ov_tsl_sign_fwd.argtypes = [P, dims_t, P, D, D, I32, P, I32, P, ctypes.POINTER(Info), ctypes.POINTER(P)]
    lib.ov_tsl_sign_vjp_tape.argtypes = [P, P, P, ctypes.POINTER(D), ctypes.POINTER(Info)]
    lib.ov_tape_destroy.argtypes = [P]
    lib.ov_tsl_eps.argtypes = [P, dims_t, P, D, D, I32, P, I32, P, ctypes.POINTER(Info)]
    lib.ov_block_tsl_eps.argtypes = [P, dims_t, P, D, D, I32, P, I32, P, D, P, ctypes.POINTER(Info)]
    lib.ov_profile_enable.argtypes = [P, I32]
    lib.ov_profile_select.argtypes = [P, ctypes.c_uint32]
    lib.ov_selftest_wait.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(D)]
    lib.ov_profile_read.argtypes = [P, I32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(D), I32]
    lib.ov_autotune.argtypes = [P, dims_t, P, D, D, I32, ctypes.POINTER(TuneReport)]
    lib.ov_set_stencil_variants.argtypes = [P, I32, I32]
    lib.ov_tridiag_eigenvalues.argtypes = [I32, P, P, P, P]
    lib.ov_tridiag_sign_nested.argtypes = [P, I32, P, P, P, I32, D, P, ctypes.POINTER(I32)]
    lib.ov_tridiag_eigenvector.argtypes = [I32, P, P, P, P, I32, P]
    lib.ov_hessenberg_eigen.argtypes = [I32, P, P, P]
    lib.ov_eigen_smallest.argtypes = [P, dims_t, P, D, D, I32, I32, P, D, I32, ctypes.POINTER(I32), P, P, P, P]
    lib.ov_tsl_ritz_triples.argtypes = [P, dims_t, P, D, D, I32, I32, I32, D, ctypes.POINTER(I32), P, P, P, P]
    lib.ov_eigen_derivatives.argtypes = [P, dims_t, P, D, D, P, D, I32, P, P, P, D, I32, P, P, P, P]
    lib.ov_overlap_apply.argtypes = [P, dims_t, P, D, D, I32, P, I32, I32, P, ctypes.POINTER(Info)]
    lib.ov_overlap_solve.argtypes = [P, dims_t, P, D, D, I32, P, I32, I32, D, I32, P, ctypes.POINTER(I32),
                                     ctypes.POINTER(D)]
    lib.ov_u1_current.argtypes = [P, dims_t, P, D, D, I32, P, I32, D, I32, P, ctypes.POINTER(D), ctypes.POINTER(Info)]
    lib.ov_debug_inject.argtypes = [P, I32, I32]
    lib.ov_kk_gemm.argtypes = [P, P, I32, P, I32, P, I32, I32]
    lib.ov_tsl_sign_deflated.argtypes = [P, dims_t, P, D, D, I32, P, I32, I32, P, P, P, P, ctypes.POINTER(Info)]
    lib.ov_tsl_sign_jvp_deflated.argtypes = [P, dims_t, P, D, D, I32, P, I32, P, D, I32, P, P, P, P, P, P, P,
                                             ctypes.POINTER(Info)]
    lib.ov_launch_count.argtypes = [P]
    lib.ov_launch_count.restype = ctypes.c_int64
    lib.ov_strerror.argtypes = [ctypes.c_int]
    lib.ov_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != 0:
        raise OVError(status, what)


def context(precision: str = "fp64", rebiorth: int = 1, passes: int = 2, device=None, segment: int = 0):
    """A cached library context for (device, current stream, options).  segment > 0
    selects the two-pass TSL with checkpoints every `segment` steps (rebiorth = 0)."""
    lib = load()
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    stream = torch.cuda.current_stream(dev).cuda_stream
    key = (dev.index, stream, precision, rebiorth, passes, segment)
    if key not in _contexts:
        opt = Options(_PREC[precision], rebiorth, passes, segment)
        opt.graphs = 1
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _check(lib.ov_context_create(ctypes.byref(h), ctypes.byref(opt), ctypes.c_void_p(stream)),
                   "ov_context_create")
        _contexts[key] = h
    return _contexts[key]


_extra = {}   # per cached context: the options not in its key (dense, diagnostics, newton, basis memory, graphs)


def _set_extra(precision, rebiorth, passes, segment, **kw):
    ctx = context(precision, rebiorth, passes, segment=segment)
    key = (precision, rebiorth, passes, segment, ctx.value)
    ex = _extra.setdefault(key, {"dense": 0, "diagnostics": 0, "newton": 0, "basis_memory": 0, "graphs": 1,
                                 "gemm": 0, "nested": 0})
    ex.update({k: int(v) for k, v in kw.items()})
    opt = Options(_PREC[precision], rebiorth, passes, segment, ex["dense"], ex["diagnostics"], ex["newton"],
                  ex["basis_memory"], ex["graphs"], ex["gemm"], ex["nested"])
    _check(load().ov_context_set_options(ctx, ctypes.byref(opt)), "ov_context_set_options")
    return ctx


def dense_mode(mode: int, precision: str = "fp64", rebiorth: int = 1, passes: int = 2, segment: int = 0):
    """How the k x k inversions run on the cached context for these options:
    0 one cooperative launch per inversion where the rows fit on chip (default),
    1 one launch per Gauss-Jordan step replayed as a graph (identical results)."""
    _set_extra(precision, rebiorth, passes, segment, dense=mode)


def diagnostics_mode(on: bool, precision: str = "fp64", rebiorth: int = 1, passes: int = 2, segment: int = 0):
    """Run diagnostics (biorthogonality loss, Ritz values, ill-posed sign check) on the
    cached context for these options; results appear in the calls' info."""
    _set_extra(precision, rebiorth, passes, segment, diagnostics=on)


def newton_rules(rules: str, precision: str = "fp64", rebiorth: int = 1, passes: int = 2, segment: int = 0):
    """Rules of the k x k Newton sign on the cached context: "norm" (Frobenius-norm
    scaling, predicted stop; the default) or "det" (determinant scaling, stagnation stop)."""
    _set_extra(precision, rebiorth, passes, segment, newton={"norm": 0, "det": 1}[rules])


def basis_memory(where: str, precision: str = "fp64", rebiorth: int = 1, passes: int = 2, segment: int = 0):
    """Where the cached context keeps the Krylov bases: "device" (default) or "host"
    (pinned host memory the kernels read over the CPU-GPU link)."""
    _set_extra(precision, rebiorth, passes, segment, basis_memory={"device": 0, "host": 1}[where])


def sweep_graphs(on: bool, precision: str = "fp64", rebiorth: int = 1, passes: int = 2, segment: int = 0):
    """Capture and replay the Krylov sweeps as CUDA graphs on the cached context (on by
    default) or launch every kernel directly; the results are the same bit for bit."""
    _set_extra(precision, rebiorth, passes, segment, graphs=int(bool(on)))


def kk_products(mode: str, precision: str = "fp64", rebiorth: int = 1, passes: int = 2, segment: int = 0):
    """How the cached context forms the k x k products of the Frechet adjoint:
    "auto" (default: BF16 tensor cores by exact digit splitting for 128 <= k <= 1024,
    else FP64), "fp64", or "split" (the tensor-core form wherever k <= 1024)."""
    _set_extra(precision, rebiorth, passes, segment, gemm={"auto": 0, "fp64": 1, "split": 2}[mode])


def nested_sign(m: int, precision: str = "fp64", rebiorth: int = 1, passes: int = 2, segment: int = 0):
    """k x k sign of the forward passes on the cached context: 0 (default) the full
    Newton sign of T_k, m > 0 the nested TSL with inner Krylov size m (one nesting level:
    Arnoldi on (T_k + T_k^-1)/2 from e_1).  The reverse mode refuses nested > 0."""
    _set_extra(precision, rebiorth, passes, segment, nested=int(m))


def debug_inject(kind: str, step: int = 0, precision: str = "fp64", rebiorth: int = 1, passes: int = 2,
                 segment: int = 0):
    """One-shot host-side fault injection on the cached context: 'breakdown' or
    'nonfinite' at Lanczos step `step`, or 'oom' after `step` successful allocations."""
    kinds = {"none": 0, "breakdown": 1, "nonfinite": 2, "oom": 3}
    ctx = context(precision, rebiorth, passes, segment=segment)
    _check(load().ov_debug_inject(ctx, kinds[kind], int(step)), "ov_debug_inject")


def overlap_apply(u, mu, m_w, b, k, dagger=False, precision="fp64", rebiorth=1, passes=2):
    """D_ov b = b + gamma5 sgn(H) b (or D_ov^dagger b), the sign by k-step TSL."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    bb, single = _spinors(b, u)
    out = torch.empty_like(bb)
    ctx = context(precision, rebiorth, passes)
    _check(lib.ov_overlap_apply(ctx, dims, _ptr(u), float(mu), float(m_w), bb.shape[0], _ptr(bb), int(k),
                                int(bool(dagger)), _ptr(out), None), "ov_overlap_apply")
    return out[0] if single else out


def overlap_solve(u, mu, m_w, rhs, k, dagger=False, tol=1e-10, maxit=300, precision="fp64", rebiorth=1,
                  passes=2, check=True):
    """x with D_ov x = rhs (or D_ov^dagger x = rhs) by restarted GMRES; returns
    (x, iterations, relative residual)."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    bb, single = _spinors(rhs, u)
    x = torch.empty_like(bb)
    it = ctypes.c_int32(0)
    res = ctypes.c_double(0.0)
    ctx = context(precision, rebiorth, passes)
    st = lib.ov_overlap_solve(ctx, dims, _ptr(u), float(mu), float(m_w), bb.shape[0], _ptr(bb), int(k),
                              int(bool(dagger)), float(tol), int(maxit), _ptr(x), ctypes.byref(it), ctypes.byref(res))
    if check:
        _check(st, "ov_overlap_solve")
    return (x[0] if single else x), it.value, res.value


def u1_current(u, mu, m_w, eta, k, tol=1e-10, maxit=300, precision="fp64", rebiorth=1, passes=2):
    """Z2-noise estimator of j_{x,nu} = Tr(D_ov^{-1} dD_ov/dTheta_{x,nu}) for all links,
    shape (Nt, Nz, Ny, Nx, 4) complex128, and of Tr(D_ov^{-1} dD_ov/dmu)."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    ee, _ = _spinors(eta, u)
    j = torch.empty(tuple(u.shape[:5]), dtype=torch.complex128, device=u.device)
    tr = (ctypes.c_double * 2)()
    ctx = context(precision, rebiorth, passes)
    _check(lib.ov_u1_current(ctx, dims, _ptr(u), float(mu), float(m_w), ee.shape[0], _ptr(ee), int(k), float(tol),
                             int(maxit), _ptr(j), tr, None), "ov_u1_current")
    return j, complex(tr[0], tr[1])


def tridiag_eigenvalues(alpha, beta, delta):
    """Eigenvalues of the TSL tridiagonal (host numpy arrays as tsl_coefficients returns
    them: complex alpha[k], complex beta[k] with beta[0] unused, real delta[k])."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.complex128))
    b = np.ascontiguousarray(np.asarray(beta, dtype=np.complex128))
    d = np.ascontiguousarray(np.asarray(delta, dtype=np.float64))
    k = a.shape[0]
    if b.shape != (k,) or d.shape != (k,):
        raise ValueError("alpha, beta, delta must have length k")
    out = np.empty(k, dtype=np.complex128)
    _check(load().ov_tridiag_eigenvalues(k, a.ctypes.data, b.ctypes.data, d.ctypes.data, out.ctypes.data),
           "ov_tridiag_eigenvalues")
    return out


def tridiag_sign_nested(alpha, beta, delta, m, beta0=1.0, device=None):
    """beta0 sgn(T) e_1 for the TSL tridiagonal (host numpy arrays as tsl_coefficients
    returns them) on the device: m = 0 the full Newton sign, m > 0 the nested
    approximation with inner Krylov size m.  Returns (y, newton_iters)."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.complex128))
    b = np.ascontiguousarray(np.asarray(beta, dtype=np.complex128))
    d = np.ascontiguousarray(np.asarray(delta, dtype=np.float64))
    k = a.shape[0]
    if b.shape != (k,) or d.shape != (k,):
        raise ValueError("alpha, beta, delta must have length k")
    y = np.empty(k, dtype=np.complex128)
    it = ctypes.c_int32(0)
    ctx = context("fp64", 1, 2, device=device)
    _check(load().ov_tridiag_sign_nested(ctx, k, a.ctypes.data, b.ctypes.data, d.ctypes.data, int(m), float(beta0),
                                         y.ctypes.data, ctypes.byref(it)), "ov_tridiag_sign_nested")
    return y, int(it.value)


def kk_gemm(a, b, ha=False, hb=False, mode="split"):
    """C = op(a) op(b) for complex128 CUDA k x k matrices (op = conjugate transpose
    when the flag is set), by FP64 arithmetic ("fp64") or the BF16 tensor-core digit
    splitting ("split", k <= 1024) of the Frechet adjoint's products."""
    for m in (a, b):
        if m.dtype != torch.complex128 or not m.is_cuda or m.dim() != 2 or m.shape[0] != m.shape[1]:
            raise ValueError("a and b must be square complex128 CUDA matrices")
    if a.shape != b.shape:
        raise ValueError("a and b must have the same shape")
    a, b = a.contiguous(), b.contiguous()
    c = torch.empty_like(a)
    ctx = context("fp64", 1, 2, device=a.device.index)
    _check(load().ov_kk_gemm(ctx, a.data_ptr(), int(bool(ha)), b.data_ptr(), int(bool(hb)), c.data_ptr(),
                             a.shape[0], {"fp64": 1, "split": 2}[mode]), "ov_kk_gemm")
    return c


def tridiag_eigenvector(alpha, beta, delta, theta, left=False):
    """Right (or, with left=True, left: z^dag T = theta z^dag) eigenvector of the TSL
    tridiagonal for the eigenvalue theta, unit norm, by inverse iteration (host)."""
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.complex128))
    b = np.ascontiguousarray(np.asarray(beta, dtype=np.complex128))
    d = np.ascontiguousarray(np.asarray(delta, dtype=np.float64))
    k = a.size
    th = np.array([complex(theta)], dtype=np.complex128)
    out = np.zeros(k, dtype=np.complex128)
    _check(load().ov_tridiag_eigenvector(k, a.ctypes.data, b.ctypes.data, d.ctypes.data, th.ctypes.data,
                                         int(bool(left)), out.ctypes.data), "ov_tridiag_eigenvector")
    return out


def hessenberg_eigen(h, vectors=True):
    """Eigenvalues (and unit right eigenvectors, as columns) of a complex upper
    Hessenberg matrix, on the host."""
    a = np.ascontiguousarray(np.asarray(h, dtype=np.complex128))
    m = a.shape[0]
    eig = np.zeros(m, dtype=np.complex128)
    vec = np.zeros((m, m), dtype=np.complex128) if vectors else None
    _check(load().ov_hessenberg_eigen(m, a.ctypes.data, eig.ctypes.data, vec.ctypes.data if vectors else None),
           "ov_hessenberg_eigen")
    return (eig, vec) if vectors else eig


def _dims(u: torch.Tensor):
    if u.dtype != torch.complex128 or not u.is_cuda or u.dim() != 7 or tuple(u.shape[4:]) != (4, 3, 3):
        raise ValueError("U must be complex128 CUDA (Nt, Nz, Ny, Nx, 4, 3, 3)")
    nt, nz, ny, nx = u.shape[:4]
    return (ctypes.c_int32 * 4)(nx, ny, nz, nt)


def _spinors(psi: torch.Tensor, u: torch.Tensor):
    if psi.dtype != torch.complex128 or not psi.is_cuda:
        raise ValueError("spinor fields must be complex128 CUDA tensors")
    lat = tuple(u.shape[:4]) + (4, 3)
    if tuple(psi.shape) == lat:
        return psi.contiguous().unsqueeze(0), True
    if psi.dim() == 7 and tuple(psi.shape[1:]) == lat:
        return psi.contiguous(), False
    raise ValueError(f"spinor shape {tuple(psi.shape)} does not match the lattice {lat}")


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def apply_H(u, mu, m_w, psi, dagger=False, precision="fp64"):
    """H(mu) psi or H(mu)^dagger psi."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    p, single = _spinors(psi, u)
    out = torch.empty_like(p)
    ctx = context(precision)
    _check(lib.ov_apply_H(ctx, dims, _ptr(u), float(mu), float(m_w), p.shape[0], _ptr(p), _ptr(out),
                          int(bool(dagger))), "ov_apply_H")
    return out[0] if single else out


def tsl_sign(u, mu, m_w, b, k, precision="fp64", rebiorth=1, passes=2, return_info=False, segment=0):
    """x ~ sgn(H(mu)) b by k-step two-sided Lanczos (per source)."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    bb, single = _spinors(b, u)
    x = torch.empty_like(bb)
    info = Info()
    ctx = context(precision, rebiorth, passes, segment=segment)
    _check(lib.ov_tsl_sign(ctx, dims, _ptr(u), float(mu), float(m_w), bb.shape[0], _ptr(bb), int(k),
                           _ptr(x), ctypes.byref(info)), "ov_tsl_sign")
    x = x[0] if single else x
    return (x, info.as_dict()) if return_info else x


class Tape:
    """The forward state kept by ov_tsl_sign_fwd for later VJPs (device memory
    until the object is freed)."""

    def __init__(self, handle, u, bb, single):
        self._h = handle
        self._u = u                # the links the reverse mode writes dU for (shape, device)
        self._shape = bb.shape
        self._single = single

    def vjp(self, xbar, return_info=False):
        """(dU, dmu) for L = sum_src Re <xbar, x> from the kept forward pass."""
        if self._h is None:
            raise RuntimeError("tape already freed")
        xb, _ = _spinors(xbar, self._u)
        if xb.shape != self._shape:
            raise ValueError("xbar must have the shape of b")
        du = torch.empty_like(self._u)
        dmu = ctypes.c_double(0.0)
        info = Info()
        _check(load().ov_tsl_sign_vjp_tape(self._h, _ptr(xb), _ptr(du), ctypes.byref(dmu), ctypes.byref(info)),
               "ov_tsl_sign_vjp_tape")
        return (du, dmu.value, info.as_dict()) if return_info else (du, dmu.value)

    def free(self):
        if self._h is not None and _lib is not None:
            _lib.ov_tape_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def tsl_sign_fwd(u, mu, m_w, b, k, precision="fp64", rebiorth=1, passes=2, segment=0):
    """(x, tape): x ~ sgn(H(mu)) b as tsl_sign, and a Tape for VJPs that skip the forward pass."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    bb, single = _spinors(b, u)
    x = torch.empty_like(bb)
    info = Info()
    h = ctypes.c_void_p()
    ctx = context(precision, rebiorth, passes, segment=segment)
    _check(lib.ov_tsl_sign_fwd(ctx, dims, _ptr(u), float(mu), float(m_w), bb.shape[0], _ptr(bb), int(k), _ptr(x),
                               ctypes.byref(info), ctypes.byref(h)), "ov_tsl_sign_fwd")
    return (x[0] if single else x), Tape(h, u, bb, single)


def tsl_sign_vjp(u, mu, m_w, b, k, xbar, precision="fp64", rebiorth=1, passes=2, want_x=True,
                 return_info=False, segment=0):
    """(dU, dmu, x) for L = sum_src Re <xbar, x>."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    bb, single = _spinors(b, u)
    xb, _ = _spinors(xbar, u)
    if xb.shape != bb.shape:
        raise ValueError("xbar must have the shape of b")
    x = torch.empty_like(bb) if want_x else None
    du = torch.empty_like(u)
    dmu = ctypes.c_double(0.0)
    info = Info()
    ctx = context(precision, rebiorth, passes, segment=segment)
    _check(lib.ov_tsl_sign_vjp(ctx, dims, _ptr(u), float(mu), float(m_w), bb.shape[0], _ptr(bb), int(k),
                               _ptr(xb), _ptr(x) if x is not None else None, _ptr(du),
                               ctypes.byref(dmu), ctypes.byref(info)), "ov_tsl_sign_vjp")
    if x is not None and single:
        x = x[0]
    out = (du, dmu.value, x)
    return out + (info.as_dict(),) if return_info else out


def tsl_sign_jvp(u, mu, m_w, b, k, e=None, m_dir=0.0, precision="fp64", rebiorth=1, passes=2,
                 return_info=False):
    """Theorem 1: (dx, x) with dx ~ d/dt sgn(H(U + tE, mu + t m_dir)) b, x ~ sgn(H) b."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    bb, single = _spinors(b, u)
    if e is not None:
        _dims(e)
        e = e.contiguous()
    x = torch.empty_like(bb)
    dx = torch.empty_like(bb)
    info = Info()
    ctx = context(precision, rebiorth, passes)
    _check(lib.ov_tsl_sign_jvp(ctx, dims, _ptr(u), float(mu), float(m_w), bb.shape[0], _ptr(bb), int(k),
                               _ptr(e) if e is not None else None, float(m_dir), _ptr(dx), _ptr(x),
                               ctypes.byref(info)), "ov_tsl_sign_jvp")
    if single:
        dx, x = dx[0], x[0]
    return (dx, x, info.as_dict()) if return_info else (dx, x)


def _eigen_args(u, lam, fields):
    """Host complex eigenvalues -> interleaved doubles; eigenvector fields -> contiguous
    complex128 CUDA tensors shaped (l, Nt, Nz, Ny, Nx, 4, 3)."""
    lam = np.ascontiguousarray(np.asarray(lam, dtype=np.complex128).reshape(-1))
    l = lam.size
    out = []
    for f in fields:
        if f is None:
            out.append(None)
            continue
        if f.dtype != torch.complex128 or not f.is_cuda or tuple(f.shape) != (l,) + tuple(u.shape[:4]) + (4, 3):
            raise ValueError("eigenvector fields must be complex128 CUDA, shaped (l, Nt, Nz, Ny, Nx, 4, 3)")
        out.append(f.contiguous())
    lam_d = lam.view(np.float64).copy()
    return l, lam_d, out


def ritz_triples(u, mu, m_w, k, lmax, tol, src=0, precision="fp64", rebiorth=1, passes=2):
    """Ritz triples (theta, R, L, residual) of the last forward pass on the cached
    context for these options (a preceding tsl_sign or tsl_sign_vjp with the same U,
    k): up to lmax with ||H R - theta R|| / ||R|| <= tol, in order of |theta|."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    shape = (lmax,) + tuple(u.shape[:4]) + (4, 3)
    R = torch.empty(shape, dtype=torch.complex128, device=u.device)
    L = torch.empty_like(R)
    lam = np.zeros(lmax, dtype=np.complex128)
    res = np.zeros(lmax, dtype=np.float64)
    nl = ctypes.c_int32(0)
    ctx = context(precision, rebiorth, passes)
    _check(lib.ov_tsl_ritz_triples(ctx, dims, _ptr(u), float(mu), float(m_w), int(src), int(k), int(lmax),
                                   float(tol), ctypes.byref(nl), lam.ctypes.data, _ptr(R), _ptr(L),
                                   res.ctypes.data), "ov_tsl_ritz_triples")
    n = nl.value
    return lam[:n], R[:n], L[:n], res[:n]


def eigen_smallest(u, mu, m_w, l, m, start, tol=1e-12, maxit=20000):
    """(lam, R, L, residuals): up to l eigen-triples of H smallest in |lambda| by
    shift-and-invert Arnoldi with m steps per side from the start field."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    st, single = _spinors(start, u)
    if st.shape[0] != 1:
        raise ValueError("one start field")
    shape = (l,) + tuple(u.shape[:4]) + (4, 3)
    R = torch.empty(shape, dtype=torch.complex128, device=u.device)
    L = torch.empty_like(R)
    lam = np.zeros(l, dtype=np.complex128)
    res = np.zeros(l, dtype=np.float64)
    nl = ctypes.c_int32(0)
    ctx = context("fp64", 1, 2)
    code = lib.ov_eigen_smallest(ctx, dims, _ptr(u), float(mu), float(m_w), int(l), int(m), _ptr(st), float(tol),
                                 int(maxit), ctypes.byref(nl), lam.ctypes.data, _ptr(R), _ptr(L), res.ctypes.data)
    if code not in (0, -9):
        _check(code, "ov_eigen_smallest")
    n = nl.value
    return lam[:n], R[:n], L[:n], res[:n]


def eigen_derivatives(u, mu, m_w, lam, R, L, e=None, m_dir=0.0, tol=1e-11, maxit=20000):
    """(dlam, dR, dL, residuals): derivatives of the eigen-triples along (E, m_dir) by
    shifted solves (CG on the normal equations; App. B, E), normalised by
    <L_i|dR_i> = <dL_i|R_i> = 0."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    if e is not None:
        _dims(e)
        e = e.contiguous()
    l, lam_d, (rr, ll) = _eigen_args(u, lam, (R, L))
    dR = torch.empty_like(rr)
    dL = torch.empty_like(ll)
    dlam = np.zeros(l, dtype=np.complex128)
    res = np.zeros(2 * l, dtype=np.float64)
    ctx = context("fp64", 1, 2)
    st = lib.ov_eigen_derivatives(ctx, dims, _ptr(u), float(mu), float(m_w), _ptr(e) if e is not None else None,
                                  float(m_dir), l, lam_d.ctypes.data, _ptr(rr), _ptr(ll), float(tol), int(maxit),
                                  dlam.ctypes.data, _ptr(dR), _ptr(dL), res.ctypes.data)
    if st not in (0, -9):     # OV_OK, or OV_ERR_NOCONV with everything written
        _check(st, "ov_eigen_derivatives")
    return dlam, dR, dL, res.reshape(l, 2)


def tsl_sign_deflated(u, mu, m_w, b, k, lam, R, L, precision="fp64", rebiorth=1, passes=2, return_info=False):
    """Standard deflation (Sec. 3): x = TSL_k(H, Pbar b) + sum_i sgn(Re lam_i) R_i (L_i^dag b)
    with the caller's eigen-triples (lam: l complex numbers; R, L: eigenvector fields)."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    bb, single = _spinors(b, u)
    l, lam_d, (rr, ll) = _eigen_args(u, lam, (R, L))
    x = torch.empty_like(bb)
    info = Info()
    ctx = context(precision, rebiorth, passes)
    _check(lib.ov_tsl_sign_deflated(ctx, dims, _ptr(u), float(mu), float(m_w), bb.shape[0], _ptr(bb), int(k), l,
                                    lam_d.ctypes.data if l else None, _ptr(rr) if l else None,
                                    _ptr(ll) if l else None, _ptr(x), ctypes.byref(info)), "ov_tsl_sign_deflated")
    if single:
        x = x[0]
    return (x, info.as_dict()) if return_info else x


def tsl_sign_jvp_deflated(u, mu, m_w, b, k, lam, R, L, dR, dL, e=None, m_dir=0.0, precision="fp64", rebiorth=1,
                          passes=2, return_info=False):
    """Generalised deflation of Theorem 1's block matrix (Sec. 3, Eq. final_res): (dx, x)
    with dx ~ d/dt sgn(H(U + tE, mu + t m_dir)) b and x ~ sgn(H) b; dR, dL are the
    eigenvector derivatives along the same direction (App. B)."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    bb, single = _spinors(b, u)
    if e is not None:
        _dims(e)
        e = e.contiguous()
    l, lam_d, (rr, ll, drr, dll) = _eigen_args(u, lam, (R, L, dR, dL))
    x = torch.empty_like(bb)
    dx = torch.empty_like(bb)
    info = Info()
    ctx = context(precision, rebiorth, passes)
    ptr = lambda t: _ptr(t) if (l and t is not None) else None
    _check(lib.ov_tsl_sign_jvp_deflated(ctx, dims, _ptr(u), float(mu), float(m_w), bb.shape[0], _ptr(bb), int(k),
                                        _ptr(e) if e is not None else None, float(m_dir), l,
                                        lam_d.ctypes.data if l else None, ptr(rr), ptr(ll), ptr(drr), ptr(dll),
                                        _ptr(dx), _ptr(x), ctypes.byref(info)), "ov_tsl_sign_jvp_deflated")
    if single:
        dx, x = dx[0], x[0]
    return (dx, x, info.as_dict()) if return_info else (dx, x)


def block_tsl_sign(u, mu, m_w, top, bottom, k, e=None, m_dir=0.0, precision="fp64", rebiorth=1, passes=2,
                   return_info=False):
    """Theorem 1 from a general block start: the halves of sgn(B) (top, bottom),
    B = [[H, dH], [0, H]]; top may be None (zero)."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    bb, single = _spinors(bottom, u)
    tt = None
    if top is not None:
        tt, single_t = _spinors(top, u)
        if tt.shape != bb.shape:
            raise ValueError("top and bottom must have the same shape")
    if e is not None:
        _dims(e)
        e = e.contiguous()
    zt = torch.empty_like(bb)
    zb = torch.empty_like(bb)
    info = Info()
    ctx = context(precision, rebiorth, passes)
    _check(lib.ov_block_tsl_sign(ctx, dims, _ptr(u), float(mu), float(m_w), bb.shape[0],
                                 _ptr(tt) if tt is not None else None, _ptr(bb), int(k),
                                 _ptr(e) if e is not None else None, float(m_dir), _ptr(zt), _ptr(zb),
                                 ctypes.byref(info)), "ov_block_tsl_sign")
    if single:
        zt, zb = zt[0], zb[0]
    return (zt, zb, info.as_dict()) if return_info else (zt, zb)


def tsl_eps(u, mu, m_w, b, k, precision="fp64", rebiorth=1, passes=2, segment=0):
    """eps_A = ||sgn(H)^2 b - b|| / (2 ||b||) per source (Sec. 4.1, Eq. error_est)."""
    import numpy as np
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    bb, single = _spinors(b, u)
    eps = np.zeros(bb.shape[0], dtype=np.float64)
    info = Info()
    ctx = context(precision, rebiorth, passes, segment=segment)
    _check(lib.ov_tsl_eps(ctx, dims, _ptr(u), float(mu), float(m_w), bb.shape[0], _ptr(bb), int(k),
                          eps.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info)), "ov_tsl_eps")
    return float(eps[0]) if single else eps


def block_tsl_eps(u, mu, m_w, b, k, e=None, m_dir=0.0, precision="fp64", rebiorth=1, passes=2):
    """eps_B = ||sgn(B)^2 (0, b) - (0, b)|| / (2 ||b||) per source (Sec. 4.1, Eq. bA_error_est)."""
    import numpy as np
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    bb, single = _spinors(b, u)
    if e is not None:
        _dims(e)
        e = e.contiguous()
    eps = np.zeros(bb.shape[0], dtype=np.float64)
    info = Info()
    ctx = context(precision, rebiorth, passes)
    _check(lib.ov_block_tsl_eps(ctx, dims, _ptr(u), float(mu), float(m_w), bb.shape[0], _ptr(bb), int(k),
                                _ptr(e) if e is not None else None, float(m_dir),
                                eps.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info)), "ov_block_tsl_eps")
    return float(eps[0]) if single else eps


def tsl_batch(problems, nworkers=4, precision="fp64", rebiorth=1, passes=2, check=True, segment=0):
    """Uneven batch: each problem is a dict with u, mu, m_w, b, k and optionally
    xbar (then the VJP is computed).  Returns one dict per problem with x and,
    with xbar, dU and dmu; plus info and status."""
    lib = load()
    n = len(problems)
    arr = (Problem * max(n, 1))()
    keep, outs = [], []
    for i, pr in enumerate(problems):
        u = pr["u"].contiguous()
        dims = _dims(u)
        bb, single = _spinors(pr["b"], u)
        xb = None
        if pr.get("xbar") is not None:
            xb, _ = _spinors(pr["xbar"], u)
            if xb.shape != bb.shape:
                raise ValueError("xbar must have the shape of b")
        x = torch.empty_like(bb)
        du = torch.empty_like(u) if xb is not None else None
        dmu = ctypes.c_double(0.0)
        p = arr[i]
        for d in range(4):
            p.dims[d] = dims[d]
        p.U, p.mu, p.m_w, p.nsrc = u.data_ptr(), float(pr["mu"]), float(pr["m_w"]), bb.shape[0]
        p.b, p.k = bb.data_ptr(), int(pr["k"])
        p.xbar = xb.data_ptr() if xb is not None else None
        p.x = x.data_ptr()
        p.dU = du.data_ptr() if du is not None else None
        p.dmu = ctypes.addressof(dmu) if xb is not None else None
        keep.append((u, bb, xb, dmu))
        outs.append((x, du, dmu, single))
    ctx = context(precision, rebiorth, passes, segment=segment)
    status = lib.ov_tsl_batch(ctx, n, arr, int(nworkers))
    res = []
    for i, (x, du, dmu, single) in enumerate(outs):
        r = {"x": x[0] if single else x, "status": arr[i].status, "info": arr[i].info.as_dict()}
        if du is not None:
            r["dU"], r["dmu"] = du, dmu.value
        res.append(r)
    if check:
        _check(status, "ov_tsl_batch")
    return res


def tsl_coefficients(k, src=0, precision="fp64", rebiorth=1, passes=2, segment=0):
    """(alpha, beta, delta) of the last TSL call on the matching context (host numpy)."""
    import numpy as np
    lib = load()
    ctx = context(precision, rebiorth, passes, segment=segment)
    a = np.zeros(k, dtype=np.complex128)
    b = np.zeros(k, dtype=np.complex128)
    d = np.zeros(k, dtype=np.float64)
    _check(lib.ov_tsl_coefficients(ctx, int(src), int(k), a.ctypes.data_as(ctypes.c_void_p),
                                   b.ctypes.data_as(ctypes.c_void_p), d.ctypes.data_as(ctypes.c_void_p)),
           "ov_tsl_coefficients")
    return a, b, d


def profile_enable(ctx, on=True):
    _check(load().ov_profile_enable(ctx, int(bool(on))), "ov_profile_enable")


def selftest_wait(limit_ns: int = 1_000_000):
    """Run the bounded-wait self-test; returns (status, device ms)."""
    ms = ctypes.c_double(0.0)
    st = load().ov_selftest_wait(context(), int(limit_ns), ctypes.byref(ms))
    return st, ms.value


def profile_select(ctx, kinds=None):
    """Time only the named kinds (None: all)."""
    mask = 0xFFFFFFFF if kinds is None else sum(1 << KINDS.index(k) for k in kinds)
    _check(load().ov_profile_select(ctx, mask), "ov_profile_select")


def profile_read(ctx, reset=False) -> dict:
    """{kind: (launches, device ms)} since the last reset."""
    lib = load()
    out = {}
    for i, name in enumerate(KINDS):
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0.0)
        _check(lib.ov_profile_read(ctx, i, ctypes.byref(n), ctypes.byref(ms), 0), "ov_profile_read")
        out[name] = (n.value, ms.value)
    if reset:
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0.0)
        _check(lib.ov_profile_read(ctx, 0, ctypes.byref(n), ctypes.byref(ms), 1), "ov_profile_read")
    return out


def launch_count(ctx) -> int:
    return int(load().ov_launch_count(ctx))


def autotune(u, mu, m_w, nsrc=1, precision="fp64", rebiorth=1, passes=2, segment=0) -> dict:
    """Time the stencil launch variants on this lattice and keep the fastest in the context."""
    lib = load()
    dims = _dims(u)
    u = u.contiguous()
    rep = TuneReport()
    ctx = context(precision, rebiorth, passes, segment=segment)
    _check(lib.ov_autotune(ctx, dims, _ptr(u), float(mu), float(m_w), int(nsrc), ctypes.byref(rep)),
           "ov_autotune")
    return {"apply_variant": rep.apply_variant, "pair_variant": rep.pair_variant,
            "apply_us": [round(v, 2) for v in rep.apply_us[:rep.n_apply]],
            "pair_us": [round(v, 2) for v in rep.pair_us[:rep.n_pair]]}


def set_stencil_variants(apply_variant, pair_variant, precision="fp64", rebiorth=1, passes=2):
    ctx = context(precision, rebiorth, passes)
    _check(load().ov_set_stencil_variants(ctx, int(apply_variant), int(pair_variant)), "ov_set_stencil_variants")
