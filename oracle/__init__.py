"""FP64 CPU oracle for the two-sided Lanczos sign function and its gauge-force VJP.

TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may import,
call or execute anything in this package; only ``tests/``, the smoke check in
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It shares no code with the CUDA path: it takes plain numpy arrays (built by the
seeded generators in ``paper_1604_08057_gb300.inputs``, which contain none of
the method's arithmetic) and returns plain numpy arrays.

Everything here is plain, slow and written to be checked against the paper by
eye: numpy complex128 throughout, library primitives (einsum, LU, matmul) as
single steps, no blocking, fusion or reordering.

Modules
-------
dirac   Wilson-Dirac operator D_w(mu), H = gamma5 D_w, H^dagger, dH/dmu and the
        link-gradient contraction (App. A, Eqs. WD_op, WD_G, dWD_op).
ksign   k x k matrix sign by scaled Newton iteration and its Frechet adjoint by
        Newton on the Theorem-1 block matrix (Sec. 2, Theorem 1).
tsl     Two-sided Lanczos approximation x ~ sgn(H) b (Sec. 1 and 2, the TSL of
        Bloch et al.), with optional re-biorthogonalisation.
vjp     Reverse-mode derivative of the TSL map with respect to all links and mu.
nested  Nested Krylov approximation of the k x k sign, one nesting level
        (Sec. 4.1): Arnoldi on S = (T_k + T_k^{-1})/2 from e_1.

Pins: every function is checked in ``tests/test_oracle_*.py`` against facts
that do not come from the oracle itself (closed forms in momentum space,
eigendecomposition sign, sgn^2 = 1, gamma5-hermiticity, gauge covariance,
Daleckii-Krein, central finite differences, autograd through a dense
restatement).
"""
from . import dirac, ksign, nested, tsl, vjp  # noqa: F401
