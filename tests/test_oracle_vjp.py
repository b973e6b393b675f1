"""Pins for the oracle's gauge-force VJP of the TSL map (generalising App. A, Eq. dWD_op).

Independent checks: central finite differences of the oracle's own forward
map, and torch autograd through a dense restatement of H and the TSL.
"""
import numpy as np
import pytest

from oracle import dirac, tsl, vjp
from paper_1604_08057_gb300 import inputs


def _setup(dims, eps, seed):
    rng = np.random.default_rng(seed)
    u = inputs.su3_links(dims, eps, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    xbar = inputs.gaussian_spinors(dims, 1, rng)[0]
    return u, b, xbar, rng


@pytest.mark.parametrize("k,rebiorth", [(40, 1), (100, 1), (60, 10)])
def test_vjp_central_differences(k, rebiorth):
    dims = (3, 3, 3, 3)
    u, b, xbar, rng = _setup(dims, 0.3, 41)
    mu, m_w = 0.3, -2.0
    du, dmu, _ = vjp.tsl_vjp(u, b, mu, m_w, k, xbar, rebiorth=rebiorth)

    def loss(uu, mm):
        return np.real(np.vdot(xbar, tsl.tsl_forward(uu, b, mm, m_w, k, rebiorth=rebiorth).x))

    h = 1e-6
    for _ in range(2):
        e = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
        fd = (loss(u + h * e, mu) - loss(u - h * e, mu)) / (2 * h)
        assert abs(fd - np.real(np.vdot(du, e))) <= 2e-7 * abs(fd)
    fd_mu = (loss(u, mu + h) - loss(u, mu - h)) / (2 * h)
    assert abs(fd_mu - dmu) <= 2e-7 * abs(fd_mu)


def test_vjp_matches_torch_autograd_dense():
    """Autograd through a dense restatement (H as a matrix, TSL with projections in the graph)."""
    torch = pytest.importorskip("torch")
    dims = (2, 2, 2, 3)
    u, b, xbar, _ = _setup(dims, 0.4, 42)
    mu, m_w, k = 0.3, -2.0, 60
    du, dmu, _ = vjp.tsl_vjp(u, b, mu, m_w, k, xbar, rebiorth=1)

    shape = inputs.lattice_shape(dims)
    vol = int(np.prod(shape))
    kappa = 1.0 / (2 * m_w + 8)
    g5 = torch.tensor(dirac.GAMMA5)
    eye4 = torch.eye(4, dtype=torch.complex128)

    def site(c):
        t, z, y, x = c
        return ((t * shape[1] + z) * shape[2] + y) * shape[3] + x

    def dense_h(ut, mut):
        # H = gamma5 D_w as a (12V x 12V) matrix assembled block by block
        blocks = [[None] * vol for _ in range(vol)]
        zero = torch.zeros(12, 12, dtype=torch.complex128)
        idx = np.ndindex(*shape)
        rows = {}
        for c in idx:
            xs = site(c)
            acc = {xs: torch.eye(12, dtype=torch.complex128)}
            for nu in range(4):
                ax = 3 - nu
                cp = list(c); cp[ax] = (cp[ax] + 1) % shape[ax]
                cm = list(c); cm[ax] = (cm[ax] - 1) % shape[ax]
                f = torch.exp(mut) if nu == 3 else torch.tensor(1.0, dtype=torch.float64)
                gp = torch.kron(eye4 + torch.tensor(dirac.GAMMA[nu]), ut[tuple(c) + (nu,)].contiguous())
                gm = torch.kron(eye4 - torch.tensor(dirac.GAMMA[nu]),
                                ut[tuple(cm) + (nu,)].conj().T.contiguous())
                yp, ym = site(cp), site(cm)
                acc[yp] = acc.get(yp, zero) - kappa * f * gp
                acc[ym] = acc.get(ym, zero) - kappa / f * gm
            rows[xs] = acc
        for xs in range(vol):
            for ys in range(vol):
                blocks[xs][ys] = rows[xs].get(ys, zero)
        d = torch.cat([torch.cat(r, 1) for r in blocks], 0)
        return torch.kron(torch.eye(vol, dtype=torch.complex128),
                          torch.kron(g5, torch.eye(3, dtype=torch.complex128))) @ d

    def sign_newton_t(a):
        x = a
        for _ in range(60):
            x = 0.5 * (x + torch.linalg.inv(x))
        return x

    ut = torch.tensor(u, requires_grad=True)
    mut = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    h = dense_h(ut, mut)
    bt = torch.tensor(b.ravel())
    b0 = torch.linalg.vector_norm(bt)
    v = [bt / b0]
    w = [bt / b0]
    al, be, de = [], [], []
    for j in range(k):
        p = h @ v[j]
        a = torch.vdot(w[j], p)
        al.append(a)
        if j == k - 1:
            break
        q = h.conj().T @ w[j]
        r = p - a * v[j] - (be[-1] * v[j - 1] if j else 0)
        s = q - a.conj() * w[j] - (de[-1] * w[j - 1] if j else 0)
        vm, wm = torch.stack(v, 1), torch.stack(w, 1)
        for _ in range(2):
            r, s = r - vm @ (wm.conj().T @ r), s - wm @ (vm.conj().T @ s)
        om = torch.vdot(s, r)
        dd = torch.sqrt(om.abs())
        bb = om / dd
        de.append(dd.to(torch.complex128))
        be.append(bb)
        v.append(r / dd)
        w.append(s / bb.conj())
    t = torch.diag(torch.stack(al)) + torch.diag(torch.stack(be), 1) + torch.diag(torch.stack(de), -1)
    y = b0 * sign_newton_t(t)[:, 0]
    x = torch.stack(v, 1) @ y
    loss = torch.real(torch.vdot(torch.tensor(xbar.ravel()), x))
    loss.backward()
    gu = ut.grad.numpy()
    assert np.linalg.norm(gu - du) <= 1e-8 * np.linalg.norm(du)
    assert abs(mut.grad.item() - dmu) <= 1e-8 * abs(dmu)


def test_vjp_fp32_emulation_is_at_the_fp32_level():
    """The FP32-vector emulation rounds the reverse sweep as well as the forward one:
    at a well-conditioned point its gradient differs from the FP64 gradient by
    roughly the FP32 rounding unit (6e-8) times a modest amplification -- neither
    zero (nothing rounded) nor O(1) (a dropped term)."""
    dims = (3, 3, 3, 3)
    u, b, xbar, _ = _setup(dims, 0.3, 43)
    mu, m_w, k = 0.3, -1.0, 40
    du, dmu, fwd = vjp.tsl_vjp(u, b, mu, m_w, k, xbar)
    du32, dmu32, fwd32 = vjp.tsl_vjp(u, b, mu, m_w, k, xbar, emulate_fp32=True)
    rel_x = np.linalg.norm(fwd32.x - fwd.x) / np.linalg.norm(fwd.x)
    rel_du = np.linalg.norm(du32 - du) / np.linalg.norm(du)
    assert 1e-9 < rel_x < 1e-5, rel_x
    assert 1e-9 < rel_du < 1e-4, rel_du
    assert abs(dmu32 - dmu) < 1e-4 * abs(dmu)
    # the reverse sweep itself is rounded: the same FP32 forward with an FP64 reverse
    # sweep gives a different gradient
    du_mixed, _, _ = vjp.tsl_vjp(u, b, mu, m_w, k, xbar, fwd=fwd32)
    assert np.linalg.norm(du_mixed - du32) > 1e-10 * np.linalg.norm(du)
