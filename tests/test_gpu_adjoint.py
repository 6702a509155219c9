"""GPU reverse-time adjoint against the FP64 oracle adjoint and finite differences."""
import numpy as np
import pytest

from oracle.adjoint import HeatSequence as OracleSeq
from synthetic import Modes, forcing_basis_indices, adjoint_parameters

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_10863_gb300 import build as b
    b.build()
    import paper_2009_10863_gb300 as sgmod
    sgmod.lib()
    return sgmod


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def _modes_matrix(E, p, nparam, coords):
    idx = forcing_basis_indices(nparam)
    cx, cy, cz = coords
    Phi = np.stack([np.einsum('k,j,i->kji', np.sin(np.pi * c * cz), np.sin(np.pi * b * cy),
                              np.sin(np.pi * a * cx)).reshape(-1) for a, b, c in idx])
    return Phi


@pytest.mark.parametrize("K,ckpt,method", [(7, 3, "extrap"), (5, 10, "extrap"), (6, 2, "qr")])
def test_adjoint_matches_oracle(sg, K, ckpt, method):
    from paper_2009_10863_gb300.adjoint import HeatSequence
    E, p, lam = (2, 2, 2), 3, 30.0
    ors = OracleSeq(*E, p, lam, exact=True)
    rng = np.random.default_rng(K + ckpt)
    F = rng.standard_normal((K, ors.op.n)) * ors.m
    Xs = 1e-2 * rng.standard_normal((K, ors.op.n)) * ors.m
    L_o, dF_o, dl_o = ors.gradients(F, Xs)
    seq = HeatSequence(*E, p, tol=1e-13, s=4, m=2, method=method, checkpoint=ckpt)
    Fd, Xd = dev(F), dev(Xs)
    L, ck = seq.forward_loss(Fd, lam, Xd)
    dF, dlam = seq.adjoint(Fd, lam, Xd, ck)
    assert abs(float(L) - L_o) <= 1e-10 * abs(L_o)
    assert np.linalg.norm(host(dF) - dF_o) <= 1e-8 * np.linalg.norm(dF_o)
    assert abs(float(dlam) - dl_o) <= 1e-8 * abs(dl_o)


def test_autograd_theta_and_lambda_small(sg):
    """theta -> forcing (torch) -> SequenceLoss (library) -> backward: gradients
    w.r.t. the 64 forcing coefficients and lambda agree with the oracle adjoint."""
    from paper_2009_10863_gb300.adjoint import HeatSequence, SequenceLoss
    E, p, lam0, K, nparam, dt = (3, 3, 3), 3, 50.0, 8, 64, 0.01
    ors = OracleSeq(*E, p, lam0, exact=True)
    Phi = _modes_matrix(E, p, nparam, ors.op.coords_1d()) * ors.m
    theta_star, w = adjoint_parameters(5, nparam)
    t = dt * np.arange(1, K + 1)
    C = np.cos(np.outer(t, w))                         # K x nparam
    Xs = np.array(ors.forward((C * theta_star) @ Phi))
    theta0 = 0.5 * theta_star + 0.1
    F0 = (C * theta0) @ Phi
    L_o, dF_o, dl_o = ors.gradients(F0, Xs)
    dtheta_o = np.einsum('kj,kn,jn->j', C, dF_o, Phi)

    seq = HeatSequence(*E, p, tol=1e-13, s=6, m=2, checkpoint=3)
    theta = dev(theta0).requires_grad_(True)
    lam = torch.tensor(lam0, dtype=torch.float64, device="cuda", requires_grad=True)
    Fd = (dev(C) * theta) @ dev(Phi)
    L = SequenceLoss.apply(Fd, lam, dev(Xs), seq)
    L.backward()
    assert abs(float(L.detach()) - L_o) <= 1e-10 * L_o
    assert np.linalg.norm(host(theta.grad) - dtheta_o) <= 1e-8 * np.linalg.norm(dtheta_o)
    assert abs(float(lam.grad) - dl_o) <= 1e-8 * abs(dl_o)


def test_full_size_directional_finite_differences(sg):
    """16^3 elements, p = 7, lambda = 1e5, 64 forcing modes: the adjoint
    directional derivative matches central differences of the loss (h = 1e-6)
    in theta and in lambda."""
    from paper_2009_10863_gb300.adjoint import HeatSequence, SequenceLoss
    E, p, lam0, K, nparam, dt = (16, 16, 16), 7, 1e5, 12, 64, 1e-3
    seq = HeatSequence(*E, p, tol=1e-12, s=6, m=2, checkpoint=5)
    op = seq.op(lam0)
    coords = op.coords_1d()
    inner = [(c > 0) & (c < 1) for c in coords]
    interior = np.einsum('k,j,i->kji', inner[2], inner[1], inner[0]).reshape(-1).astype(np.float64)
    Phi = dev(_modes_matrix(E, p, nparam, coords) * interior)
    theta_star, w = adjoint_parameters(5, nparam)
    C = dev(np.cos(np.outer(dt * np.arange(1, K + 1), w)))
    Xs = torch.stack([dev(Modes(9, 8, 3).field(*coords, dt * k) * interior * 1e-6) for k in range(1, K + 1)])
    theta = dev(theta_star + 0.3).requires_grad_(True)
    lam = torch.tensor(lam0, dtype=torch.float64, device="cuda", requires_grad=True)
    L = SequenceLoss.apply((C * theta) @ Phi, lam, Xs, seq)
    L.backward()
    rng = np.random.default_rng(1)
    d = dev(rng.standard_normal(nparam))
    h = 1e-6
    with torch.no_grad():
        Lp = SequenceLoss.apply((C * (theta + h * d)) @ Phi, lam, Xs, seq)
        Lm = SequenceLoss.apply((C * (theta - h * d)) @ Phi, lam, Xs, seq)
    fd = float(Lp - Lm) / (2 * h)
    ad = float(theta.grad @ d)
    assert abs(fd - ad) <= 1e-5 * abs(ad)
    hl = 1e-6 * lam0
    with torch.no_grad():
        Lp = SequenceLoss.apply((C * theta) @ Phi, lam0 + hl, Xs, seq)
        Lm = SequenceLoss.apply((C * theta) @ Phi, lam0 - hl, Xs, seq)
    fdl = float(Lp - Lm) / (2 * hl)
    assert abs(fdl - float(lam.grad)) <= 1e-4 * abs(float(lam.grad))
