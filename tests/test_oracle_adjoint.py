"""Pins for the oracle's reverse-time adjoint (CPU only).

With exact (dense Cholesky) solves on a tiny mesh the loss is a quadratic in
the forcing and smooth in lambda, so central finite differences are exact up
to rounding: they pin dL/dF and dL/dlam independently of the adjoint algebra.
"""
import numpy as np
import pytest

from oracle.adjoint import HeatSequence
from oracle.sem import SemOperator


def _setup(K=6, seed=0, lam=30.0):
    hs = HeatSequence(2, 2, 2, 3, lam, exact=True)
    rng = np.random.default_rng(seed)
    n = hs.op.n
    F = rng.standard_normal((K, n)) * hs.m
    Xs = rng.standard_normal((K, n)) * hs.m * 1e-2
    return hs, F, Xs, rng


def test_mass_integrates_constants():
    op1, op0 = SemOperator(3, 2, 2, 4, 1.0), SemOperator(3, 2, 2, 4, 0.0)
    ones = np.ones(op1.n)
    m1 = op1.apply(ones, mask=False) - op0.apply(ones, mask=False)
    assert abs(m1.sum() - 1.0) < 1e-13          # volume of the unit box


def test_adjoint_matches_central_differences_in_forcing():
    hs, F, Xs, rng = _setup()
    L, dF, _ = hs.gradients(F, Xs)
    D = rng.standard_normal(F.shape) * hs.m
    h = 1e-3
    fd = (hs.loss(F + h * D, Xs) - hs.loss(F - h * D, Xs)) / (2 * h)
    assert abs(fd - np.sum(dF * D)) <= 1e-9 * abs(fd)
    assert L == pytest.approx(hs.loss(F, Xs), rel=1e-14)


def test_adjoint_matches_central_differences_in_lambda():
    hs, F, Xs, _ = _setup(lam=30.0)
    _, _, dlam = hs.gradients(F, Xs)
    h = 1e-4
    lp = HeatSequence(2, 2, 2, 3, 30.0 + h, exact=True).loss(F, Xs)
    lm = HeatSequence(2, 2, 2, 3, 30.0 - h, exact=True).loss(F, Xs)
    fd = (lp - lm) / (2 * h)
    assert abs(fd - dlam) <= 1e-6 * abs(fd)


def test_pcg_and_exact_adjoints_agree():
    hs, F, Xs, _ = _setup(K=4, seed=3)
    hp = HeatSequence(2, 2, 2, 3, 30.0, tol=1e-13)
    _, dF1, dl1 = hs.gradients(F, Xs)
    _, dF2, dl2 = hp.gradients(F, Xs)
    assert np.linalg.norm(dF1 - dF2) <= 1e-10 * np.linalg.norm(dF1)
    assert abs(dl1 - dl2) <= 1e-10 * abs(dl1)
