"""Pins of the contour form for a non-Stieltjes f (Algorithm 2 with a fixed
contour; the parabola of Sec. 5.2), f(z) = e^{-z}: the rule reproduces the
scalar function on points the contour encloses, the approximants built with
it are exact on invariant Krylov spaces and converge to expm(-A) b, and the
sFOM quadrature form equals the closed form exp(-M)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import quadrature as oq
from oracle import sketched as osk
from oracle.arnoldi import arnoldi_trunc
from oracle.exact import fAb_dense
from oracle.sketch import Sketch


def test_contour_rule_reproduces_exp_on_real_points():
    t, w = oq.rule("exp_neg", 128, 0.25, alpha=0.5)
    for z in np.linspace(0.1, 20.0, 40):
        val = np.sum(w / (t + z)).real
        assert abs(val - math.exp(-z)) <= 1e-12 * max(1.0, math.exp(-z)) + 1e-15


def test_contour_rule_reproduces_exp_on_complex_pairs():
    """For a real operator the eigenvalues come in conjugate pairs; the
    half-rule's real part then gives f at the pair: Re sum w/(t+z) summed over
    z and conj(z) equals e^{-z} + e^{-conj z} = 2 Re e^{-z}."""
    t, w = oq.rule("exp_neg", 256, 0.05, alpha=0.0)
    for z in [0.5 + 1.0j, 2.0 + 3.0j, 5.0 - 2.5j]:
        # -z and -conj(z) lie left of the parabola: Re(-z) < -0.05 Im(z)^2
        assert -z.real < -0.05 * z.imag ** 2
        half = (np.sum(w / (t + z)) + np.sum(w / (t + np.conj(z)))).real
        assert abs(half - 2 * np.exp(-z).real) <= 1e-10


def test_contour_approximants_exact_on_invariant_space():
    """A with 5 distinct eigenvalues: K_5(A, b) is invariant, so sFOM and
    sGMRES give expm(-A) b up to the rule's error (S = sparse sign)."""
    rng = np.random.default_rng(2)
    lam = np.array([0.3, 0.9, 1.7, 2.5, 4.0])
    X = rng.standard_normal((40, 40))
    D = np.repeat(lam, 8)
    A = X @ np.diag(D) @ np.linalg.inv(X)
    b = rng.standard_normal(40)
    S = Sketch("sparse_sign", 40, 30, 4, 7)
    ref = sla.expm(-A) @ b
    for method in ("sgmres", "sfom_quad", "sfom"):
        x, info = osk.solve(A, b, "exp_neg", 5, 5, S, 0.2, method=method, ell=160, alpha=0.2)
        assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_contour_sgmres_converges_to_expm_on_convection_diffusion():
    from workloads import convdiff_2d, csr_to_scipy
    A = convdiff_2d(12, (20.0, 10.0))
    As = csr_to_scipy(A) / 50.0            # real spectrum in [3.27, 23.8]
    b = np.ones(A.n) / math.sqrt(A.n)
    ref = fAb_dense(As.toarray(), b, "exp_neg")
    S = Sketch("sparse_sign", A.n, 160, 8, 13)
    errs = []
    for m in (5, 10, 30):
        x, _ = osk.solve(As, b, "exp_neg", m, 2, S, 0.1, method="sgmres", ell=64, alpha=0.5)
        errs.append(np.linalg.norm(x - ref) / np.linalg.norm(ref))
    assert errs[2] < 1e-10 and errs[2] < 1e-6 * errs[0]
    # sFOM by quadrature equals the closed form exp(-M) c on the same sketches
    ar = arnoldi_trunc(As, b, 20, 2, S)
    W = osk.whiten(ar["SV"], ar["SAV"], S @ b)
    yq, _ = osk.sfom_quadrature(W, "exp_neg", 0.1, ell=64, alpha=0.5)
    yc = osk.sfom_closed(W, "exp_neg")
    assert np.linalg.norm(ar["V"] @ (yq - yc)) <= 1e-10 * np.linalg.norm(ar["V"] @ yc)
