"""Pins for the oracle's reference-element tables (Sec. 3.3 nodal basis, Sec. 3.5 subcells)
against closed forms and a library routine."""
import math

import numpy as np
import pytest
import torch

from oracle.refelem import RefElement, gauss_legendre


@pytest.mark.parametrize("n", range(1, 9))
def test_nodes_match_library_gauss_legendre(n):
    x, w = gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x.astype(float), (xr + 1) / 2, atol=1e-15, rtol=0)
    assert np.allclose(w.astype(float), wr / 2, atol=1e-15, rtol=0)


@pytest.mark.parametrize("N", range(1, 7))
def test_quadrature_exact_to_degree_2N_plus_1(N):
    r = RefElement(N)
    for k in range(2 * N + 2):
        assert abs(float((r.w * r.x ** k).sum()) - 1.0 / (k + 1)) < 1e-15
    # one degree more is no longer exact
    k = 2 * N + 2
    assert abs(float((r.w * r.x ** k).sum()) - 1.0 / (k + 1)) > 1e-12


@pytest.mark.parametrize("N", range(1, 7))
def test_derivative_and_end_values_exact_on_polynomials(N):
    r = RefElement(N)
    for k in range(N + 1):
        f = r.x ** k
        df = k * r.x ** (k - 1) if k > 0 else torch.zeros_like(r.x)
        assert torch.allclose(r.D @ f, df, atol=1e-12 * (N + 1) ** 2, rtol=0)
        assert abs(float(r.e0 @ f) - (1.0 if k == 0 else 0.0)) < 1e-13
        assert abs(float(r.e1 @ f) - 1.0) < 1e-13
    # symmetry of the nodes, x_m = 1 - x_{N-m}
    assert torch.allclose(r.x, 1.0 - r.x.flip(0), atol=1e-15)


@pytest.mark.parametrize("N", range(1, 7))
def test_time_matrix_properties(N):
    """K1 1 = e0 (a constant in time solves the predictor with zero right-hand side), and K1 is
    the weak time derivative: sum_l K1[k,l] f(x_l) = f(1) e1[k] - int phi_k' f for f of degree <= N."""
    r = RefElement(N)
    ones = torch.ones(N + 1, dtype=torch.float64)
    assert torch.allclose(r.K1 @ ones, r.e0, atol=1e-13)
    for j in range(N + 1):
        f = r.x ** j
        # int_0^1 phi_k'(x) x^j dx computed with a finer rule
        xf, wf = gauss_legendre(N + 3)
        xf = torch.tensor(xf.astype(float))
        wf = torch.tensor(wf.astype(float))
        dphi = r.derivatives_at(xf.numpy())  # [nf, n]
        integ = (wf[:, None] * dphi * (xf ** j)[:, None]).sum(0)
        assert torch.allclose(r.K1 @ f, r.e1 * 1.0 - integ, atol=1e-12)


@pytest.mark.parametrize("N", range(1, 7))
def test_subcell_projection_and_reconstruction(N):
    r = RefElement(N)
    ns = 2 * N + 1
    assert r.P1.shape == (ns, N + 1)
    # P1 gives exact subcell averages of polynomials of degree <= N
    for k in range(N + 1):
        f = r.x ** k
        a = torch.arange(ns, dtype=torch.float64) / ns
        b = (torch.arange(ns, dtype=torch.float64) + 1) / ns
        exact = (b ** (k + 1) - a ** (k + 1)) / (k + 1) * ns
        assert torch.allclose(r.P1 @ f, exact, atol=1e-13)
    # R1 is a left inverse and preserves the mean
    assert torch.allclose(r.R1 @ r.P1, torch.eye(N + 1, dtype=torch.float64), atol=1e-12)
    assert torch.allclose(r.w @ r.R1, torch.full((ns,), 1.0 / ns, dtype=torch.float64), atol=1e-14)
    # rows of P1 average the basis: sum over nodes is one (partition of unity)
    assert torch.allclose(r.P1.sum(1), torch.ones(ns, dtype=torch.float64), atol=1e-14)
