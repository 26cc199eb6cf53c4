"""Pins of the oracle's Euler physics: fluxes from primitives (Eq. euler1,
Eq. euler2), the Jacobian-vector products h, xi, eta, theta of Eq. EQ3
against central finite differences of the flux, and the eigen-systems used by
the local characteristic decomposition: L R = I, A R = R Lambda with A from
finite differences, and Roe's property F(U_R) - F(U_L) = A(U_Roe)(U_R - U_L)."""
import numpy as np
import pytest

import oracle as O

G = 1.4


def prob(dim, eig_avg=0):
    return O.problem(O.EQ_EULER, dim, 8, 8, gas_gamma=G, eig_avg=eig_avg)


def random_state(rng, dim):
    rho, p = rng.uniform(0.2, 3.0), rng.uniform(0.2, 5.0)
    u = rng.uniform(-2, 2, size=dim)
    E = p / (G - 1) + 0.5 * rho * np.sum(u * u)
    return np.array([rho, *(rho * u), E]), rho, u, p


@pytest.mark.parametrize("dim", [1, 2])
def test_flux_from_primitives(dim):
    rng = np.random.default_rng(1)
    P = prob(dim)
    for _ in range(20):
        U, rho, u, p = random_state(rng, dim)
        H = (U[-1] + p)
        for d in range(dim):
            ud = u[d]
            ref = [rho * ud] + [rho * ud * u[k] + (p if k == d else 0.0) for k in range(dim)] + [ud * H]
            assert np.allclose(O.flux(P, d, U), ref, rtol=1e-14, atol=1e-14)
        c = np.sqrt(G * p / rho)
        for d in range(dim):
            assert abs(O.wave_speed(P, d, U) - (abs(u[d]) + c)) < 1e-14 * (1 + c)


@pytest.mark.parametrize("dim", [1, 2])
def test_jvp_is_flux_derivative(dim):
    rng = np.random.default_rng(2)
    P = prob(dim)
    for _ in range(20):
        U = random_state(rng, dim)[0]
        D = rng.standard_normal(U.size)
        e = 1e-6
        for d in range(dim):
            fd = (O.flux(P, d, U + e * D) - O.flux(P, d, U - e * D)) / (2 * e)
            assert np.allclose(O.jvp(P, d, U, D), fd, rtol=1e-7, atol=1e-7)


def fd_jacobian(P, d, U):
    m, e = U.size, 1e-6
    A = np.zeros((m, m))
    for k in range(m):
        dU = np.zeros(m)
        dU[k] = e
        A[:, k] = (O.flux(P, d, U + dU) - O.flux(P, d, U - dU)) / (2 * e)
    return A


@pytest.mark.parametrize("dim", [1, 2])
def test_eigenvectors_at_a_state(dim):
    rng = np.random.default_rng(3)
    P = prob(dim)
    for _ in range(20):
        U = random_state(rng, dim)[0]
        for d in range(dim):
            R, L, lam = O.eigen(P, d, U)
            assert np.allclose(L @ R, np.eye(U.size), atol=1e-12)
            A = fd_jacobian(P, d, U)
            assert np.allclose(A @ R, R * lam, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("dim", [1, 2])
def test_roe_property(dim):
    """The Roe-averaged Jacobian R diag(lambda) L maps U_R - U_L onto
    F(U_R) - F(U_L) exactly (up to rounding)."""
    rng = np.random.default_rng(4)
    P = prob(dim, eig_avg=0)
    for _ in range(20):
        UL, UR = random_state(rng, dim)[0], random_state(rng, dim)[0]
        for d in range(dim):
            R, L, lam = O.eigen(P, d, UL, UR)
            assert np.allclose(L @ R, np.eye(UL.size), atol=1e-12)
            lhs = (R * lam) @ L @ (UR - UL)
            rhs = O.flux(P, d, UR) - O.flux(P, d, UL)
            assert np.allclose(lhs, rhs, rtol=1e-11, atol=1e-11 * np.max(np.abs(rhs)))


def test_arithmetic_mean_option():
    """eig_avg = 1 takes the eigenvectors at (U_L + U_R)/2."""
    rng = np.random.default_rng(5)
    P = prob(2, eig_avg=1)
    UL, UR = random_state(rng, 2)[0], random_state(rng, 2)[0]
    R, L, lam = O.eigen(P, 0, UL, UR)
    R2, L2, lam2 = O.eigen(P, 0, 0.5 * (UL + UR))
    assert np.allclose(R, R2, rtol=1e-13) and np.allclose(L, L2, rtol=1e-13)
