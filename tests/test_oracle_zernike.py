"""Pins for the oracle's Zernike basis (Sec. 3.1) against facts the paper and
the mathematics fix: the paper's three-term radial recursion (a different
formula from the oracle's factorial closed form), R_n^m(1) = 1,
Z_n^0(0) = (-1)^(n/2) (Sec. 3.4), the orthogonality relation of Sec. 3.1 and
the parity Z(-p) = (-1)^n Z(p)."""
import numpy as np
import pytest


def radial_by_recursion(n, m, rho):
    """R_n^m = rho (R_{n-1}^{|m-1|} + R_{n-1}^{m+1}) - R_{n-2}^m, R_0^0 = 1 (Sec. 3.1)."""
    memo = {}

    def R(nn, mm):
        mm = abs(mm)
        if mm > nn or (nn - mm) % 2:
            return np.zeros_like(rho)
        if (nn, mm) in memo:
            return memo[(nn, mm)]
        if nn == 0:
            v = np.ones_like(rho)
        else:
            v = rho * (R(nn - 1, abs(mm - 1)) + R(nn - 1, mm + 1)) - R(nn - 2, mm)
        memo[(nn, mm)] = v
        return v

    return R(n, m)


@pytest.mark.parametrize("Np", [2, 4, 8])
def test_closed_form_matches_paper_recursion(oracle_mod, Np):
    rng = np.random.default_rng(10)
    rho = np.sqrt(rng.uniform(0, 1, 200))
    phi = rng.uniform(0, 2 * np.pi, 200)
    Z = oracle_mod.zernike(Np, rho * np.cos(phi), rho * np.sin(phi))
    for n, m in oracle_mod.zernike_nm(Np):
        R = radial_by_recursion(n, m, rho)
        ang = np.cos(m * phi) if m >= 0 else np.sin(-m * phi)
        np.testing.assert_allclose(Z[:, oracle_mod.zernike_index(n, m)], R * ang, atol=1e-12)


def test_radial_at_one_and_center(oracle_mod):
    Np = 10
    Z1 = oracle_mod.zernike(Np, [1.0], [0.0])[0]
    Z0 = oracle_mod.zernike(Np, [0.0], [0.0])[0]
    for n, m in oracle_mod.zernike_nm(Np):
        i = oracle_mod.zernike_index(n, m)
        if m >= 0:
            assert Z1[i] == pytest.approx(1.0, abs=1e-12)  # R_n^m(1) cos(0) = 1
        if m == 0:
            assert Z0[i] == pytest.approx((-1) ** (n // 2), abs=1e-12)
        else:
            assert abs(Z0[i]) < 1e-14


def test_orthogonality(oracle_mod):
    """Int Z_n^m Z_n'^m' rho drho dphi = eps_m pi/(2n+2) delta (Sec. 3.1):
    Gauss in u = rho^2 (the integrand is a polynomial in u times a trig
    polynomial) and a trapezoid rule in phi, both exact here."""
    Np = 8
    x, w = np.polynomial.legendre.leggauss(16)
    u = 0.5 * (x + 1)
    wu = 0.5 * w * 0.5  # rho drho = du/2
    K = 64
    phi = 2 * np.pi * np.arange(K) / K
    rho = np.sqrt(u)
    RR, PP = np.meshgrid(rho, phi, indexing="ij")
    W = np.outer(wu, np.full(K, 2 * np.pi / K))
    Z = oracle_mod.zernike(Np, (RR * np.cos(PP)).ravel(), (RR * np.sin(PP)).ravel())
    G = Z.T @ (Z * W.ravel()[:, None])
    expect = np.diag(1.0 / oracle_mod.zernike_invnorm(Np))
    np.testing.assert_allclose(G, expect, atol=1e-12)
    # the inverse norm of Sec. 3.2 is (2n+2)/(eps_m pi)
    for (n, m), N in zip(oracle_mod.zernike_nm(Np), oracle_mod.zernike_invnorm(Np)):
        assert N == pytest.approx((2 * n + 2) / ((2 if m == 0 else 1) * np.pi))


def test_parity(oracle_mod):
    rng = np.random.default_rng(3)
    p = rng.uniform(-0.7, 0.7, (50, 2))
    Np = 6
    Zp = oracle_mod.zernike(Np, p[:, 0], p[:, 1])
    Zm = oracle_mod.zernike(Np, -p[:, 0], -p[:, 1])
    sign = np.array([(-1) ** n for n, m in oracle_mod.zernike_nm(Np)])
    np.testing.assert_allclose(Zm, Zp * sign, atol=1e-13)


def test_closed_form_and_orthogonality_at_order_20(oracle_mod):
    """The orders of the cuboid verification (Sec. 4.1, up to N_p = 20): the
    closed form against the paper's recursion (its alternating sums lose about
    1e-10 near rho = 1 at n = 20) and the orthogonality relation, with Gauss in
    u = rho^2 exact to degree 47 and a 64-point trapezoid rule in phi exact for
    the angular products up to degree 40."""
    Np = 20
    rng = np.random.default_rng(20)
    rho = np.sqrt(rng.uniform(0, 1, 100))
    phi = rng.uniform(0, 2 * np.pi, 100)
    Z = oracle_mod.zernike(Np, rho * np.cos(phi), rho * np.sin(phi))
    for n, m in oracle_mod.zernike_nm(Np):
        R = radial_by_recursion(n, m, rho)
        ang = np.cos(m * phi) if m >= 0 else np.sin(-m * phi)
        np.testing.assert_allclose(Z[:, oracle_mod.zernike_index(n, m)], R * ang, atol=2e-9)
    x, w = np.polynomial.legendre.leggauss(24)
    u = 0.5 * (x + 1)
    wu = 0.5 * w * 0.5
    K = 64
    ph = 2 * np.pi * np.arange(K) / K
    RR, PP = np.meshgrid(np.sqrt(u), ph, indexing="ij")
    W = np.outer(wu, np.full(K, 2 * np.pi / K))
    Z = oracle_mod.zernike(Np, (RR * np.cos(PP)).ravel(), (RR * np.sin(PP)).ravel())
    G = Z.T @ (Z * W.ravel()[:, None])
    np.testing.assert_allclose(G, np.diag(1.0 / oracle_mod.zernike_invnorm(Np)), atol=1e-9)
