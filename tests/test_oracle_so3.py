"""Pins of the oracle's spherical harmonics, Wigner matrices and coupling tensors.

Everything here is fixed by mathematics, not by the oracle's own formulas: quadrature
orthonormality, the addition theorem (against scipy's Legendre polynomials), the closed
form of D_1, group homomorphism, and the closed-form coupling tensors of the simplest
paths (identity, dot product, cross product).
"""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import so3


def _sphere_quadrature(n_theta=8, n_phi=16):
    x, w = np.polynomial.legendre.leggauss(n_theta)
    phi = 2 * np.pi * np.arange(n_phi) / n_phi
    ct = np.repeat(x, n_phi)
    wt = np.repeat(w, n_phi) * (2 * np.pi / n_phi)
    ph = np.tile(phi, n_theta)
    st = np.sqrt(1 - ct ** 2)
    u = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    return u, wt


def _rand_units(n, seed):
    u = np.random.default_rng(seed).normal(size=(n, 3))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_sh_component_normalisation(l):
    u = _rand_units(100, l)
    np.testing.assert_allclose((so3.sh(l, u) ** 2).sum(axis=1), 2 * l + 1, rtol=1e-13)


def test_sh_orthonormal_by_quadrature():
    u, w = _sphere_quadrature()
    Y = np.concatenate([so3.sh(l, u) for l in range(3)], axis=1)   # [N, 9]
    gram = (Y * w[:, None]).T @ Y / (4 * np.pi)
    np.testing.assert_allclose(gram, np.eye(9), atol=1e-13)


@pytest.mark.parametrize("l", [1, 2])
def test_sh_addition_theorem(l):
    a, b = _rand_units(50, 1), _rand_units(50, 2)
    lhs = (so3.sh(l, a) * so3.sh(l, b)).sum(axis=1)
    rhs = (2 * l + 1) * eval_legendre(l, (a * b).sum(axis=1))
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_sh_parity(l):
    u = _rand_units(20, 3)
    np.testing.assert_allclose(so3.sh(l, -u), (-1) ** l * so3.sh(l, u), atol=1e-14)


@pytest.mark.parametrize("l", [1, 2])
def test_sh_gradient_tangential_fd(l):
    u = _rand_units(10, 4)
    G = so3.sh_grad_u(l, u)
    h = 1e-6
    for k in range(3):
        t = np.random.default_rng(k).normal(size=(10, 3))
        t -= (t * u).sum(1, keepdims=True) * u                      # tangent direction
        up = u + h * t
        um = u - h * t
        up /= np.linalg.norm(up, axis=1, keepdims=True)
        um /= np.linalg.norm(um, axis=1, keepdims=True)
        fd = (so3.sh(l, up) - so3.sh(l, um)) / (2 * h)
        an = np.einsum("nmk,nk->nm", G, t)
        np.testing.assert_allclose(an, fd, atol=1e-7)


def test_wigner_d1_closed_form_and_homomorphism():
    rng = np.random.default_rng(5)
    P = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], dtype=float)   # (x,y,z) -> (y,z,x)
    for _ in range(3):
        R1, R2 = so3.random_rotation(rng), so3.random_rotation(rng)
        np.testing.assert_allclose(so3.wigner_d(1, R1), P @ R1 @ P.T, atol=1e-12)
        for l in range(3):
            D1, D2 = so3.wigner_d(l, R1), so3.wigner_d(l, R2)
            np.testing.assert_allclose(so3.wigner_d(l, R1 @ R2), D1 @ D2, atol=1e-12)
            np.testing.assert_allclose(D1 @ D1.T, np.eye(2 * l + 1), atol=1e-12)


TRIPLES = [(l1, l2, l3) for l1 in range(3) for l2 in range(3)
           for l3 in range(abs(l1 - l2), min(l1 + l2, 2) + 1)]


@pytest.mark.parametrize("l1,l2,l3", TRIPLES)
def test_coupling_equivariance_fresh_rotations(l1, l2, l3):
    C = so3.coupling(l1, l2, l3)
    rng = np.random.default_rng(99)
    for _ in range(3):
        R = so3.random_rotation(rng)
        D1, D2, D3 = (so3.wigner_d(l, R, seed=7) for l in (l1, l2, l3))
        a, b = rng.normal(size=2 * l1 + 1), rng.normal(size=2 * l2 + 1)
        lhs = np.einsum("ijk,i,j->k", C, D1 @ a, D2 @ b)
        rhs = D3 @ np.einsum("ijk,i,j->k", C, a, b)
        np.testing.assert_allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_coupling_special_cases(l):
    n = 2 * l + 1
    np.testing.assert_allclose(so3.coupling(l, 0, l)[:, 0, :], np.eye(n), atol=1e-12)
    np.testing.assert_allclose(so3.coupling(0, l, l)[0, :, :], np.eye(n), atol=1e-12)
    np.testing.assert_allclose(so3.coupling(l, l, 0)[:, :, 0], np.eye(n) / math.sqrt(n),
                               atol=1e-12)


def test_coupling_cross_product_and_symmetric_traceless():
    eps = np.zeros((3, 3, 3))
    for (a, b, c), s in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1,
                         (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}.items():
        eps[a, b, c] = s
    np.testing.assert_allclose(so3.coupling(1, 1, 1), eps / math.sqrt(2), atol=1e-12)
    C = so3.coupling(1, 1, 2)
    np.testing.assert_allclose(C, C.transpose(1, 0, 2), atol=1e-12)
    np.testing.assert_allclose(np.einsum("mmk->k", C), 0, atol=1e-12)


@pytest.mark.parametrize("l1,l2", [(1, 1), (1, 2), (2, 2), (2, 1)])
def test_coupling_orthogonality(l1, l2):
    cols = []
    for l3 in range(abs(l1 - l2), l1 + l2 + 1):
        if l3 > 2:
            continue
        C = so3.coupling(l1, l2, l3)
        cols.append(C.reshape(-1, 2 * l3 + 1))
    M = np.concatenate(cols, axis=1)
    np.testing.assert_allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-12)


def test_path_tables():
    layers = so3.model_paths(2, 3)
    assert [len(p) for _, p, _ in layers] == [15, 27, 3]
    assert layers[0][2] == [(0, 1), (1, -1), (1, 1), (2, 1), (2, -1)]
    assert layers[1][2] == [(0, 1), (0, -1), (1, -1), (1, 1), (2, 1), (2, -1)]
    for irr_in, paths, outs in layers:
        for i_in, l2, out in paths:
            l1, p1 = irr_in[i_in]
            assert abs(l1 - l2) <= out[0] <= l1 + l2
            assert out[1] == p1 * (-1) ** l2
    small = so3.model_paths(1, 2)
    assert [len(p) for _, p, _ in small] == [5, 2]
