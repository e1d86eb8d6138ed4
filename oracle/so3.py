"""O(3) pieces of the FP64 oracle: real spherical harmonics and coupling tensors.

TEST INFRASTRUCTURE.  Only tests/, the smoke check and the benchmark's CPU-baseline leg
may import this package; the CUDA path never does.

Allegro-FM builds on e3nn irreps "with l = 2 in full O(3) symmetry" (Methodology, Model
Training).  The paper prints no basis, so this module fixes one (a reading):
  * real spherical harmonics of the unit vector with component normalisation
    (sum_m Y_lm^2 = 2l+1), m ordered -l..l:  Y_1 = sqrt(3)(y, z, x),
    Y_2 = (sqrt15 xy, sqrt15 yz, sqrt5/2 (3z^2-1), sqrt15 xz, sqrt15/2 (x^2-y^2));
  * coupling tensors C^{l1 l2 l3}: the unique (up to sign) rotation-invariant tensor in
    the real basis, scaled to sum C^2 = 2 l3 + 1 ("component" normalisation), sign fixed
    so that its first non-zero entry in (m1, m2, m3) lexicographic order is positive.
The coupling tensors are computed here from first principles: the Wigner matrices D_l(R)
are fitted from the harmonics at rotated points, and C is the null space of the
invariance constraint (D1 x D2 x D3 - 1) vec C = 0 over several random rotations.
"""
from __future__ import annotations

import functools
import math

import numpy as np

S3 = math.sqrt(3.0)
S5 = math.sqrt(5.0)
S15 = math.sqrt(15.0)


def sh(l: int, u: np.ndarray) -> np.ndarray:
    """Real, component-normalised spherical harmonics Y_l of unit vectors u[..., 3]."""
    x, y, z = u[..., 0], u[..., 1], u[..., 2]
    if l == 0:
        return np.ones(u.shape[:-1] + (1,))
    if l == 1:
        return S3 * np.stack([y, z, x], axis=-1)
    if l == 2:
        return np.stack([S15 * x * y, S15 * y * z, 0.5 * S5 * (3.0 * z * z - 1.0),
                         S15 * x * z, 0.5 * S15 * (x * x - y * y)], axis=-1)
    raise ValueError("l <= 2 only")


def sh_grad_u(l: int, u: np.ndarray) -> np.ndarray:
    """d Y_l / d u (the polynomial's gradient), shape [..., 2l+1, 3]."""
    x, y, z = u[..., 0], u[..., 1], u[..., 2]
    zero = np.zeros_like(x)
    if l == 0:
        return np.zeros(u.shape[:-1] + (1, 3))
    if l == 1:
        one = np.ones_like(x)
        rows = [[zero, one, zero], [zero, zero, one], [one, zero, zero]]
        return S3 * np.stack([np.stack(r, axis=-1) for r in rows], axis=-2)
    if l == 2:
        rows = [[S15 * y, S15 * x, zero],
                [zero, S15 * z, S15 * y],
                [zero, zero, 3.0 * S5 * z],
                [S15 * z, zero, S15 * x],
                [S15 * x, -S15 * y, zero]]
        return np.stack([np.stack(r, axis=-1) for r in rows], axis=-2)
    raise ValueError("l <= 2 only")


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random proper rotation (QR of a Gaussian matrix, sign-fixed)."""
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def wigner_d(l: int, R: np.ndarray, n_pts: int = 64, seed: int = 0) -> np.ndarray:
    """D_l(R) with Y_l(R u) = D_l(R) Y_l(u), fitted by least squares over sample points."""
    rng = np.random.default_rng(seed + 17 * l)
    u = rng.normal(size=(n_pts, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    Y = sh(l, u)                    # [n, 2l+1]
    YR = sh(l, u @ R.T)             # [n, 2l+1]
    Dt, *_ = np.linalg.lstsq(Y, YR, rcond=None)
    return Dt.T


@functools.lru_cache(maxsize=None)
def coupling(l1: int, l2: int, l3: int) -> np.ndarray:
    """Real coupling tensor C[m1, m2, m3] (see module docstring for the conventions)."""
    if not (abs(l1 - l2) <= l3 <= l1 + l2):
        raise ValueError("triangle rule violated")
    rng = np.random.default_rng(1234 + 100 * l1 + 10 * l2 + l3)
    n = (2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1)
    rows = []
    for _ in range(4):
        R = random_rotation(rng)
        K = np.kron(np.kron(wigner_d(l1, R), wigner_d(l2, R)), wigner_d(l3, R))
        rows.append(K - np.eye(n))
    A = np.concatenate(rows, axis=0)
    _, sv, vt = np.linalg.svd(A)
    # one-dimensional null space: the smallest singular value vanishes, the next does not
    assert sv[-1] < 1e-9 and (n == 1 or sv[-2] > 1e-3), (l1, l2, l3, sv[-3:])
    c = vt[-1]
    c[np.abs(c) < 1e-13] = 0.0
    c *= math.sqrt(2 * l3 + 1) / np.linalg.norm(c)
    first = c[np.nonzero(np.abs(c) > 1e-9)[0][0]]
    if first < 0:
        c = -c
    return c.reshape(2 * l1 + 1, 2 * l2 + 1, 2 * l3 + 1)


# ---------------------------------------------------------------------------------------
# Irreps and tensor-product paths (the "full O(3)" reading of the paper's l = 2 model).
# An irrep is (l, p) with p = +1 (even) or -1 (odd).  Canonical order: by l, and for each
# l the natural parity (-1)^l first.
# ---------------------------------------------------------------------------------------

def canonical(irreps):
    return sorted(set(irreps), key=lambda ir: (ir[0], 0 if ir[1] == (-1) ** ir[0] else 1))


def natural_irreps(lmax: int):
    return [(l, (-1) ** l) for l in range(lmax + 1)]


def layer_paths(in_irreps, lmax: int, last: bool):
    """Paths (l1,p1) x (l2,(-1)^l2) -> (l3, p1*(-1)^l2) of one layer, in canonical order.

    For the last layer only scalar (0e) outputs are kept; otherwise every l3 <= lmax.
    Returns (paths, out_irreps) with paths as tuples (i_in, l2, (l3, p3)).
    """
    paths = []
    for i_in, (l1, p1) in enumerate(in_irreps):
        for l2 in range(lmax + 1):
            p2 = (-1) ** l2
            for l3 in range(abs(l1 - l2), min(l1 + l2, lmax) + 1):
                out = (l3, p1 * p2)
                if last and out != (0, 1):
                    continue
                paths.append((i_in, l2, out))
    outs = canonical([p[2] for p in paths])
    return paths, outs


def model_paths(lmax: int, n_layers: int):
    """Per layer L = 1..n_layers: (in_irreps, paths, out_irreps)."""
    layers = []
    irr = natural_irreps(lmax)
    for L in range(1, n_layers + 1):
        paths, outs = layer_paths(irr, lmax, last=(L == n_layers))
        layers.append((list(irr), paths, outs))
        irr = outs
    return layers
