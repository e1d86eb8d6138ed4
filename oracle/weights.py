"""Seeded random-init weights of the FP64 oracle (SplitMix64, unit-variance uniform).

TEST INFRASTRUCTURE (see oracle/__init__.py).

Allegro-FM initialises all MLPs from "a uniform distribution of unit variance"
(Methodology, Model Training): U(-sqrt3, sqrt3).  The random stream is SplitMix64
(Steele, Lea & Flood, OOPSLA 2014; the constants of Vigna's reference splitmix64.c),
used as a counter-based generator:

    out(s, n) = mix(s + n * GAMMA)            (the n-th output of a stream seeded with s)
    key_t     = out(seed, t + 1)              (stream of tensor t)
    bits      = out(key_t, k + 1)             (element k of tensor t)
    w         = sqrt(3) * (2 * (bits >> 11) * 2^-53 - 1)

All arithmetic is modulo 2^64.
"""
from __future__ import annotations

import math

import numpy as np

from . import so3

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK = (1 << 64) - 1
N_SPECIES = 89


def mix(z):
    """SplitMix64 output function on numpy uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
    return z ^ (z >> np.uint64(31))


def stream(seed: int, n: int) -> np.ndarray:
    """First n outputs of SplitMix64 seeded with `seed`."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = np.uint64(seed & MASK) + k * np.uint64(GAMMA)
    return mix(s)


def tensor_uniform(seed: int, t: int, n: int) -> np.ndarray:
    key = int(stream(seed, t + 1)[-1])
    bits = stream(key, n)
    u = (bits >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return math.sqrt(3.0) * (2.0 * u - 1.0)


def param_shapes(hp: dict):
    """Ordered list of (name, shape) of every weight tensor; the order fixes tensor ids.

    two-body MLP  W2b.k   [fan_in, width]     fan_in_0 = 2*89 + n_basis (one-hot Z_i,
                                              one-hot Z_j, radial basis)
    per layer L   Wenv.L  [D, (lmax+1)*C]     column = l*C + c
                  theta.L [n_paths_L, C]      (layers L < n_layers only)
                  Wlat.L.k [fan_in, width]    fan_in_0 = D + (lmax+1)*C, input [x || s],
                                              s index = k_path*C + c
    edge energy   We.k    [fan_in, width]     last width 1
    Each matrix is row-major [in][out] and is applied as x @ W / sqrt(fan_in).
    """
    C = hp["channels"]
    lmax = hp["lmax"]
    D = hp["two_body"][-1]
    out = []
    fan = 2 * N_SPECIES + hp["n_basis"]
    for k, w in enumerate(hp["two_body"]):
        out.append((f"W2b.{k}", (fan, w)))
        fan = w
    layers = so3.model_paths(lmax, hp["n_layers"])
    for L in range(1, hp["n_layers"] + 1):
        out.append((f"Wenv.{L}", (D, (lmax + 1) * C)))
        if L < hp["n_layers"]:
            out.append((f"theta.{L}", (len(layers[L - 1][1]), C)))
        fan = D + (lmax + 1) * C
        for k, w in enumerate(hp["latent"]):
            out.append((f"Wlat.{L}.{k}", (fan, w)))
            fan = w
    fan = D
    for k, w in enumerate(list(hp["edge_eng"]) + [1]):
        out.append((f"We.{k}", (fan, w)))
        fan = w
    return out


def init_params(hp: dict, seed: int) -> dict:
    params = {}
    for t, (name, shape) in enumerate(param_shapes(hp)):
        n = int(np.prod(shape))
        params[name] = tensor_uniform(seed, t, n).reshape(shape)
    return params


def count_params(hp: dict) -> int:
    return int(sum(np.prod(s) for _, s in param_shapes(hp)))
