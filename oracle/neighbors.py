"""Brute-force neighbour lists of the FP64 oracle.

TEST INFRASTRUCTURE (see oracle/__init__.py).

Allegro is strictly local: an atom interacts only with the atoms inside a radial cutoff
(Abstract; Methodology, Model Training: "radial cutoff").  An edge is an ordered triple
(i, j, s) of a centre atom i, a neighbour atom j and an integer periodic image shift s,
with i != j or s != 0, whose separation  d = x_j + s*L - x_i  is shorter than the cutoff.

The membership test is fixed in float32 so that the edge list is exactly defined (a
reading; the paper does not discuss it): with xf = float32 positions, Lf = float32 box,

    d_k = (xf_j,k - xf_i,k) + float32(s_k) * Lf_k          (each operation rounded)
    r2  = (d_x*d_x + d_y*d_y) + d_z*d_z
    edge  <=>  r2 < float32(rl * rl),  rl = float32(float32(rc) + float32(skin))

with no fused multiply-add (numpy float32 ufuncs round every operation).  Edges are
sorted by (i, j, s) with s compared lexicographically.  Atoms of different systems
(sys_ptr) never pair; non-periodic axes have s_k = 0.
"""
from __future__ import annotations

import math

import numpy as np


def cutoff_sq_f32(rc: float, skin: float = 0.0) -> np.float32:
    rl = np.float32(np.float32(rc) + np.float32(skin))
    return np.float32(rl * rl)


def _shift_ranges(box, pbc, rl):
    rng = []
    for k in range(3):
        if pbc[k]:
            m = int(math.ceil(rl / box[k])) + 1
            rng.append(np.arange(-m, m + 1))
        else:
            rng.append(np.array([0]))
    return rng


def _pairs_for_centre(i, cand, xf, Lf, pbc, box, rl2, rl):
    """All (j, s) of centre i among candidate atoms `cand` (FP32 predicate)."""
    out_j, out_s = [], []
    xi = xf[i]
    d0 = xf[cand] - xi                                          # float32
    # base image of each candidate (closest one in float64), then a window around it
    base = np.zeros((cand.shape[0], 3), dtype=np.int64)
    for k in range(3):
        if pbc[k]:
            base[:, k] = -np.round(d0[:, k].astype(np.float64) / box[k]).astype(np.int64)
    win = _shift_ranges(box, pbc, rl)
    for a in win[0]:
        for b in win[1]:
            for c in win[2]:
                s = base + np.array([a, b, c])
                sf = s.astype(np.float32)
                d = d0 + sf * Lf                                # float32, rounded per op
                r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
                ok = r2 < rl2
                ok &= ~((cand == i) & np.all(s == 0, axis=1))
                if ok.any():
                    out_j.append(cand[ok])
                    out_s.append(s[ok])
    if not out_j:
        return np.zeros(0, np.int64), np.zeros((0, 3), np.int64)
    j = np.concatenate(out_j)
    s = np.concatenate(out_s)
    # window sets overlap for tiny boxes: drop duplicates, then sort by (j, s0, s1, s2)
    key = np.stack([j, s[:, 0], s[:, 1], s[:, 2]], axis=1)
    key = np.unique(key, axis=0)          # unique sorts lexicographically
    return key[:, 0], key[:, 1:]


def _is_tiny(box, pbc, rl):
    return any(pbc[k] and box[k] < 2.0 * rl + 0.1 for k in range(3))


def _pairs_chunk(ids, lo, hi, pos, xf, Lf, pbc, box, rl2, rl):
    """Edges of the centres `ids` (one system [lo, hi)) for boxes where only the nearest
    image of each atom can lie inside the cutoff: every periodic box edge is longer than
    2*rl + 0.1, so two images of one atom are never both within rl of a centre."""
    cand = np.arange(lo, hi)
    d = pos[cand][None, :, :] - pos[ids][:, None, :]                  # float64
    base = np.zeros(d.shape, dtype=np.int64)
    for k in range(3):
        if pbc[k]:
            base[..., k] = -np.round(d[..., k] / box[k]).astype(np.int64)
            d[..., k] += base[..., k] * box[k]
    near = np.einsum("abk,abk->ab", d, d) < (rl + 0.01) ** 2
    ci, cj = np.nonzero(near)
    i = ids[ci]
    j = cand[cj]
    s = base[ci, cj]
    df = (xf[j] - xf[i]) + s.astype(np.float32) * Lf                  # float32 per op
    r2 = (df[:, 0] * df[:, 0] + df[:, 1] * df[:, 1]) + df[:, 2] * df[:, 2]
    ok = (r2 < rl2) & ~((i == j) & np.all(s == 0, axis=1))
    i, j, s = i[ok], j[ok], s[ok]
    key = np.stack([i, j, s[:, 0], s[:, 1], s[:, 2]], axis=1)
    order = np.lexsort(key.T[::-1])
    return key[order]


def neighbor_list(pos, box, pbc, rc, skin=0.0, sys_ptr=None, centres=None):
    """Sorted edge list.  Returns (row_ptr [n+1], col [E], shift [E,3]) over all centres,
    or, when `centres` is given, a dict centre -> (col, shift) for those atoms only."""
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    box = np.asarray(box, dtype=np.float64)
    pbc = np.asarray(pbc, dtype=bool)
    if sys_ptr is None:
        sys_ptr = np.array([0, n])
    sys_ptr = np.asarray(sys_ptr, dtype=np.int64)
    xf = pos.astype(np.float32)
    Lf = box.astype(np.float32)
    rl2 = cutoff_sq_f32(rc, skin)
    rl = float(np.float32(np.float32(rc) + np.float32(skin)))
    want = np.arange(n) if centres is None else np.asarray(sorted(set(centres)), np.int64)
    sys_of = np.searchsorted(sys_ptr, want, side="right") - 1
    rows = []
    if _is_tiny(box, pbc, rl):
        for i, si in zip(want, sys_of):
            j, s = _pairs_for_centre(int(i), np.arange(sys_ptr[si], sys_ptr[si + 1]), xf,
                                     Lf, pbc, box, rl2, rl)
            rows.append(np.concatenate([np.full((j.shape[0], 1), i), j[:, None], s], 1))
    else:
        for si in np.unique(sys_of):
            ids_all = want[sys_of == si]
            lo, hi = int(sys_ptr[si]), int(sys_ptr[si + 1])
            chunk = max(1, min(512, 4_000_000 // max(1, hi - lo)))
            for c0 in range(0, ids_all.shape[0], chunk):
                rows.append(_pairs_chunk(ids_all[c0:c0 + chunk], lo, hi, pos, xf, Lf,
                                         pbc, box, rl2, rl))
    key = np.concatenate(rows) if rows else np.zeros((0, 5), np.int64)
    key = key[np.lexsort(key.T[::-1])]
    if centres is not None:
        res = {}
        for i in want:
            m = key[:, 0] == i
            res[int(i)] = (key[m, 1], key[m, 2:])
        return res
    counts = np.bincount(key[:, 0], minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, key[:, 1].copy(), key[:, 2:].copy()


def reverse_index(row_ptr, col, shift):
    """rev[e] = index of the edge (j, i, -s) for e = (i, j, s) (it always exists)."""
    n = row_ptr.shape[0] - 1
    lookup = {}
    for i in range(n):
        for e in range(row_ptr[i], row_ptr[i + 1]):
            lookup[(i, int(col[e]), *map(int, shift[e]))] = e
    rev = np.empty(col.shape[0], dtype=np.int64)
    for i in range(n):
        for e in range(row_ptr[i], row_ptr[i + 1]):
            j = int(col[e])
            s = shift[e]
            rev[e] = lookup[(j, i, -int(s[0]), -int(s[1]), -int(s[2]))]
    return rev
