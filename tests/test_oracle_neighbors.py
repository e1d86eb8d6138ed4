"""Pins of the oracle's brute-force neighbour lists.

Cross-checks against scipy's periodic k-d tree (an independent library routine) and an
explicit image enumeration, plus the symmetries the definition implies.  Pairs whose
distance lies within 1e-4 A of the cutoff are left out of the library comparison: there
the float32 membership test legitimately differs from float64 distances.
"""
import itertools

import numpy as np
import pytest
from scipy.spatial import cKDTree

import synth
from oracle import neighbors


def _pairs_set(row_ptr, col):
    i = np.repeat(np.arange(row_ptr.shape[0] - 1), np.diff(row_ptr))
    return set(zip(i.tolist(), col.tolist()))


@pytest.mark.parametrize("make,rc", [(lambda: synth.csh_system(sub=True), 6.0),
                                     (lambda: synth.water_system(300, L=20.0, seed=3), 6.0)])
def test_matches_periodic_kdtree(make, rc):
    s = make()
    row_ptr, col, shift = neighbors.neighbor_list(s.pos, s.box, s.pbc, rc)
    tree = cKDTree(s.pos, boxsize=s.box)
    ref = set()
    for a, b in tree.query_pairs(rc + 1e-4):
        ref.add((a, b))
        ref.add((b, a))
    got = _pairs_set(row_ptr, col)

    def dist(a, b):
        d = s.pos[b] - s.pos[a]
        d -= s.box * np.round(d / s.box)
        return np.linalg.norm(d)

    for a, b in ref ^ got:
        assert abs(dist(a, b) - rc) < 1e-4, (a, b, dist(a, b))


def test_tiny_box_matches_image_enumeration():
    s = synth.config1_system()
    rc = 5.0
    row_ptr, col, shift = neighbors.neighbor_list(s.pos, s.box, s.pbc, rc)
    got = set()
    for i in range(s.n):
        for e in range(row_ptr[i], row_ptr[i + 1]):
            got.add((i, int(col[e]), *map(int, shift[e])))
    ref = set()
    near = set()
    for i in range(s.n):
        for j in range(s.n):
            for sv in itertools.product(range(-2, 3), repeat=3):
                if i == j and sv == (0, 0, 0):
                    continue
                d = np.linalg.norm(s.pos[j] + np.array(sv) * s.box - s.pos[i])
                if d < rc - 1e-4:
                    ref.add((i, j, *sv))
                elif d < rc + 1e-4:
                    near.add((i, j, *sv))
    assert ref <= got
    assert got - ref <= near


def test_sorted_symmetric_and_reverse_index():
    s = synth.config1_system()
    row_ptr, col, shift = neighbors.neighbor_list(s.pos, s.box, s.pbc, 5.0)
    for i in range(s.n):
        seg = list(zip(col[row_ptr[i]:row_ptr[i + 1]].tolist(),
                       map(tuple, shift[row_ptr[i]:row_ptr[i + 1]].tolist())))
        assert seg == sorted(seg) and len(set(seg)) == len(seg)
    rev = neighbors.reverse_index(row_ptr, col, shift)
    np.testing.assert_array_equal(rev[rev], np.arange(col.shape[0]))
    i = np.repeat(np.arange(s.n), np.diff(row_ptr))
    np.testing.assert_array_equal(col[rev], i)
    np.testing.assert_array_equal(shift[rev], -shift)


def test_mean_count_matches_density():
    s = synth.csh_system(sub=True)
    row_ptr, _, _ = neighbors.neighbor_list(s.pos, s.box, s.pbc, 6.0)
    n = s.n / np.prod(s.box)
    expect = 4.0 / 3.0 * np.pi * 6.0 ** 3 * n
    assert abs(row_ptr[-1] / s.n - expect) / expect < 0.05


def test_supercell_replication():
    s = synth.config1_system()
    rp1, _, _ = neighbors.neighbor_list(s.pos, s.box, s.pbc, 5.0)
    reps = [s.pos + np.array(v) * s.box for v in itertools.product(range(2), repeat=3)]
    pos2 = np.concatenate(reps)
    rp2, _, _ = neighbors.neighbor_list(pos2, 2 * s.box, s.pbc, 5.0)
    c1 = np.diff(rp1)
    c2 = np.diff(rp2).reshape(8, s.n)
    for r in range(8):
        np.testing.assert_array_equal(c2[r], c1)


def test_systems_do_not_interact_and_nonperiodic():
    s = synth.molecules_system(8, seed=5)
    row_ptr, col, shift = neighbors.neighbor_list(s.pos, s.box, s.pbc, 6.0, sys_ptr=s.sys_ptr)
    i = np.repeat(np.arange(s.n), np.diff(row_ptr))
    sys_of = np.searchsorted(s.sys_ptr, np.arange(s.n), side="right") - 1
    np.testing.assert_array_equal(sys_of[i], sys_of[col])
    assert np.all(shift == 0)


def test_centre_subset_equals_full_list():
    s = synth.config1_system()
    row_ptr, col, shift = neighbors.neighbor_list(s.pos, s.box, s.pbc, 5.0, skin=0.5)
    sub = neighbors.neighbor_list(s.pos, s.box, s.pbc, 5.0, skin=0.5, centres=[3, 50])
    for i in (3, 50):
        np.testing.assert_array_equal(sub[i][0], col[row_ptr[i]:row_ptr[i + 1]])
        np.testing.assert_array_equal(sub[i][1], shift[row_ptr[i]:row_ptr[i + 1]])
