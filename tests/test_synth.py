"""Pins of the seeded synthetic inputs against the recipes they claim to follow.

Every benchmark and parity case draws its positions, species, boxes and velocities from
`synth`, so a drifted recipe (a wrong density, a broken molecule, a species count off by
one) would silently change what is measured.  These checks recompute each stated property
from the generated arrays with plain geometry and SI constants: stoichiometry, density,
bond lengths and angles, exclusion distances, lattice occupancy, float32 exactness,
periodic wrapping, seed determinism, and the Maxwell-Boltzmann temperature.
"""
import math

import numpy as np
import pytest

import synth

# SI constants (CODATA 2018 exact / recommended values).
E_CHARGE = 1.602176634e-19          # J per eV
AMU = 1.66053906660e-27             # kg
K_BOLTZMANN = 1.380649e-23          # J/K
G_CM3_PER_AMU_A3 = AMU * 1e3 / 1e-24   # amu/A^3 -> g/cm^3

# Float32 rounding of positions up to ~400 A moves a distance by at most a few 1e-5 A.
TOL_LEN = 1e-4


def _min_image(d, box):
    return d - box * np.round(d / box)


def _density(s):
    return s.masses.sum() / np.prod(s.box) * G_CM3_PER_AMU_A3


def _f32_exact(pos):
    return np.array_equal(pos, pos.astype(np.float32).astype(np.float64))


def _wrapped(s):
    return bool(np.all(s.pos >= 0.0) and np.all(s.pos < s.box[None, :]))


def _counts(Z):
    u, c = np.unique(Z, return_counts=True)
    return dict(zip(u.tolist(), c.tolist()))


def _min_pair_distance(p, box=None, chunk=512):
    best = np.inf
    for a in range(0, p.shape[0], chunk):
        d = p[a:a + chunk, None, :] - p[None, :, :]
        if box is not None:
            d = _min_image(d, box)
        r2 = (d * d).sum(-1)
        idx = np.arange(a, min(a + chunk, p.shape[0]))
        r2[idx - a, idx] = np.inf
        best = min(best, float(r2.min()))
    return math.sqrt(best)


def _water_geometry(O, H1, H2, box):
    d1 = _min_image(H1 - O, box)
    d2 = _min_image(H2 - O, box)
    r1 = np.linalg.norm(d1, axis=1)
    r2 = np.linalg.norm(d2, axis=1)
    cos = (d1 * d2).sum(1) / (r1 * r2)
    ang = np.degrees(np.arccos(np.clip(cos, -1.0, 1.0)))
    return np.concatenate([r1, r2]), ang


@pytest.fixture(scope="module")
def water12288():
    return synth.bench_workloads()["water12288"]["make"]()


@pytest.fixture(scope="module")
def mixture():
    return synth.nanoparticle_mixture_system(1005)


def test_unit_constants_follow_from_si():
    # 1 eV/amu in (A/fs)^2 and k_B in eV/K, from the SI definitions.
    v2 = E_CHARGE / AMU * (1e10 / 1e15) ** 2
    assert synth.systems.EV_PER_AMU_A2_FS2 == pytest.approx(v2, rel=1e-9)
    assert synth.systems.K_B == pytest.approx(K_BOLTZMANN / E_CHARGE, rel=1e-9)
    # standard atomic weights (IUPAC conventional values)
    ref = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999, 14: 28.085, 20: 40.078}
    for z, m in ref.items():
        assert synth.MASSES[z] == pytest.approx(m, abs=1e-3)


def test_water_recipe(water12288):
    s = water12288
    n_mol = s.n // 3
    assert s.n == 12288 and s.pbc.all() and s.sys_ptr.tolist() == [0, s.n]
    assert np.array_equal(s.Z, np.tile(np.array([8, 1, 1], dtype=np.int32), n_mol))
    assert _f32_exact(s.pos) and _wrapped(s)
    assert _density(s) == pytest.approx(1.0, rel=2e-3)
    O, H1, H2 = s.pos[0::3], s.pos[1::3], s.pos[2::3]
    r, ang = _water_geometry(O, H1, H2, s.box)
    assert r.min() >= 0.94 - TOL_LEN and r.max() <= 0.98 + TOL_LEN
    assert ang.min() >= 101.5 - 0.02 and ang.max() <= 107.5 + 0.02
    # uniform draws fill their ranges
    assert r.min() < 0.942 and r.max() > 0.978
    assert ang.min() < 101.7 and ang.max() > 107.3
    # random sequential addition respects the O-O exclusion distance
    assert _min_pair_distance(O, s.box) >= 2.4 - TOL_LEN


def test_water_default_box_hits_the_density():
    s = synth.water_system(200, seed=11)
    assert _density(s) == pytest.approx(1.0, rel=1e-9)
    assert s.meta["L"] == pytest.approx(s.box[0])


def test_water_orientations_are_isotropic(water12288):
    s = water12288
    d = _min_image(s.pos[1::3] - s.pos[0::3], s.box)
    u = d / np.linalg.norm(d, axis=1, keepdims=True)
    # uniform unit vectors: mean ~ 0 and second moment ~ I/3
    assert np.abs(u.mean(0)).max() < 0.05
    assert np.abs(u.T @ u / u.shape[0] - np.eye(3) / 3.0).max() < 0.03


def _lattice_check(s, n_xyz, spacing, jitter):
    idx = np.floor(s.pos / spacing).astype(np.int64)
    nx, ny, nz = n_xyz
    idx %= np.array([nx, ny, nz])
    site = (idx[:, 0] * ny + idx[:, 1]) * nz + idx[:, 2]
    assert np.unique(site).shape[0] == s.n                    # one atom per site
    centre = (idx + 0.5) * spacing
    dev = _min_image(s.pos - centre, s.box)
    # 8 sigma: beyond the largest of ~1e7 normal draws, well inside half a spacing
    assert np.abs(dev).max() < 8.0 * jitter
    return dev


def test_csh_full_recipe():
    s = synth.csh_system(False, 1002)
    assert s.n == 131072 and s.pbc.all()
    np.testing.assert_allclose(s.box, np.array([32, 64, 64]) * 2.228)
    c = _counts(s.Z)
    assert c == {20: 20825, 14: 12250, 8: 66148, 1: 31849}
    # Ca:Si:O:H = 1.7 : 1 : 5.4 : 2.6
    assert c[20] / c[14] == pytest.approx(1.7, abs=1e-3)
    assert c[8] / c[14] == pytest.approx(5.4, abs=1e-3)
    assert c[1] / c[14] == pytest.approx(2.6, abs=1e-3)
    assert _density(s) == pytest.approx(2.6, rel=5e-3)
    assert _f32_exact(s.pos) and _wrapped(s)
    dev = _lattice_check(s, (32, 64, 64), 2.228, 0.1)
    assert dev.std() == pytest.approx(0.1, rel=0.01)
    assert np.abs(dev.mean(0)).max() < 2e-3
    # species are shuffled over the sites: each species' mean position is near the centre
    for z in (20, 14, 8, 1):
        np.testing.assert_allclose(s.pos[s.Z == z].mean(0), s.box / 2, rtol=0.03)


def test_csh_sub_box_recipe():
    s = synth.csh_system(True, 1002)
    assert s.n == 512
    np.testing.assert_allclose(s.box, [8 * 2.228] * 3)
    c = _counts(s.Z)
    assert c == {20: 81, 14: 48, 8: 258, 1: 125}
    assert _density(s) == pytest.approx(2.6, rel=0.01)
    _lattice_check(s, (8, 8, 8), 2.228, 0.1)


def test_sio2_recipe():
    s = synth.sio2_system(162, 4194304, 1004)
    assert s.n == 4194304 and s.pbc.all()
    np.testing.assert_allclose(s.box, [162 * 2.4614] * 3)
    c = _counts(s.Z)
    assert c == {14: 4194304 // 3, 8: 4194304 - 4194304 // 3}
    assert c[8] / c[14] == pytest.approx(2.0, abs=1e-5)
    assert _density(s) == pytest.approx(2.2, rel=2e-3)
    assert _f32_exact(s.pos) and _wrapped(s)
    _lattice_check(s, (162, 162, 162), 2.4614, 0.1)


def test_cubic96_recipe():
    s = synth.config1_system(1000)
    assert s.n == 96
    np.testing.assert_allclose(s.box, [10.0] * 3)
    assert set(np.unique(s.Z).tolist()) <= {1, 6, 8, 14}
    assert _f32_exact(s.pos) and _wrapped(s)
    _lattice_check(s, (5, 5, 5), 2.0, 0.1)


def test_molecules_recipe():
    s = synth.molecules_system(64, 1003)
    assert not s.pbc.any() and _f32_exact(s.pos)
    assert s.sys_ptr.shape[0] == 65 and s.sys_ptr[0] == 0 and s.sys_ptr[-1] == s.n
    valence = {6: 4, 7: 3, 8: 2}
    lo = s.pos.min(0)
    assert np.all(s.pos - lo < s.box)                          # the binning extent covers all
    n_heavy = []
    for m in range(64):
        a, b = s.sys_ptr[m], s.sys_ptr[m + 1]
        Z, p = s.Z[a:b], s.pos[a:b]
        heavy = Z != 1
        k = int(heavy.sum())
        n_heavy.append(k)
        assert 7 <= k <= 23
        assert np.all(heavy[:k]) and not np.any(heavy[k:])      # heavy atoms first, then H
        assert set(Z[:k].tolist()) <= {6, 7, 8}
        # a bonded tree of k-1 bonds leaves sum(valence) - 2(k-1) free valences for H
        free = sum(valence[int(z)] for z in Z[:k]) - 2 * (k - 1)
        assert 0 <= (b - a) - k <= free
        # local coordinates: the first atom starts at the origin (plus noise)
        assert np.linalg.norm(p[0]) < 0.05 * 6
        # every atom lies within a bond length (1.0-1.5 A, plus noise) of another;
        # no two atoms are closer than the 1.0 A rejection distance minus noise
        d = np.linalg.norm(p[:, None] - p[None], axis=-1)
        np.fill_diagonal(d, np.inf)
        assert d.min() > 1.0 - 0.05 * math.sqrt(2) * 5
        assert d.min(1).max() < 1.5 + 0.05 * math.sqrt(2) * 5
    assert min(n_heavy) < 10 and max(n_heavy) > 20               # the U{7..23} draw spans


def test_nanoparticle_mixture_recipe(mixture):
    s = mixture
    assert s.n == 6326 and s.pbc.all()
    np.testing.assert_allclose(s.box, [45.7] * 3)
    assert _counts(s.Z) == {6: 267, 20: 90, 14: 133, 8: 2577, 1: 3259}
    assert _f32_exact(s.pos) and _wrapped(s)
    n_p = s.meta["n_particle"]
    assert n_p == 90 + 133 + 718 + 609
    assert _counts(s.Z[:n_p]) == {20: 90, 14: 133, 8: 718, 1: 609}
    assert 718 / 133 == pytest.approx(5.4, abs=0.01)
    # the particle is compact about the box centre; its lattice spacing gives C-S-H density
    c = s.box / 2
    r = np.linalg.norm(_min_image(s.pos[:n_p] - c, s.box), axis=1)
    assert r.max() <= s.meta["r_particle"] + 0.7
    vol = 4.0 / 3.0 * math.pi * s.meta["r_particle"] ** 3
    assert n_p / vol == pytest.approx(1.0 / 2.228 ** 3, rel=0.1)


def test_nanoparticle_mixture_fluid(mixture):
    s = mixture
    n_p = s.meta["n_particle"]
    fl = s.pos[n_p:].reshape(-1, 3, 3)
    fz = s.Z[n_p:].reshape(-1, 3)
    co2 = np.all(fz == [6, 8, 8], axis=1)
    h2o = np.all(fz == [8, 1, 1], axis=1)
    assert co2.sum() == 267 and h2o.sum() == 1325 and np.all(co2 | h2o)
    # CO2: linear O=C=O at 1.16 A
    g = fl[co2]
    d1 = _min_image(g[:, 1] - g[:, 0], s.box)
    d2 = _min_image(g[:, 2] - g[:, 0], s.box)
    np.testing.assert_allclose(np.linalg.norm(d1, axis=1), 1.16, atol=TOL_LEN)
    np.testing.assert_allclose(np.linalg.norm(d2, axis=1), 1.16, atol=TOL_LEN)
    np.testing.assert_allclose(d1 + d2, 0.0, atol=TOL_LEN)
    # water as in the bulk-water recipe
    w = fl[h2o]
    r, ang = _water_geometry(w[:, 0], w[:, 1], w[:, 2], s.box)
    assert r.min() >= 0.94 - TOL_LEN and r.max() <= 0.98 + TOL_LEN
    assert ang.min() >= 101.5 - 0.02 and ang.max() <= 107.5 + 0.02
    # molecule centres (C of CO2, O of H2O): outside the particle, 2.6 A apart
    centres = fl[:, 0]
    rc = np.linalg.norm(_min_image(centres - s.box / 2, s.box), axis=1)
    assert rc.min() >= s.meta["r_particle"] + 1.8 - TOL_LEN
    assert _min_pair_distance(centres, s.box) >= 2.6 - TOL_LEN


@pytest.mark.parametrize("make", [
    lambda seed: synth.water_system(100, seed=seed),
    lambda seed: synth.csh_system(True, seed),
    lambda seed: synth.molecules_system(8, seed),
    lambda seed: synth.config1_system(seed),
])
def test_generators_are_seeded(make):
    a, b, c = make(5), make(5), make(6)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.Z, b.Z)
    assert np.array_equal(a.sys_ptr, b.sys_ptr)
    assert not (a.pos.shape == c.pos.shape and np.array_equal(a.pos, c.pos))


def test_maxwell_boltzmann_temperature_and_momentum(water12288):
    m = water12288.masses
    T = 300.0
    v = synth.maxwell_boltzmann(m, T, seed=7)
    assert np.array_equal(v, synth.maxwell_boltzmann(m, T, seed=7))
    p = (m[:, None] * v).sum(0)
    assert np.abs(p).max() < 1e-12 * np.sqrt(m.sum())
    # kinetic temperature (SI arithmetic): sum(m v^2) / (3 N k_B)
    v_si = v * 1e5                                            # A/fs -> m/s
    t_kin = (m[:, None] * AMU * v_si ** 2).sum() / (3 * m.shape[0] * K_BOLTZMANN)
    # sampling error of the estimate ~ sqrt(2 / (3N)) = 0.7%
    assert t_kin == pytest.approx(T, rel=0.03)
    # each species has the same temperature (velocity variance ~ 1/m)
    for z in (8, 1):
        sel = water12288.Z == z
        tz = (m[sel, None] * AMU * v_si[sel] ** 2).sum() / (3 * sel.sum() * K_BOLTZMANN)
        assert tz == pytest.approx(T, rel=0.05)
