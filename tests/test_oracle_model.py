"""Pins of the oracle's energy and hand-derived forces.

What the physics and the definition fix, independent of the oracle's own code:
central finite differences (with the O(h^2) convergence of the difference), zero net
force, invariance of E and covariance of F under rotations, inversion, translations and
permutations, extensivity under periodic replication, strict locality, the isolated
atom, the dimer (forces along the bond, smooth decay at the cutoff), the pair-potential
special case with the environment switched off, and NVE energy conservation with
fluctuations that scale as dt^2 and no secular drift over a long run.
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import Allegro64, md, neighbors, pool, so3

SMALL = synth.preset("small")
WATER = synth.preset("fm_water")


@pytest.fixture(scope="module")
def small():
    return Allegro64(SMALL, 42)


@pytest.fixture(scope="module")
def big():
    return Allegro64(WATER, 42)


@pytest.fixture(scope="module")
def cfg1(small):
    s = synth.config1_system()
    E, Ea, F = small.evaluate(s.pos, s.Z, s.box, s.pbc)
    return s, E, Ea, F


def _energy(model, s, pos):
    return model.evaluate(pos, s.Z, s.box, s.pbc, forces=False)[0].sum()


def test_forces_match_central_differences(small, cfg1):
    s, _, _, F = cfg1
    errs = {}
    for h in (1e-3, 5e-4):
        err = []
        for a, k in [(0, 0), (17, 1), (50, 2), (95, 0)]:
            p1, p2 = s.pos.copy(), s.pos.copy()
            p1[a, k] += h
            p2[a, k] -= h
            fd = -(_energy(small, s, p1) - _energy(small, s, p2)) / (2 * h)
            err.append(abs(fd - F[a, k]))
            assert abs(fd - F[a, k]) < 1e-7 + 1e-5 * abs(F[a, k])
        errs[h] = np.array(err)
    ratio = errs[1e-3].sum() / errs[5e-4].sum()
    assert 3.0 < ratio < 5.0, ratio           # truncation error ~ h^2


def test_forces_fd_l2_three_layers(big):
    s = synth.csh_system(sub=True)
    h = 1e-4
    for a, k in [(3, 0), (200, 2)]:
        Fs, _ = big.sampled_forces(s.pos, s.Z, s.box, s.pbc, [a])
        p1, p2 = s.pos.copy(), s.pos.copy()
        p1[a, k] += h
        p2[a, k] -= h
        # only the energies of `a` and of its neighbours depend on x_a
        nl = neighbors.neighbor_list(s.pos, s.box, s.pbc, WATER["rc"], 0.1, centres=[a])
        near = sorted({a} | set(int(j) for j in nl[a][0]))
        e1 = big.centre_terms(p1, s.Z, s.box, s.pbc, near)
        e2 = big.centre_terms(p2, s.Z, s.box, s.pbc, near)
        fd = -(sum(v[0] for v in e1.values()) - sum(v[0] for v in e2.values())) / (2 * h)
        assert abs(fd - Fs[a][k]) < 1e-8 + 1e-5 * abs(Fs[a][k]), (fd, Fs[a][k])


def test_zero_net_force(cfg1):
    _, _, _, F = cfg1
    assert np.abs(F.sum(axis=0)).max() < 1e-13 * F.shape[0]


@pytest.mark.parametrize("which", ["small", "big"])
def test_rotation_inversion_invariance(which, small, big):
    model = small if which == "small" else big
    s = synth.cluster_system(14, seed=3)
    E0, _, F0 = model.evaluate(s.pos, s.Z, s.box, s.pbc)
    rng = np.random.default_rng(11)
    for improper in (False, True):
        R = so3.random_rotation(rng) * (-1.0 if improper else 1.0)
        c = s.pos.mean(axis=0)
        pos = (s.pos - c) @ R.T + c
        E1, _, F1 = model.evaluate(pos, s.Z, s.box, s.pbc)
        assert abs(E1[0] - E0[0]) < 1e-12 * max(1.0, abs(E0[0]))
        np.testing.assert_allclose(F1, F0 @ R.T, atol=1e-12 * np.abs(F0).max())


def test_periodic_translation_and_axis_permutation(small, cfg1):
    s, E0, _, F0 = cfg1
    pos = np.mod(s.pos + np.array([1.25, -3.5, 0.75]), s.box)
    E1, _, F1 = small.evaluate(pos, s.Z, s.box, s.pbc)
    assert abs(E1[0] - E0[0]) < 1e-11
    np.testing.assert_allclose(F1, F0, atol=1e-11)
    perm = [2, 0, 1]
    E2, _, F2 = small.evaluate(s.pos[:, perm], s.Z, s.box[perm], s.pbc)
    assert abs(E2[0] - E0[0]) < 1e-11
    np.testing.assert_allclose(F2, F0[:, perm], atol=1e-11)


def test_permutation(small, cfg1):
    s, E0, Ea0, F0 = cfg1
    p = np.random.default_rng(2).permutation(s.n)
    E1, Ea1, F1 = small.evaluate(s.pos[p], s.Z[p], s.box, s.pbc)
    assert abs(E1[0] - E0[0]) < 1e-11
    np.testing.assert_allclose(Ea1, Ea0[p], atol=1e-12)
    np.testing.assert_allclose(F1, F0[p], atol=1e-12)


def test_supercell_extensive(small, cfg1):
    s, E0, Ea0, F0 = cfg1
    reps = [s.pos + np.array(v) * s.box for v in itertools.product(range(2), repeat=3)]
    pos2 = np.concatenate(reps)
    E2, Ea2, F2 = small.evaluate(pos2, np.tile(s.Z, 8), 2 * s.box, s.pbc)
    assert abs(E2[0] - 8 * E0[0]) < 1e-10
    np.testing.assert_allclose(Ea2, np.tile(Ea0, 8), atol=1e-12)
    np.testing.assert_allclose(F2, np.tile(F0, (8, 1)), atol=1e-12)


def test_isolated_atom_and_locality(small):
    s = synth.cluster_system(10, seed=4)
    E, Ea, F = small.evaluate(s.pos, s.Z, s.box, s.pbc)
    far = np.array([[40.0, 40.0, 40.0]])
    pos = np.concatenate([s.pos, far])
    Z = np.concatenate([s.Z, [14]])
    box = np.array([60.0, 60.0, 60.0])
    E2, Ea2, F2 = small.evaluate(pos, Z, box, s.pbc)
    assert Ea2[-1] == 0.0 and np.all(F2[-1] == 0.0)
    np.testing.assert_allclose(Ea2[:-1], Ea, atol=1e-14)
    np.testing.assert_allclose(F2[:-1], F, atol=1e-14)


def test_dimer_forces_along_bond_and_smooth_cutoff(small):
    rc = SMALL["rc"]
    d = np.array([1.0, 2.0, -0.5])
    s = synth.dimer_system(2.1, 8, 1, d)
    E, _, F = small.evaluate(s.pos, s.Z, s.box, s.pbc)
    np.testing.assert_allclose(F[0], -F[1], atol=1e-14)
    u = d / np.linalg.norm(d)
    assert np.linalg.norm(F[0] - (F[0] @ u) * u) < 1e-13
    e = []
    for delta in (2e-2, 1e-2):
        sd = synth.dimer_system(rc - delta, 8, 1, d)
        e.append(small.evaluate(sd.pos, sd.Z, sd.box, sd.pbc, forces=False)[0][0])
    assert abs(e[0] / e[1] - 8.0) < 0.5            # E ~ (rc - r)^3 at the cutoff
    sd = synth.dimer_system(rc + 1e-3, 8, 1, d)
    assert small.evaluate(sd.pos, sd.Z, sd.box, sd.pbc)[0][0] == 0.0


def test_pair_potential_special_case(small):
    """With every environment projection zeroed the model is a pair potential."""
    params = {k: v.copy() for k, v in small.params.items()}
    for k in params:
        if k.startswith("Wenv."):
            params[k][:] = 0.0
    pair = Allegro64(SMALL, params=params)
    s = synth.cluster_system(8, seed=6, radius=2.5)
    E = pair.evaluate(s.pos, s.Z, s.box, s.pbc, forces=False)[0][0]
    total = 0.0
    for a, b in itertools.combinations(range(s.n), 2):
        pos = s.pos[[a, b]]
        total += pair.evaluate(pos, s.Z[[a, b]], s.box, s.pbc, forces=False)[0][0]
    assert abs(E - total) < 1e-12 * max(1.0, abs(E))
    # the full model is genuinely many-body
    Efull = small.evaluate(s.pos, s.Z, s.box, s.pbc, forces=False)[0][0]
    tot_full = sum(small.evaluate(s.pos[[a, b]], s.Z[[a, b]], s.box, s.pbc,
                                  forces=False)[0][0]
                   for a, b in itertools.combinations(range(s.n), 2))
    assert abs(Efull - tot_full) > 1e-6


def test_chunking_and_drivers_agree(small, cfg1):
    s, E0, Ea0, F0 = cfg1
    E1, Ea1, F1 = small.evaluate(s.pos, s.Z, s.box, s.pbc, chunk_edges=300)
    np.testing.assert_allclose(Ea1, Ea0, atol=1e-13)
    np.testing.assert_allclose(F1, F0, atol=1e-13)
    Fs, Es = small.sampled_forces(s.pos, s.Z, s.box, s.pbc, [0, 9, 77])
    for m in (0, 9, 77):
        np.testing.assert_allclose(Fs[m], F0[m], atol=1e-13)
        assert abs(Es[m] - Ea0[m]) < 1e-13
    E2, Ea2, F2 = pool.evaluate(SMALL, 42, s.pos, s.Z, s.box, s.pbc, workers=2)
    np.testing.assert_allclose(F2, F0, atol=1e-13)
    Fp, Ep = pool.sampled_forces(SMALL, 42, s.pos, s.Z, s.box, s.pbc, [9], workers=2)
    np.testing.assert_allclose(Fp[9], F0[9], atol=1e-13)


def test_nve_energy_fluctuation_scales_dt2(small):
    s = synth.cluster_system(12, seed=8, radius=2.6)
    m = s.masses
    v0 = synth.maxwell_boltzmann(m, 600.0, seed=1)
    fl = []
    for dt, n in ((2.0, 20), (1.0, 40)):
        _, _, ep, ek = md.run_nve(small, s.pos, v0, s.Z, s.box, s.pbc, m, dt, n)
        et = ep + ek
        fl.append(et.max() - et.min())
    assert 3.0 < fl[0] / fl[1] < 5.0, fl


@pytest.mark.slow
def test_nve_no_secular_drift(small):
    """Velocity Verlet is symplectic: over many steps the total energy fluctuates about a
    constant without a trend.  Eight atoms in a periodic 6.5 A box (they keep
    interacting through the images), 800 steps of 1 fs from 300 K: the fitted linear drift
    over the run is far below the fluctuation, and the fluctuation is small next to the
    potential-energy excursions it is made of."""
    s = synth.lattice_system("box8", (2, 2, 2), 3.25, 8, [1, 6, 8, 14], 21)
    m = s.masses
    v0 = synth.maxwell_boltzmann(m, 300.0, seed=3)
    n = 800
    _, _, ep, ek = md.run_nve(small, s.pos, v0, s.Z, s.box, s.pbc, m, 1.0, n)
    et = ep + ek
    slope = np.polyfit(np.arange(n, dtype=np.float64), et, 1)[0]
    assert abs(slope * n) < 0.25 * et.std(), (slope * n, et.std())
    assert et.max() - et.min() < 5e-3 * (ep.max() - ep.min())
    # the two halves of the run have the same mean energy within the fluctuation
    assert abs(et[: n // 2].mean() - et[n // 2:].mean()) < 0.25 * et.std()


def test_virial_matches_strain_derivative_cluster(small):
    """Non-periodic cluster: every component of dE/d(eps) by central differences of a
    homogeneous strain equals -W^T."""
    s = synth.cluster_system(10, seed=12)
    W = small.virial(s.pos, s.Z, s.box, s.pbc)[0]
    c = s.pos.mean(axis=0)
    h = 1e-5
    for a in range(3):
        for b in range(3):
            eps = np.zeros((3, 3))
            eps[a, b] = h
            Ep = small.evaluate((s.pos - c) @ (np.eye(3) + eps).T + c, s.Z, s.box, s.pbc,
                                forces=False)[0][0]
            Em = small.evaluate((s.pos - c) @ (np.eye(3) - eps).T + c, s.Z, s.box, s.pbc,
                                forces=False)[0][0]
            assert abs((Ep - Em) / (2 * h) + W[b, a]) < 1e-7, (a, b)
    np.testing.assert_allclose(W, W.T, atol=1e-10)      # rotation invariance


def test_virial_matches_box_strain_periodic(small, cfg1):
    """Periodic box: scaling one box edge together with the positions."""
    s = cfg1[0]
    W = small.virial(s.pos, s.Z, s.box, s.pbc)[0]
    h = 1e-5
    for a in range(3):
        sc = np.ones(3)
        sc[a] = 1 + h
        Ep = small.evaluate(s.pos * sc, s.Z, s.box * sc, s.pbc, forces=False)[0][0]
        sc[a] = 1 - h
        Em = small.evaluate(s.pos * sc, s.Z, s.box * sc, s.pbc, forces=False)[0][0]
        assert abs((Ep - Em) / (2 * h) + W[a, a]) < 1e-7, a


def test_nvt_conserved_quantity_scales_dt2_and_large_q_is_nve(small):
    s = synth.cluster_system(12, seed=8, radius=2.6)
    m = s.masses
    v0 = synth.maxwell_boltzmann(m, 900.0, seed=2)
    fl = []
    for dt, n in ((2.0, 20), (1.0, 40)):
        *_, H, _, _ = md.run_nvt(small, s.pos, v0, s.Z, s.box, s.pbc, m, dt, n, 300.0, 20.0)
        fl.append(H.max() - H.min())
    assert 3.0 < fl[0] / fl[1] < 5.0, fl
    # an infinitely heavy thermostat leaves the NVE trajectory
    x1, v1, ep1, ek1, *_ = md.run_nvt(small, s.pos, v0, s.Z, s.box, s.pbc, m, 1.0, 10, 300.0, 1e12)
    x2, v2, ep2, ek2 = md.run_nve(small, s.pos, v0, s.Z, s.box, s.pbc, m, 1.0, 10)
    np.testing.assert_allclose(x1, x2, atol=1e-12)
    np.testing.assert_allclose(v1, v2, atol=1e-12)


def test_nvt_drives_temperature_towards_target(small):
    """Nose-Hoover feedback sign: a cold start (50 K) under a 600 K thermostat heats up,
    a hot start (6000 K) under a 300 K thermostat cools down."""
    s = synth.cluster_system(12, seed=8, radius=2.6)
    m = s.masses
    v0 = synth.maxwell_boltzmann(m, 50.0, seed=2)
    *_, ek, H, xi, _ = md.run_nvt(small, s.pos, v0, s.Z, s.box, s.pbc, m, 1.0, 30, 600.0, 10.0)
    assert ek.max() > 2.0 * md.kinetic(v0, m)
    v1 = synth.maxwell_boltzmann(m, 6000.0, seed=2)
    *_, ek, H, xi, _ = md.run_nvt(small, s.pos, v1, s.Z, s.box, s.pbc, m, 1.0, 30, 300.0, 10.0)
    assert ek.min() < 0.5 * md.kinetic(v1, m)


def test_readout_scale_bounds_the_edge_energies():
    """The readout scale sum_j sum_d |x_ijd w_d| bounds sum_j |E_ij| (triangle inequality,
    E_ij = sum_d x_ijd w_d for the linear readout) and hence |E_i|; it is positive for an
    atom with edges and zero for an isolated one."""
    hp = synth.preset("small")
    s = synth.config1_system()
    model = Allegro64(hp, 42)
    atoms = [0, 5, 17, 42]
    sc = model.readout_scale(s.pos, s.Z, s.box, s.pbc, atoms)
    terms = model.centre_terms(s.pos, s.Z, s.box, s.pbc, atoms)
    for a in atoms:
        assert sc[a] > 0 and abs(terms[a][0]) <= sc[a]
    iso = np.array([[0.0, 0.0, 0.0], [20.0, 20.0, 20.0]])
    sc2 = model.readout_scale(iso, np.array([1, 8]), np.array([40.0, 40.0, 40.0]),
                              np.array([False, False, False]), [0, 1])
    assert sc2[0] == 0.0 and sc2[1] == 0.0

