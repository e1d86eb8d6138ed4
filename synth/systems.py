"""Seeded synthetic systems shaped like the workloads of Allegro-FM (arXiv 2502.06073).

The paper's own systems (tobermorite, C-S-H nanoparticles in H2O/CO2, organic molecules;
Results and Methodology/MD) and its datasets are not available, so every input here is a
seeded stand-in with the shape, density and species mix of those workloads.  This module
holds no arithmetic of the potential itself: it only draws positions, species, boxes,
masses and Maxwell-Boltzmann velocities.  Both the CUDA path's tests/benchmarks and the
FP64 oracle take their inputs from here.

Conventions: Angstrom, amu, fs.  Positions are returned as float64 arrays whose values are
exactly representable in float32 (the generators round them), so a float32 copy carries
the very same numbers.  Periodic positions are wrapped into [0, L).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Standard atomic masses (amu) of the elements used by the synthetic systems.
MASSES = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999, 14: 28.085, 20: 40.078}

# eV per K.
K_B = 8.617333262e-5
# 1 eV/amu expressed in (A/fs)^2.
EV_PER_AMU_A2_FS2 = 9.648533212e-3


@dataclasses.dataclass
class System:
    name: str
    pos: np.ndarray          # [n, 3] float64 (float32-exact values)
    Z: np.ndarray            # [n] int32, atomic numbers in 1..89
    box: np.ndarray          # [3] float64 orthorhombic edge lengths (binning extent if non-periodic)
    pbc: np.ndarray          # [3] bool
    sys_ptr: np.ndarray      # [n_sys + 1] int32 atom offsets of independent systems
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def masses(self) -> np.ndarray:
        return np.array([MASSES[int(z)] for z in self.Z], dtype=np.float64)


def _round_f32(pos: np.ndarray, box: np.ndarray, pbc: np.ndarray) -> np.ndarray:
    pos = np.array(pos, dtype=np.float64)
    for k in range(3):
        if pbc[k]:
            pos[:, k] = np.mod(pos[:, k], box[k])
    p32 = pos.astype(np.float32)
    for k in range(3):
        if pbc[k]:
            L32 = np.float32(box[k])
            col = p32[:, k]
            col[col >= L32] = np.float32(0.0)
            col[col < 0] = np.float32(0.0)
    return p32.astype(np.float64)


def lattice_system(name, n_xyz, spacing, n_atoms, species, seed, jitter=0.1, counts=None):
    """Atoms on a jittered simple-cubic/orthorhombic site lattice.

    n_xyz sites per axis with the given spacing fill a periodic box of n_xyz*spacing.
    n_atoms sites are drawn without replacement; species are either drawn uniformly from
    `species` (counts=None) or assigned from exact `counts` and shuffled over the sites.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = n_xyz
    box = np.array([nx * spacing, ny * spacing, nz * spacing], dtype=np.float64)
    n_sites = nx * ny * nz
    sites = rng.choice(n_sites, size=n_atoms, replace=False)
    sites.sort()
    ix = sites // (ny * nz)
    iy = (sites // nz) % ny
    iz = sites % nz
    pos = (np.stack([ix, iy, iz], axis=1).astype(np.float64) + 0.5) * spacing
    pos += rng.normal(0.0, jitter, size=pos.shape)
    if counts is None:
        Z = rng.choice(np.asarray(species), size=n_atoms)
    else:
        assert sum(counts) == n_atoms
        Z = np.concatenate([np.full(c, s) for s, c in zip(species, counts)])
        rng.shuffle(Z)
    pbc = np.array([True, True, True])
    pos = _round_f32(pos, box, pbc)
    return System(name, pos, Z.astype(np.int32), box, pbc,
                  np.array([0, n_atoms], dtype=np.int32),
                  dict(seed=seed, spacing=spacing, n_xyz=n_xyz, jitter=jitter))


def config1_system(seed=1000):
    """96 atoms, cubic 10 A periodic box, Z uniform over {1,6,8,14}, sigma=0.1 A jitter."""
    return lattice_system("cubic96", (5, 5, 5), 2.0, 96, [1, 6, 8, 14], seed)


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def water_system(n_mol=4096, L=None, seed=1001, density=1.0, d_min_oo=2.4):
    """Water-like fluid: n_mol H2O at `density` g/cm^3 in a periodic cube.

    Molecular (O) centres are uniform in the box, drawn by random sequential addition
    with an O-O exclusion distance d_min_oo; O-H lengths U(0.94, 0.98) A, H-O-H angles
    U(101.5, 107.5) deg, uniformly random orientations.
    """
    rng = np.random.default_rng(seed)
    m_h2o = 2 * MASSES[1] + MASSES[8]
    if L is None:
        # n * m [amu] / (L^3 [A^3]) = density [g/cm^3] / 1.66053907
        L = (n_mol * m_h2o / (density / 1.66053906660)) ** (1.0 / 3.0)
    ncell = max(1, int(L // d_min_oo))
    cw = L / ncell
    grid = {}
    centres = []
    attempts = 0
    while len(centres) < n_mol:
        attempts += 1
        if attempts > 200 * n_mol:
            raise RuntimeError("water packing failed")
        p = rng.uniform(0.0, L, size=3)
        c = tuple((p // cw).astype(int) % ncell)
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = ((c[0] + dx) % ncell, (c[1] + dy) % ncell, (c[2] + dz) % ncell)
                    for q in grid.get(key, ()):
                        d = p - q
                        d -= L * np.round(d / L)
                        if d @ d < d_min_oo * d_min_oo:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            grid.setdefault(c, []).append(p)
            centres.append(p)
    centres = np.array(centres)
    pos = np.zeros((3 * n_mol, 3))
    Z = np.zeros(3 * n_mol, dtype=np.int32)
    for m in range(n_mol):
        r1, r2 = rng.uniform(0.94, 0.98, size=2)
        th = math.radians(rng.uniform(101.5, 107.5))
        R = _random_rotation(rng)
        a = R @ np.array([1.0, 0.0, 0.0])
        b = R @ np.array([math.cos(th), math.sin(th), 0.0])
        pos[3 * m] = centres[m]
        pos[3 * m + 1] = centres[m] + r1 * a
        pos[3 * m + 2] = centres[m] + r2 * b
        Z[3 * m:3 * m + 3] = (8, 1, 1)
    box = np.array([L, L, L])
    pbc = np.array([True, True, True])
    pos = _round_f32(pos, box, pbc)
    return System(f"water{3 * n_mol}", pos, Z, box, pbc,
                  np.array([0, 3 * n_mol], dtype=np.int32), dict(seed=seed, L=L))


def csh_system(sub=False, seed=1002):
    """Calcium-silicate-hydrate-like solid at 2.6 g/cm^3 (Ca:Si:O:H = 1.7:1:5.4:2.6).

    Full: 131,072 atoms on a 32x64x64 site lattice with spacing 2.228 A.
    Sub-box: a separate periodic 8x8x8 lattice (512 atoms, L = 17.82 A).
    """
    if sub:
        return lattice_system("csh512", (8, 8, 8), 2.228, 512, [20, 14, 8, 1], seed,
                              counts=[81, 48, 258, 125])
    return lattice_system("csh131072", (32, 64, 64), 2.228, 131072, [20, 14, 8, 1], seed,
                          counts=[20825, 12250, 66148, 31849])


def sio2_system(n_side=162, n_atoms=4194304, seed=1004):
    """SiO2-like amorphous solid at 2.2 g/cm^3: sites of an n_side^3 lattice (2.461 A)."""
    n_si = n_atoms // 3
    n_o = n_atoms - n_si
    return lattice_system(f"sio2_{n_atoms}", (n_side,) * 3, 2.4614, n_atoms, [14, 8], seed,
                          counts=[n_si, n_o])


def molecules_system(n_mol=1024, seed=1003, noise=0.05):
    """Independent organic molecules (non-periodic), built by seeded random bonded growth.

    Heavy atoms k ~ U{7..23}, each uniformly C/N/O; each new heavy atom bonds to a random
    heavy atom with free valence (C 4, N 3, O 2) at a length U(1.0, 1.5) A, rejected if
    closer than 1.0 A to a non-bonded atom; then H atoms fill the remaining valences with
    the same rule, and all atoms receive N(0, noise) displacements.  Molecules are stored
    one after the other (sys_ptr) with local coordinates; they never interact.
    """
    rng = np.random.default_rng(seed)
    valence = {6: 4, 7: 3, 8: 2}
    all_pos, all_Z, ptr = [], [], [0]

    def place(pos_list, parent, exclude_parent=True):
        for _ in range(200):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            p = pos_list[parent] + rng.uniform(1.0, 1.5) * d
            ok = True
            for q_i, q in enumerate(pos_list):
                if q_i == parent:
                    continue
                if np.linalg.norm(p - q) < 1.0:
                    ok = False
                    break
            if ok:
                return p
        return None

    for _ in range(n_mol):
        k = int(rng.integers(7, 24))
        zs = [int(rng.choice([6, 7, 8]))]
        ps = [np.zeros(3)]
        free = [valence[zs[0]]]
        while len(zs) < k:
            cand = [a for a in range(len(zs)) if free[a] > 0]
            parent = int(rng.choice(cand))
            z = int(rng.choice([6, 7, 8]))
            p = place(ps, parent)
            if p is None:
                continue
            zs.append(z)
            ps.append(p)
            free[parent] -= 1
            free.append(valence[z] - 1)
        n_heavy = len(zs)
        for a in range(n_heavy):
            for _h in range(free[a]):
                p = place(ps, a)
                if p is None:
                    continue
                zs.append(1)
                ps.append(p)
        ps = np.array(ps) + rng.normal(0.0, noise, size=(len(ps), 3))
        all_pos.append(ps)
        all_Z.extend(zs)
        ptr.append(ptr[-1] + len(zs))
    pos = np.concatenate(all_pos).astype(np.float32).astype(np.float64)
    extent = pos.max(axis=0) - pos.min(axis=0) + 1.0
    return System(f"molecules{n_mol}", pos, np.array(all_Z, dtype=np.int32), extent,
                  np.array([False, False, False]), np.array(ptr, dtype=np.int32),
                  dict(seed=seed))


def nanoparticle_mixture_system(seed=1005):
    """Stand-in for the paper's reactive MD system (Methodology, MD Simulations of C-S-H
    Nanoparticle Reaction): 6,326 atoms -- 267 C, 90 Ca, 133 Si, 2,577 O, 3,259 H -- in a
    periodic (45.7 A)^3 box, a C-S-H nanoparticle immersed in H2O and CO2.

    Reading of the composition (the paper gives only the totals): all carbon is CO2 (267
    molecules), the particle has Ca 90, Si 133 and the C-S-H ratio O/Si = 5.4 (718 O), the
    rest of the oxygen is water (1,325 H2O) and the rest of the hydrogen (609) sits in
    the particle.  The particle is a sphere of jittered lattice sites (2.228 A, the C-S-H
    density) at the box centre; molecule centres are placed outside it by random
    sequential addition (2.6 A exclusion), with random orientations.
    """
    rng = np.random.default_rng(seed)
    L = 45.7
    box = np.array([L, L, L])
    n_np = {20: 90, 14: 133, 8: 718, 1: 609}
    n_co2, n_h2o = 267, 1325
    # particle: the sum(n_np) lattice sites closest to the centre
    sp = 2.228
    k = int(np.ceil(L / sp))
    g = (np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij"), -1)
         .reshape(-1, 3) + 0.5) * sp
    c = np.array([L / 2] * 3)
    d = np.linalg.norm(g - c, axis=1)
    n_p = sum(n_np.values())
    sites = g[np.argsort(d, kind="stable")[:n_p]]
    r_np = np.linalg.norm(sites - c, axis=1).max()
    p_pos = sites + rng.normal(0.0, 0.1, size=sites.shape)
    p_Z = np.concatenate([np.full(v, z) for z, v in n_np.items()])
    rng.shuffle(p_Z)
    # fluid molecules by random sequential addition outside the particle
    kinds = np.array([0] * n_co2 + [1] * n_h2o)
    rng.shuffle(kinds)
    centres = []
    dmin = 2.6
    ncell = int(L // dmin)
    cw = L / ncell
    grid = {}
    for _ in kinds:
        for _try in range(10000):
            p = rng.uniform(0.0, L, size=3)
            dc = p - c
            dc -= L * np.round(dc / L)
            if np.linalg.norm(dc) < r_np + 1.8:
                continue
            cc = tuple((p // cw).astype(int) % ncell)
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for q in grid.get(((cc[0] + dx) % ncell, (cc[1] + dy) % ncell,
                                           (cc[2] + dz) % ncell), ()):
                            dd = p - q
                            dd -= L * np.round(dd / L)
                            if dd @ dd < dmin * dmin:
                                ok = False
            if ok:
                grid.setdefault(cc, []).append(p)
                centres.append(p)
                break
        else:
            raise RuntimeError("fluid packing failed")
    f_pos, f_Z = [], []
    for kind, p in zip(kinds, centres):
        R = _random_rotation(rng)
        if kind == 0:       # CO2: O=C=O, 1.16 A
            ax = R @ np.array([1.0, 0.0, 0.0])
            f_pos += [p, p + 1.16 * ax, p - 1.16 * ax]
            f_Z += [6, 8, 8]
        else:               # H2O
            r1, r2 = rng.uniform(0.94, 0.98, size=2)
            th = math.radians(rng.uniform(101.5, 107.5))
            f_pos += [p, p + r1 * (R @ np.array([1.0, 0.0, 0.0])),
                      p + r2 * (R @ np.array([math.cos(th), math.sin(th), 0.0]))]
            f_Z += [8, 1, 1]
    pos = np.concatenate([p_pos, np.array(f_pos)])
    Z = np.concatenate([p_Z, np.array(f_Z)]).astype(np.int32)
    pbc = np.array([True, True, True])
    pos = _round_f32(pos, box, pbc)
    return System("csh_np6326", pos, Z, box, pbc, np.array([0, pos.shape[0]], dtype=np.int32),
                  dict(seed=seed, n_particle=n_p, r_particle=float(r_np)))


def dimer_system(r, Zi=8, Zj=1, direction=(1.0, 0.0, 0.0), L=None):
    """Two atoms at distance r along `direction`; non-periodic unless L is given."""
    d = np.asarray(direction, dtype=np.float64)
    d /= np.linalg.norm(d)
    pos = np.array([[0.0, 0.0, 0.0], r * d])
    if L is None:
        box = np.array([20.0, 20.0, 20.0])
        pbc = np.array([False, False, False])
        pos = pos + 10.0
    else:
        box = np.array([L, L, L])
        pbc = np.array([True, True, True])
        pos = np.mod(pos + 0.5 * L, L)
    return System("dimer", pos, np.array([Zi, Zj], dtype=np.int32), box, pbc,
                  np.array([0, 2], dtype=np.int32))


def cluster_system(n=12, seed=7, radius=3.0, species=(1, 6, 8, 14), d_min=1.0):
    """A compact non-periodic cluster (for rotation/reflection tests), float32-exact."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.uniform(-radius, radius, size=3)
        if np.linalg.norm(p) > radius:
            continue
        if all(np.linalg.norm(p - q) >= d_min for q in pts):
            pts.append(p)
    pos = np.array(pts).astype(np.float32).astype(np.float64)
    Z = rng.choice(np.asarray(species), size=n).astype(np.int32)
    return System("cluster", pos, Z, np.array([2 * radius + 2] * 3),
                  np.array([False, False, False]), np.array([0, n], dtype=np.int32))


def maxwell_boltzmann(masses, T, seed):
    """Velocities (A/fs) drawn at temperature T (K) with zero centre-of-mass momentum."""
    rng = np.random.default_rng(seed)
    m = np.asarray(masses, dtype=np.float64)
    sd = np.sqrt(K_B * T / m * EV_PER_AMU_A2_FS2)
    v = rng.normal(size=(m.shape[0], 3)) * sd[:, None]
    p = (m[:, None] * v).sum(axis=0)
    v -= p / m.sum()
    return v


def bench_workloads():
    """Named synthetic workloads with their model preset and seeds."""
    return {
        "cubic96": dict(make=lambda: config1_system(1000), model="small"),
        "water12288": dict(make=lambda: water_system(4096, L=49.67, seed=1001), model="fm_water"),
        "water4095": dict(make=lambda: water_system(1365, L=34.44, seed=1001), model="fm_water"),
        "csh131072": dict(make=lambda: csh_system(False, 1002), model="fm_water"),
        "csh512": dict(make=lambda: csh_system(True, 1002), model="fm_water"),
        "molecules1024": dict(make=lambda: molecules_system(1024, 1003), model="fm_water"),
        "csh_np6326": dict(make=lambda: nanoparticle_mixture_system(1005), model="fm_water"),
        "sio2_4194304": dict(make=lambda: sio2_system(162, 4194304, 1004), model="fm_water"),
        "sio2_4096": dict(make=lambda: sio2_system(16, 4096, 1004), model="fm_water"),
    }
