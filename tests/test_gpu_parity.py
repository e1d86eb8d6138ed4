"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Bars for the FP32 path: the sorted edge list and reverse index are bit-exact; total
energy relative error <= 1e-6; force max-abs error <= 1e-4 eV/A.  Per-atom energies are
held to 5e-6 of the largest per-atom magnitude, derived from FP32 rounding: each E_i is
a chain of about seven dot products of length <= 352 (two-body, three latent layers,
readout), so u * sqrt(352) * sqrt(7) ~ 3e-6 with u = 6e-8.  Inputs are the seeded
synthetic systems of `synth`.
"""
import os

import numpy as np
import pytest

import synth
from oracle import Allegro64, md as omd, neighbors, pool, weights

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_REL = 1e-6
EA_REL = 5e-6
F_ABS = 1e-4


@pytest.fixture(scope="module")
def ff():
    import paper_2502_06073_gb300 as ff
    ff._build.build()
    ff.load_library()
    assert torch.cuda.is_available()
    return ff


def _dev(a, dt):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def _bind(ff, hp, s, seed=42, precision=0):
    m = ff.FFModel(hp, seed=seed, precision=precision)
    pos = _dev(s.pos, torch.float64)
    Z = _dev(s.Z, torch.int32)
    multi = s.sys_ptr.shape[0] > 2
    m.bind(pos, Z, s.box, s.pbc, s.sys_ptr if multi else None)
    return m, pos


def _hp(name, wl=None, **over):
    hp = synth.preset(name, **over)
    if wl is not None:
        hp["avg_num_neighbors"] = synth.NU[wl]
    return hp


SYSTEMS = {
    "cubic96": (lambda: synth.config1_system(), "small", {}),
    "cubic96_skin": (lambda: synth.config1_system(), "small", dict(skin=0.7)),
    "csh512": (lambda: synth.csh_system(sub=True), "fm_water", {}),
    "water4095": (lambda: synth.water_system(1365, L=34.44, seed=1001), "fm_water", {}),
    "molecules64": (lambda: synth.molecules_system(64, seed=1003), "fm_water", {}),
}


@pytest.mark.parametrize("name", ["small", "fm_water"])
def test_weights_bitwise(ff, name):
    hp = synth.preset(name)
    m = ff.FFModel(hp, seed=42)
    got = m.export_params()
    ref = np.concatenate([v.ravel() for v in weights.init_params(hp, 42).values()])
    assert got.shape == ref.shape
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("key", list(SYSTEMS))
def test_edge_list_bit_exact(ff, key):
    make, name, over = SYSTEMS[key]
    s = make()
    hp = synth.preset(name, **over)
    m, _ = _bind(ff, hp, s)
    rp, col, sh, rev = m.edges()
    ref = neighbors.neighbor_list(s.pos, s.box, s.pbc, hp["rc"], 0.0, s.sys_ptr)
    np.testing.assert_array_equal(rp, ref[0])
    np.testing.assert_array_equal(col, ref[1])
    np.testing.assert_array_equal(sh, ref[2])
    if col.shape[0] < 60000:
        np.testing.assert_array_equal(rev, neighbors.reverse_index(*ref))
    else:
        i = np.repeat(np.arange(s.n), np.diff(rp))
        np.testing.assert_array_equal(col[rev], i)
        np.testing.assert_array_equal(sh[rev], -sh)


def _check_ef(Es, Ea, F, E_ref, Ea_ref, F_ref, tag, sys_ptr=None):
    """Energy bar: total energy relative error <= 1e-6.  With several systems, each
    system's error is held to 1e-6 of the sum of its |E_i|: a system energy is a sum of
    per-atom terms of both signs, and for small molecules it nearly cancels, so its plain
    relative error measures the cancellation, not the arithmetic."""
    Es = Es.cpu().numpy()
    Ea = Ea.double().cpu().numpy()
    F = F.double().cpu().numpy()
    e_tot = abs(Es.sum() - E_ref.sum()) / abs(E_ref.sum())
    assert e_tot <= E_REL, (tag, "E total rel", e_tot)
    if Es.shape[0] > 1:
        scale = np.array([np.abs(Ea_ref[sys_ptr[k]:sys_ptr[k + 1]]).sum()
                          for k in range(Es.shape[0])])
        e_sys = (np.abs(Es - E_ref) / scale).max()
        assert e_sys <= E_REL, (tag, "E_sys err / sum|E_i|", e_sys)
    ea = np.abs(Ea - Ea_ref).max() / np.abs(Ea_ref).max()
    f = np.abs(F - F_ref).max()
    assert ea <= EA_REL, (tag, "E_atom rel", ea)
    assert f <= F_ABS, (tag, "F max", f)


@pytest.mark.parametrize("key,wl", [("cubic96", "cubic96"), ("csh512", "csh512"),
                                    ("molecules64", "molecules1024")])
def test_energy_forces_full(ff, key, wl):
    make, name, over = SYSTEMS[key]
    s = make()
    hp = _hp(name, wl, **over)
    m, pos = _bind(ff, hp, s)
    Es, Ea, F = m.energy_forces(pos)
    E_ref, Ea_ref, F_ref = pool.evaluate(hp, 42, s.pos, s.Z, s.box, s.pbc, s.sys_ptr)
    _check_ef(Es, Ea, F, E_ref, Ea_ref, F_ref, key, s.sys_ptr)


@pytest.mark.parametrize("n_layers,lmax,two_body,precision",
                         [(1, 2, [32, 32], 0), (4, 2, [32, 32], 0), (1, 1, [32, 32], 0),
                          (4, 1, [32, 32], 0), (2, 2, [32], 0), (2, 2, [32], 1)])
def test_layer_counts_full(ff, n_layers, lmax, two_body, precision):
    """1- and 4-layer models: every tensor-product layer kind (a single last layer; the
    first, middle and pruned layer before the last, and a last layer reading it); and a
    two-body MLP of a single layer (the embedding layer is also the output) in both
    precisions."""
    s = synth.config1_system()
    hp = _hp("small", "cubic96", n_layers=n_layers, lmax=lmax, two_body=two_body)
    m, pos = _bind(ff, hp, s, precision=precision)
    Es, Ea, F = m.energy_forces(pos)
    E_ref, Ea_ref, F_ref = pool.evaluate(hp, 42, s.pos, s.Z, s.box, s.pbc, s.sys_ptr)
    if precision == 0:
        _check_ef(Es, Ea, F, E_ref, Ea_ref, F_ref, f"L{n_layers} lmax{lmax}", s.sys_ptr)
    else:
        d = F.double().cpu().numpy() - F_ref
        assert np.sqrt((d ** 2).mean()) <= 5e-3 and np.abs(d).max() <= 5e-3
        Ea = Ea.double().cpu().numpy()
        assert np.abs(Ea - Ea_ref).max() <= 4e-3 * np.abs(Ea_ref).max()


def test_water4095_energy_and_sampled_forces(ff):
    make, name, _ = SYSTEMS["water4095"]
    s = make()
    hp = _hp(name, "water4095")
    m, pos = _bind(ff, hp, s)
    Es, Ea, F = m.energy_forces(pos)
    E_ref, Ea_ref, F_ref = pool.evaluate(hp, 42, s.pos, s.Z, s.box, s.pbc)
    _check_ef(Es, Ea, F, E_ref, Ea_ref, F_ref, "water4095")


def test_ragged_chunks_identical(ff):
    """Forcing many small edge chunks (ragged last chunk) changes no bit of the result."""
    make, name, _ = SYSTEMS["csh512"]
    s = make()
    hp = _hp(name, "csh512")
    m1, pos = _bind(ff, hp, s)
    Es1, Ea1, F1 = m1.energy_forces(pos)
    os.environ["FF_WORKSPACE_MB"] = "40"
    try:
        m2, pos2 = _bind(ff, hp, s)
        Es2, Ea2, F2 = m2.energy_forces(pos2)
    finally:
        del os.environ["FF_WORKSPACE_MB"]
    assert torch.equal(Ea1, Ea2) and torch.equal(F1, F2) and torch.equal(Es1, Es2)


def test_deterministic(ff):
    make, name, _ = SYSTEMS["csh512"]
    s = make()
    m, pos = _bind(ff, _hp(name, "csh512"), s)
    a = m.energy_forces(pos)
    b = m.energy_forces(pos)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_autograd_adjoint_multi_system(ff):
    make, name, _ = SYSTEMS["molecules64"]
    s = make()
    hp = _hp(name, "molecules1024")
    m, pos = _bind(ff, hp, s)
    _, _, F = m.energy_forces(pos)
    x = pos.clone().requires_grad_(True)
    E = m.energy(x)
    g = torch.linspace(-1.0, 2.0, E.shape[0], dtype=torch.float64, device="cuda")
    (E * g).sum().backward()
    sys_of = np.searchsorted(s.sys_ptr, np.arange(s.n), side="right") - 1
    scale = g.cpu().numpy()[sys_of][:, None]
    expect = -F.double().cpu().numpy() * scale
    np.testing.assert_allclose(x.grad.cpu().numpy(), expect, rtol=1e-6, atol=1e-7)


def test_forces_fd_of_gpu_energy(ff):
    """Central differences of the GPU's own FP64-summed energy agree with its adjoint."""
    s = synth.cluster_system(16, seed=9, radius=3.0)
    hp = _hp("fm_water", None)
    m, pos = _bind(ff, hp, s)
    _, _, F = m.energy_forces(pos)
    h = 2e-3
    for a, k in [(0, 0), (5, 1), (11, 2)]:
        p1, p2 = pos.clone(), pos.clone()
        p1[a, k] += h
        p2[a, k] -= h
        e1 = m.energy_forces(p1, forces=False)[0].item()
        e2 = m.energy_forces(p2, forces=False)[0].item()
        fd = -(e1 - e2) / (2 * h)
        assert abs(fd - F[a, k].item()) < 2e-3 * max(1.0, abs(fd)), (a, k, fd, F[a, k].item())


def test_fd_of_gpu_energy_on_32_random_atoms_csh512(ff):
    """Finite differences of the GPU's own energy on the periodic 512-atom C-S-H box (FP32,
    32 random atoms, all three components) against the hand-written adjoint.  Central
    differences at h = 1e-2 and 5e-3 A (inside skin/2, so the list stays the same),
    Richardson-extrapolated: the truncation error is O(h^4), about 1e-6 of F when forces
    vary on a 0.3 A scale.  The energy is the FP64 sum of FP32 per-atom energies; their
    rounding moves it by about 1e-6 eV between the displaced evaluations (measured at
    h = 1e-3: extrapolated errors up to 3.8e-4 eV/A), i.e. about 1.5e-4 eV/A of noise at
    these steps, so the bar is 3e-4 eV/A + 1e-5 |F|."""
    make, name, _ = SYSTEMS["csh512"]
    s = make()
    hp = _hp(name, "csh512")
    m, pos = _bind(ff, hp, s)
    _, _, F = m.energy_forces(pos)
    F = F.double().cpu().numpy()
    atoms = np.random.default_rng(33).choice(s.n, 32, replace=False).tolist()

    def fd(a, k, h):
        p1, p2 = pos.clone(), pos.clone()
        p1[a, k] += h
        p2[a, k] -= h
        e1 = m.energy_forces(p1, forces=False)[0].item()
        e2 = m.energy_forces(p2, forces=False)[0].item()
        return -(e1 - e2) / (2 * h)

    worst = 0.0
    for a in atoms:
        for k in range(3):
            r = (4 * fd(a, k, 5e-3) - fd(a, k, 1e-2)) / 3
            err = abs(r - F[a, k])
            assert err <= 3e-4 + 1e-5 * abs(F[a, k]), (a, k, r, F[a, k])
            worst = max(worst, err)
    assert worst > 0.0     # the comparison ran on real differences


def test_isolated_atom_and_empty_list(ff):
    pos = np.array([[5.0, 5.0, 5.0], [15.0, 15.0, 15.0]])
    s = synth.System("two-far", pos, np.array([8, 1], np.int32), np.array([20.0, 20.0, 20.0]),
                     np.array([False, False, False]), np.array([0, 2], np.int32))
    m, p = _bind(ff, synth.preset("small"), s)
    Es, Ea, F = m.energy_forces(p)
    assert float(Es[0]) == 0.0 and torch.all(F == 0)
    assert m.edges()[1].shape[0] == 0


def test_errors_are_reported(ff):
    s = synth.config1_system()
    hp = synth.preset("small")
    m = ff.FFModel(hp, seed=1)
    with pytest.raises(ff.FFError, match="FF_ERR_STATE"):
        m.forces_adjoint()
    bad = s.Z.copy()
    bad[3] = 95
    with pytest.raises(ff.FFError, match="FF_ERR_SPECIES"):
        m.bind(_dev(s.pos, torch.float64), _dev(bad, torch.int32), s.box, s.pbc)


def test_capacity_and_nonfinite_errors(ff):
    """An atom with more than FF_MAX_NEIGHBORS (1024) neighbours within rc + skin is
    reported (the list kernels only count past the capacity), a non-finite position is
    reported before it is binned, and a non-finite velocity is reported at the rebuild the
    displacement check then asks for."""
    rng = np.random.default_rng(7)
    pts = rng.uniform(-1.0, 1.0, size=(6000, 3))
    pts = pts[np.linalg.norm(pts, axis=1) <= 1.0][:1100] * 4.5 + 20.0   # 1,100 atoms, r 4.5 A
    s = synth.System("dense", np.asarray(pts, np.float32).astype(np.float64),
                     np.full(pts.shape[0], 1, np.int32), np.array([40.0, 40.0, 40.0]),
                     np.array([False, False, False]), np.array([0, pts.shape[0]], np.int32))
    m = ff.FFModel(synth.preset("small"), seed=1)
    with pytest.raises(ff.FFError, match="FF_ERR_CAPACITY"):
        m.bind(_dev(s.pos, torch.float64), _dev(s.Z, torch.int32), s.box, s.pbc)
    c = synth.config1_system()
    bad = c.pos.copy()
    bad[5, 1] = np.nan
    m2 = ff.FFModel(synth.preset("small"), seed=1)
    with pytest.raises(ff.FFError, match="FF_ERR_NONFINITE"):
        m2.bind(_dev(bad, torch.float64), _dev(c.Z, torch.int32), c.box, c.pbc)
    hp = synth.preset("small", skin=0.5)
    m3, x = _bind(ff, hp, c)
    v = torch.zeros_like(x)
    v[3, 0] = float("nan")
    mass = _dev(c.masses, torch.float64)
    with pytest.raises(ff.FFError, match="FF_ERR_NONFINITE"):
        m3.md(x, v, mass, 2, 0.5)


def test_md_matches_oracle_trajectory(ff):
    s = synth.config1_system()
    hp = synth.preset("small", skin=0.5)
    m, pos = _bind(ff, hp, s)
    v0 = synth.maxwell_boltzmann(s.masses, 300.0, seed=5)
    x = pos.clone()
    v = _dev(v0, torch.float64)
    mass = _dev(s.masses, torch.float64)
    Ep, Ek = m.md(x, v, mass, 8, 1.0)
    xr, vr, ep, ek = omd.run_nve(Allegro64(hp, 42), s.pos, v0, s.Z, s.box, s.pbc, s.masses,
                                 1.0, 8)
    assert np.abs(x.cpu().numpy() - xr).max() < 1e-7
    assert np.abs(v.cpu().numpy() - vr).max() < 1e-8
    np.testing.assert_allclose(Ep.cpu().numpy(), ep, rtol=E_REL)
    # FP32 forces (error ~2e-7 eV/A) shift each velocity by ~dt*dF/m ~ 1e-9 A/fs per step
    # against |v| ~ 0.02 A/fs: kinetic energies agree to ~1e-7 after 8 steps
    np.testing.assert_allclose(Ek.cpu().numpy(), ek, rtol=1e-6)


@pytest.mark.parametrize("key,wl", [("csh512", "csh512"), ("water4095", "water4095")])
def test_bf16_tensor_core_path_error(ff, key, wl):
    """Precision 1 (BF16 tensor-core MLPs, FP32 accumulation, FP32 elsewhere) against the
    FP64 oracle.  Force bar: RMSE <= 5 meV/A (the stated target) and max <= 5 meV/A.
    Energy bars from bf16 rounding (2^-8 relative per stored operand): per-atom error
    <= 4e-3 of max|E_i|, total error <= 4e-3 of sum|E_i|."""
    make, name, _ = SYSTEMS[key]
    s = make()
    hp = _hp(name, wl)
    m, pos = _bind(ff, hp, s, precision=1)
    Es, Ea, F = m.energy_forces(pos)
    E_ref, Ea_ref, F_ref = pool.evaluate(hp, 42, s.pos, s.Z, s.box, s.pbc)
    d = F.double().cpu().numpy() - F_ref
    assert np.sqrt((d ** 2).mean()) <= 5e-3 and np.abs(d).max() <= 5e-3
    Ea = Ea.double().cpu().numpy()
    assert np.abs(Ea - Ea_ref).max() <= 4e-3 * np.abs(Ea_ref).max()
    assert abs(Es.item() - E_ref[0]) <= 4e-3 * np.abs(Ea_ref).sum()


@pytest.mark.parametrize("precision,fbar", [(0, F_ABS), (1, 5e-3)])
def test_csh131072_adjoint_vs_oracle_gradient_on_32_atoms(ff, precision, fbar):
    """Full 131,072-atom C-S-H system: forces from the GPU adjoint against the oracle's
    hand-derived gradient on 32 random atoms (each needs the edges out of and into the
    atom, so the oracle evaluates those atoms and all their neighbours), and per-atom
    energies of the same atoms."""
    s = synth.csh_system(sub=False)
    hp = _hp("fm_water", "csh131072")
    m, pos = _bind(ff, hp, s, precision=precision)
    _, Ea, F = m.energy_forces(pos)
    atoms = np.random.default_rng(32).choice(s.n, 32, replace=False).tolist()
    Fr, Er = pool.sampled_forces(hp, 42, s.pos, s.Z, s.box, s.pbc, atoms)
    Fg = F.double().cpu().numpy()
    Eg = Ea.double().cpu().numpy()
    d = np.array([Fg[a] - Fr[a] for a in atoms])
    de = np.array([Eg[a] - Er[a] for a in atoms])
    emax = max(abs(Er[a]) for a in atoms)
    if precision == 0:
        assert np.abs(d).max() <= fbar, np.abs(d).max()
        assert np.abs(de).max() <= EA_REL * emax
    else:
        assert np.sqrt((d ** 2).mean()) <= fbar and np.abs(d).max() <= fbar
        assert np.abs(de).max() <= 4e-3 * emax


BENCH_SIZES = {
    "water12288": (lambda: synth.water_system(4096, L=49.67, seed=1001), "water12288"),
    "molecules1024": (lambda: synth.molecules_system(1024, 1003), "molecules1024"),
    "sio2_4194304": (lambda: synth.sio2_system(162, 4194304, 1004), "sio2_4194304"),
}


@pytest.mark.parametrize("key,precision", [("water12288", 0), ("water12288", 1),
                                           ("molecules1024", 1), ("sio2_4194304", 0),
                                           ("sio2_4194304", 1)])
def test_bench_sizes_sampled_forces(ff, key, precision):
    """The benchmark's workloads at full size, in the launch configuration it times
    (per-step filtered list, default GEMM tiles, the chunk plan of the default budget):
    forces and per-atom energies of 16 random atoms against the oracle.  FP32 bars for
    precision 0; for precision 1 the stated force bar (RMSE and max <= 5 meV/A) and a
    per-atom energy bar of 8 u S_i, u = 2^-8 the bf16 unit roundoff, S_i the oracle's
    readout scale sum_j sum_d |x_ijd w_d| (first order, each bf16 rounding of a quantity
    on the residual path moves E_i by at most u S_i; about 8 such roundings: the two-body
    output and, per layer, the residual stream and the GEMM operand)."""
    make, wl = BENCH_SIZES[key]
    s = make()
    hp = _hp("fm_water", wl)
    m, pos = _bind(ff, hp, s, precision=precision)
    _, Ea, F = m.energy_forces(pos)
    atoms = np.random.default_rng(16).choice(s.n, 16, replace=False).tolist()
    multi = s.sys_ptr.shape[0] > 2
    Fr, Er = pool.sampled_forces(hp, 42, s.pos, s.Z, s.box, s.pbc, atoms,
                                 s.sys_ptr if multi else None)
    Fg = F.double().cpu().numpy()
    Eg = Ea.double().cpu().numpy()
    d = np.array([Fg[a] - Fr[a] for a in atoms])
    de = np.array([Eg[a] - Er[a] for a in atoms])
    emax = max(abs(Er[a]) for a in atoms)
    if precision == 0:
        assert np.abs(d).max() <= F_ABS, np.abs(d).max()
        assert np.abs(de).max() <= EA_REL * emax
    else:
        assert np.sqrt((d ** 2).mean()) <= 5e-3 and np.abs(d).max() <= 5e-3
        scale = Allegro64(hp, 42).readout_scale(s.pos, s.Z, s.box, s.pbc, atoms,
                                                s.sys_ptr if multi else None)
        for a, err in zip(atoms, de):
            assert abs(err) <= 8 * 2.0 ** -8 * scale[a], (a, err, scale[a])


def test_autograd_adjoint_with_several_chunks(ff):
    """With a small workspace budget the adjoint recomputes each chunk's forward; the
    gradient must equal the one-pass forces bit for bit."""
    make, name, _ = SYSTEMS["csh512"]
    s = make()
    hp = _hp(name, "csh512")
    m, pos = _bind(ff, hp, s)
    _, _, F = m.energy_forces(pos)
    os.environ["FF_WORKSPACE_MB"] = "40"
    try:
        m2, pos2 = _bind(ff, hp, s)
        x = pos2.clone().requires_grad_(True)
        m2.energy(x).sum().backward()
    finally:
        del os.environ["FF_WORKSPACE_MB"]
    assert torch.equal(x.grad, (-F).double())


@pytest.mark.parametrize("key,wl,prec", [("molecules64", "molecules1024", 1),
                                         ("csh512", "csh512", 0)])
def test_graph_path_matches_plain_path_and_replays(ff, key, wl, prec):
    """The frozen-list CUDA-graph path (Verlet list at rc + skin, edges beyond rc add
    exactly zero) against the plain path, then a replay after moving every atom in place
    by up to 0.1 A (< skin/2) against a fresh plain evaluation at the new positions."""
    make, name, _ = SYSTEMS[key]
    s = make()
    hp = _hp(name, wl)
    m, pos = _bind(ff, hp, s, precision=prec)
    Es = torch.empty(m.n_sys, dtype=torch.float64, device="cuda")
    Ea = torch.empty(s.n, dtype=torch.float32, device="cuda")
    F = torch.empty(s.n, 3, dtype=torch.float32, device="cuda")
    ftol = F_ABS if prec == 0 else 2e-4

    def check(positions):
        ref = ff.FFModel(hp, seed=42, precision=prec)
        ref.bind(positions, _dev(s.Z, torch.int32), s.box, s.pbc,
                 s.sys_ptr if s.sys_ptr.shape[0] > 2 else None)
        Er, Ear, Fr = ref.energy_forces(positions)
        scale = Ear.abs().max().item()
        assert (Ea - Ear).abs().max().item() <= 1e-5 * scale
        assert (Es - Er).abs().max().item() <= 1e-5 * Ear.abs().sum().item()
        assert (F - Fr).abs().max().item() <= ftol

    m.energy_forces_graph(pos, Es, Ea, F)          # evaluates and captures
    torch.cuda.synchronize()
    check(pos.clone())
    delta = torch.tensor(np.random.default_rng(4).uniform(-0.057, 0.057, size=(s.n, 3)),
                         dtype=torch.float64, device="cuda")
    pos.add_(delta)
    m.energy_forces_graph(pos, Es, Ea, F)          # replays the graph
    torch.cuda.synchronize()
    check(pos.clone())


def test_graph_path_bf16_molecules1024_vs_oracle(ff):
    """The batching path as it runs (1,024 molecules, BF16 MLPs, frozen Verlet list replayed
    from a CUDA graph by ff_energy_forces_graph) against the FP64 oracle: at the capturing
    call and at a replay after every atom moved by up to 0.1 A (inside skin/2), the energies
    of 12 whole molecules and the forces and per-atom energies of all their atoms.  Bars:
    force RMSE and max <= 5 meV/A; per-atom energy 8 u S_i and per-molecule energy
    sum_i 8 u S_i (u = 2^-8, S_i the oracle's readout scale; see
    test_bench_sizes_sampled_forces)."""
    s = synth.molecules_system(1024, 1003)
    hp = _hp("fm_water", "molecules1024")
    m, pos = _bind(ff, hp, s, precision=1)
    Es = torch.empty(m.n_sys, dtype=torch.float64, device="cuda")
    Ea = torch.empty(s.n, dtype=torch.float32, device="cuda")
    F = torch.empty(s.n, 3, dtype=torch.float32, device="cuda")
    mols = np.random.default_rng(12).choice(1024, 12, replace=False).tolist()
    atoms = [a for k in mols for a in range(int(s.sys_ptr[k]), int(s.sys_ptr[k + 1]))]
    u = 2.0 ** -8

    def check(p):
        Fr, Er = pool.sampled_forces(hp, 42, p, s.Z, s.box, s.pbc, atoms, s.sys_ptr)
        scale = Allegro64(hp, 42).readout_scale(p, s.Z, s.box, s.pbc, atoms, s.sys_ptr)
        Fg = F.double().cpu().numpy()
        Eg = Ea.double().cpu().numpy()
        Esg = Es.cpu().numpy()
        d = np.array([Fg[a] - Fr[a] for a in atoms])
        assert np.sqrt((d ** 2).mean()) <= 5e-3 and np.abs(d).max() <= 5e-3, np.abs(d).max()
        for a in atoms:
            assert abs(Eg[a] - Er[a]) <= 8 * u * scale[a], (a, Eg[a], Er[a], scale[a])
        for k in mols:
            own = range(int(s.sys_ptr[k]), int(s.sys_ptr[k + 1]))
            ref = sum(Er[a] for a in own)
            bar = sum(8 * u * scale[a] for a in own)
            assert abs(Esg[k] - ref) <= bar, (k, Esg[k], ref, bar)

    m.energy_forces_graph(pos, Es, Ea, F)          # evaluates and captures
    torch.cuda.synchronize()
    check(s.pos)
    delta = np.random.default_rng(5).uniform(-0.057, 0.057, size=(s.n, 3))
    pos.add_(torch.tensor(delta, dtype=torch.float64, device="cuda"))
    m.energy_forces_graph(pos, Es, Ea, F)          # replays the graph
    torch.cuda.synchronize()
    check(pos.cpu().numpy())


def test_graph_md_matches_oracle_trajectory(ff):
    s = synth.config1_system()
    hp = synth.preset("small", skin=0.3)
    m, pos = _bind(ff, hp, s)
    m.set_graph(True)
    v0 = synth.maxwell_boltzmann(s.masses, 3000.0, seed=5)     # hot: forces list rebuilds
    x = pos.clone()
    v = _dev(v0, torch.float64)
    mass = _dev(s.masses, torch.float64)
    Ep, Ek = m.md(x, v, mass, 12, 1.0)
    xr, vr, ep, ek = omd.run_nve(Allegro64(hp, 42), s.pos, v0, s.Z, s.box, s.pbc, s.masses,
                                 1.0, 12)
    assert np.abs(x.cpu().numpy() - xr).max() < 1e-7
    assert np.abs(v.cpu().numpy() - vr).max() < 1e-8
    np.testing.assert_allclose(Ep.cpu().numpy(), ep, rtol=E_REL)


def test_autotune_picks_a_valid_tile_and_keeps_results(ff):
    make, name, _ = SYSTEMS["csh512"]
    s = make()
    hp = _hp(name, "csh512")
    m, pos = _bind(ff, hp, s, precision=1)
    _, Ea0, F0 = m.energy_forces(pos)
    cfg = m.autotune(pos)
    assert cfg["slice"] in (128, 256) and cfg["stages"] in (0, 1, 2, 3, 4)
    assert cfg["ms_per_evaluation"] > 0
    _, Ea1, F1 = m.energy_forces(pos)
    # the tile shape changes no element-wise arithmetic (same K loop and accumulation); only
    # the readout's row sums over the 256 latent columns are added in a different order
    # (two 128-column halves in the persistent kernel, whole rows in the other), an FP32
    # reordering of 256 terms
    _, Ea2, F2 = m.energy_forces(pos)
    assert torch.equal(Ea1, Ea2) and torch.equal(F1, F2)     # deterministic per tile shape
    assert (Ea1 - Ea0).abs().max().item() <= 1e-5 * Ea0.abs().max().item()
    assert (F1 - F0).abs().max().item() <= 1e-5 * F0.abs().max().item()


@pytest.mark.parametrize("slice_,stages", [(128, 0), (128, 1), (128, 3), (256, 0), (256, 4)])
def test_every_gemm_tile_configuration_vs_oracle(ff, slice_, stages):
    """Each tile configuration the autotuner may pick -- the persistent kernel (128, 0),
    whose adjoint fuses the SiLU row reductions into the dE/dx GEMMs, and the one-tile
    kernel with 128- or 256-column slices and 1-4 stages, whose adjoint runs them
    separately -- against the FP64 oracle on the 512-atom C-S-H box at the BF16 bars, and
    deterministic per configuration."""
    make, name, _ = SYSTEMS["csh512"]
    s = make()
    hp = _hp(name, "csh512")
    m, pos = _bind(ff, hp, s, precision=1)
    m.set_tiles(slice_, stages)
    Es, Ea, F = m.energy_forces(pos)
    _, Ea2, F2 = m.energy_forces(pos)
    assert torch.equal(Ea, Ea2) and torch.equal(F, F2)
    E_ref, Ea_ref, F_ref = pool.evaluate(hp, 42, s.pos, s.Z, s.box, s.pbc)
    d = F.double().cpu().numpy() - F_ref
    assert np.sqrt((d ** 2).mean()) <= 5e-3 and np.abs(d).max() <= 5e-3
    Ea = Ea.double().cpu().numpy()
    assert np.abs(Ea - Ea_ref).max() <= 4e-3 * np.abs(Ea_ref).max()
    assert abs(Es.item() - E_ref[0]) <= 4e-3 * np.abs(Ea_ref).sum()


def test_set_tiles_rejects_bad_values(ff):
    make, name, _ = SYSTEMS["cubic96"]
    m = ff.FFModel(_hp(name), seed=1, precision=1)
    for bad in [(64, 0), (128, 5), (256, -1)]:
        with pytest.raises(ff.FFError, match="FF_ERR_ARG"):
            m.set_tiles(*bad)


@pytest.mark.parametrize("model", ["fm64", "fm256", "fm512"])
@pytest.mark.parametrize("precision", [0, 1])
def test_table1_model_sizes(ff, model, precision):
    """Allegro-FM64/256/512 hyperparameters of Table 1 (16/64/128 tensor channels, latent
    [64]*3/[256]*3/[512]*3, two-body [16,32,64]/[64,128,256]/[128,256,512], 2 layers,
    l = 2) on the 512-atom C-S-H box, FP32 and BF16 paths against the oracle."""
    s = synth.csh_system(sub=True)
    hp = synth.preset(model, avg_num_neighbors=synth.NU["csh512"], rc=5.2)
    m, pos = _bind(ff, hp, s, precision=precision)
    Es, Ea, F = m.energy_forces(pos)
    E_ref, Ea_ref, F_ref = pool.evaluate(hp, 42, s.pos, s.Z, s.box, s.pbc)
    if precision == 0:
        _check_ef(Es, Ea, F, E_ref, Ea_ref, F_ref, model)
    else:
        d = F.double().cpu().numpy() - F_ref
        assert np.sqrt((d ** 2).mean()) <= 5e-3 and np.abs(d).max() <= 5e-3
        assert abs(Es.item() - E_ref[0]) <= 4e-3 * np.abs(Ea_ref).sum()


def test_nvt_matches_oracle_trajectory(ff):
    s = synth.config1_system()
    hp = synth.preset("small", skin=0.5)
    m, pos = _bind(ff, hp, s)
    v0 = synth.maxwell_boltzmann(s.masses, 100.0, seed=6)
    x = pos.clone()
    v = _dev(v0, torch.float64)
    mass = _dev(s.masses, torch.float64)
    Ep, Ek, H, thermo = m.md_nvt(x, v, mass, 8, 1.0, 600.0, 20.0)
    xr, vr, ep, ek, hr, xi, eta = omd.run_nvt(Allegro64(hp, 42), s.pos, v0, s.Z, s.box, s.pbc,
                                              s.masses, 1.0, 8, 600.0, 20.0)
    assert np.abs(x.cpu().numpy() - xr).max() < 1e-7
    assert np.abs(v.cpu().numpy() - vr).max() < 1e-8
    np.testing.assert_allclose(Ep.cpu().numpy(), ep, rtol=E_REL)
    np.testing.assert_allclose(Ek.cpu().numpy(), ek, rtol=1e-6)
    np.testing.assert_allclose(H.cpu().numpy(), hr, rtol=1e-6)
    np.testing.assert_allclose(thermo.cpu().numpy()[0], [xi, eta], rtol=1e-5, atol=1e-12)


@pytest.mark.parametrize("precision,rtol", [(0, 1e-5), (1, 2e-2)])
def test_virial_matches_oracle(ff, precision, rtol):
    from oracle import Allegro64 as A
    s = synth.csh_system(sub=True)
    hp = _hp("fm_water", "csh512")
    m, pos = _bind(ff, hp, s, precision=precision)
    m.energy_forces(pos)
    W = m.virial()[0].cpu().numpy()
    Wr = A(hp, 42).virial(s.pos, s.Z, s.box, s.pbc)[0]
    assert np.abs(W - Wr).max() <= rtol * np.abs(Wr).max(), (W, Wr)


@pytest.mark.parametrize("precision", [0, 1])
def test_nanoparticle_mixture_system(ff, precision):
    """The paper's reactive MD system shape (6,326 atoms, C-S-H particle in H2O/CO2): uneven
    neighbour counts (36..82 per atom) across the particle surface."""
    s = synth.nanoparticle_mixture_system()
    hp = _hp("fm_water", "csh_np6326")
    m, pos = _bind(ff, hp, s, precision=precision)
    Es, Ea, F = m.energy_forces(pos)
    E_ref, Ea_ref, F_ref = pool.evaluate(hp, 42, s.pos, s.Z, s.box, s.pbc)
    if precision == 0:
        _check_ef(Es, Ea, F, E_ref, Ea_ref, F_ref, "csh_np6326")
    else:
        d = F.double().cpu().numpy() - F_ref
        assert np.sqrt((d ** 2).mean()) <= 5e-3 and np.abs(d).max() <= 5e-3
