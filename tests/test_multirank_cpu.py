"""Multi-process (gloo, CPU) checks of how the path shards.

Strict locality (Abstract: "strictly-local") lets disjoint sets of centre atoms be
evaluated independently: each rank computes the energies of its centres and the edge
gradients of their edges, scatters them into a force array (F_i += g_e, F_j -= g_e) and
one all-reduce sums the ranks.  The result must equal the single-process evaluation.
The benchmark's replica mode is checked too: the timed value uses the maximum time over
ranks and every rank's atoms.

The spatial decomposition that a multi-GPU run would use (the paper's billion-atom runs
scale this way; Abstract, Methodology, MD Simulations) is checked with bricks: the
periodic box is cut into slabs along one axis, one per rank; a rank starts with its own
atoms only, receives in a halo exchange (point-to-point, both neighbours) the atoms of
the adjacent slabs within a halo of rc + skin of its slab, evaluates the energies and
edge gradients of its own centres on that local set (same periodic box, so every edge
and its float32 membership test are the whole box's), and sends the forces that landed
on ghost atoms back to their owners (reverse exchange).  Energies and forces of the
owned atoms must equal the whole-box evaluation.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth
    from oracle import Allegro64
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    hp = synth.preset("small")
    s = synth.config1_system()
    model = Allegro64(hp, 42)
    mine = list(range(rank, s.n, world))                       # interleaved centre atoms
    terms = model.centre_terms(s.pos, s.Z, s.box, s.pbc, mine)
    F = np.zeros((s.n, 3))
    E = 0.0
    for i, (Ei, col, _sh, g) in terms.items():
        E += Ei
        if g.shape[0]:
            F[i] += g.sum(axis=0)
            np.add.at(F, col, -g)
    Ft = torch.tensor(F)
    Et = torch.tensor([E], dtype=torch.float64)
    dist.all_reduce(Ft)
    dist.all_reduce(Et)
    # replica timing reduction of bench.py: max over ranks, whole-job atoms
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        np.savez(out_path, F=Ft.numpy(), E=Et.numpy(), t=t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_centre_decomposition_matches_single_process(tmp_path):
    import synth
    from oracle import Allegro64
    out = str(tmp_path / "ranks.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    res = np.load(out)
    s = synth.config1_system()
    E, _, F = Allegro64(synth.preset("small"), 42).evaluate(s.pos, s.Z, s.box, s.pbc)
    np.testing.assert_allclose(res["F"], F, atol=1e-13)
    assert abs(res["E"][0] - E[0]) < 1e-12
    assert res["t"][0] == 2.0


def _brick_worker(rank, world, port, axis, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth
    from oracle import Allegro64, neighbors
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    hp = synth.preset("small", skin=1.0)
    halo = hp["rc"] + hp["skin"]
    full = synth.water_system(310, L=21.0, seed=1001)
    L = float(full.box[axis])
    width = L / world
    assert width >= halo                 # ghosts come from the two adjacent slabs only
    xw = np.mod(full.pos[:, axis], L)
    owner = np.minimum((xw // width).astype(int), world - 1)
    own = np.flatnonzero(owner == rank)
    lo, hi = rank * width, (rank + 1) * width
    left, right = (rank - 1) % world, (rank + 1) % world

    def exchange(sends):
        """{peer: (ids int64, rows float64 [k, 3])} -> what the peers sent to this rank."""
        peers = sorted(sends)
        out = {}
        reqs = []
        cnt_in = {q: torch.zeros(1, dtype=torch.int64) for q in peers}
        for q in peers:
            reqs.append(dist.isend(torch.tensor([len(sends[q][0])], dtype=torch.int64), q))
            reqs.append(dist.irecv(cnt_in[q], q))
        for r in reqs:
            r.wait()
        reqs = []
        buf = {}
        for q in peers:
            ids, rows = sends[q]
            reqs.append(dist.isend(torch.tensor(ids, dtype=torch.int64), q))
            reqs.append(dist.isend(torch.tensor(rows, dtype=torch.float64).reshape(-1, 3), q))
            k = int(cnt_in[q].item())
            buf[q] = (torch.zeros(k, dtype=torch.int64), torch.zeros(k, 3, dtype=torch.float64))
            reqs.append(dist.irecv(buf[q][0], q))
            reqs.append(dist.irecv(buf[q][1], q))
        for r in reqs:
            r.wait()
        for q in peers:
            out[q] = (buf[q][0].numpy(), buf[q][1].numpy())
        return out

    # halo exchange of positions: my atoms within the halo of each shared slab face
    near_lo = own[xw[own] < lo + halo]
    near_hi = own[xw[own] >= hi - halo]
    sends = {}
    for q, ids in ((left, near_lo), (right, near_hi)):
        if q == rank:
            continue
        prev = sends.get(q, (np.zeros(0, np.int64), np.zeros((0, 3))))[0]
        merged = np.union1d(prev, ids).astype(np.int64)
        sends[q] = (merged, full.pos[merged])
    got = exchange(sends)
    ghost_ids = np.unique(np.concatenate([g[0] for g in got.values()] + [np.zeros(0, np.int64)]))
    ghost_pos = {}
    for ids, rows in got.values():
        for i, r in zip(ids, rows):
            ghost_pos[int(i)] = r
    local = np.concatenate([own, ghost_ids]).astype(np.int64)      # local index -> global id
    pos = np.array([full.pos[i] for i in own] + [ghost_pos[int(i)] for i in ghost_ids])
    Z = full.Z[local]
    model = Allegro64(hp, 42)
    n_own = own.shape[0]
    terms = model.centre_terms(pos, Z, full.box, full.pbc, list(range(n_own)))
    # every edge of an owned centre is present (same count as in the whole box)
    nl_full = neighbors.neighbor_list(full.pos, full.box, full.pbc, hp["rc"], 0.0,
                                      centres=own.tolist())
    for a, g_id in enumerate(own):
        assert terms[a][1].shape[0] == nl_full[int(g_id)][0].shape[0]
    F = np.zeros((local.shape[0], 3))
    E = 0.0
    for a, (Ei, col, _sh, g) in terms.items():
        E += Ei
        if g.shape[0]:
            F[a] += g.sum(axis=0)
            np.add.at(F, col, -g)
    # reverse exchange: forces on ghosts go back to their owners, in ascending global id
    back = {}
    for q in sorted(set([left, right]) - {rank}):
        sel = np.flatnonzero(owner[local[n_own:]] == q) + n_own
        back[q] = (local[sel], F[sel])
    ret = exchange(back)
    F_own = F[:n_own].copy()
    where = {int(g_id): a for a, g_id in enumerate(own)}
    for q in sorted(ret):
        ids, rows = ret[q]
        for i, r in zip(ids, rows):
            F_own[where[int(i)]] += r
    Ft = torch.zeros(full.n, 3, dtype=torch.float64)
    Ft[torch.tensor(own)] = torch.tensor(F_own)
    Et = torch.tensor([E], dtype=torch.float64)
    nghost = torch.tensor([float(ghost_ids.shape[0])], dtype=torch.float64)
    dist.all_reduce(Ft)
    dist.all_reduce(Et)
    dist.all_reduce(nghost)
    if rank == 0:
        np.savez(out_path, F=Ft.numpy(), E=Et.numpy(), nghost=nghost.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,axis", [(2, 0), (3, 2)])
def test_brick_decomposition_with_halo_matches_whole_box(tmp_path, world, axis):
    """Slabs of a periodic water box (930 atoms, 21 A, l <= 1 model, halo rc + skin =
    6 A): two ranks along x (both neighbours are the same rank) and three along z
    (distinct left and right neighbours).  Owned energies and forces, after the reverse
    ghost-force exchange, equal the single-process evaluation."""
    import synth
    from oracle import Allegro64
    out = str(tmp_path / "bricks.npz")
    mp.start_processes(_brick_worker, args=(world, _free_port(), axis, out), nprocs=world,
                       join=True, start_method="spawn")
    res = np.load(out)
    s = synth.water_system(310, L=21.0, seed=1001)
    E, _, F = Allegro64(synth.preset("small", skin=1.0), 42).evaluate(s.pos, s.Z, s.box,
                                                                       s.pbc)
    assert res["nghost"][0] > 0
    np.testing.assert_allclose(res["F"], F, rtol=0, atol=1e-12 * max(1.0, np.abs(F).max()))
    assert abs(res["E"][0] - E[0]) <= 1e-12 * abs(E[0])


def _exchange(sends):
    """Point-to-point exchange with the peers of `sends` ({peer: (ids int64, rows float64
    [k, 3])}); returns what each of those peers sent to this rank."""
    peers = sorted(sends)
    cnt_in = {q: torch.zeros(1, dtype=torch.int64) for q in peers}
    reqs = []
    for q in peers:
        reqs.append(dist.isend(torch.tensor([len(sends[q][0])], dtype=torch.int64), q))
        reqs.append(dist.irecv(cnt_in[q], q))
    for r in reqs:
        r.wait()
    reqs, buf = [], {}
    for q in peers:
        ids, rows = sends[q]
        reqs.append(dist.isend(torch.tensor(ids, dtype=torch.int64), q))
        reqs.append(dist.isend(torch.tensor(rows, dtype=torch.float64).reshape(-1, 3), q))
        k = int(cnt_in[q].item())
        buf[q] = (torch.zeros(k, dtype=torch.int64), torch.zeros(k, 3, dtype=torch.float64))
        reqs.append(dist.irecv(buf[q][0], q))
        reqs.append(dist.irecv(buf[q][1], q))
    for r in reqs:
        r.wait()
    return {q: (buf[q][0].numpy(), buf[q][1].numpy()) for q in peers}


def _grid_worker(rank, world, port, dims, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth
    from oracle import Allegro64, neighbors
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    hp = synth.preset("small", skin=1.0)
    halo = hp["rc"] + hp["skin"]
    full = synth.water_system(310, L=21.0, seed=1001)
    L = np.asarray(full.box, dtype=np.float64)
    dims = tuple(dims)
    width = L / np.array(dims)
    for ax in range(3):
        assert dims[ax] == 1 or width[ax] >= halo   # ghosts come from adjacent bricks only
    me = np.array(np.unravel_index(rank, dims))
    xw = np.mod(full.pos, L)
    brick = np.minimum((xw // width).astype(int), np.array(dims) - 1)
    owner = np.ravel_multi_index(tuple(brick.T), dims)
    own = np.flatnonzero(owner == rank)
    held = {int(i): full.pos[i] for i in own}          # global id -> position, owned first

    def peer(ax, step):
        c = me.copy()
        c[ax] = (c[ax] + step) % dims[ax]
        return int(np.ravel_multi_index(tuple(c), dims))

    # forward halo exchange, one axis after the other: what a rank forwards along a later
    # axis includes the ghosts it received along the earlier ones, so the atoms of diagonal
    # bricks arrive through an intermediate rank
    stages = []
    for ax in range(3):
        if dims[ax] == 1:
            continue
        lo, hi = me[ax] * width[ax], (me[ax] + 1) * width[ax]
        ids = np.array(sorted(held), dtype=np.int64)
        x = np.mod(np.array([held[i][ax] for i in ids]), L[ax])
        sends = {}
        for q, sel in ((peer(ax, -1), ids[x < lo + halo]), (peer(ax, +1), ids[x >= hi - halo])):
            prev = sends.get(q, (np.zeros(0, np.int64),))[0]
            merged = np.union1d(prev, sel).astype(np.int64)
            sends[q] = (merged, np.array([held[int(i)] for i in merged]).reshape(-1, 3))
        got = _exchange(sends)
        recv = {}
        for q, (gids, rows) in got.items():
            for i, r in zip(gids, rows):
                assert int(i) not in held             # every atom arrives exactly once
                held[int(i)] = r
            recv[q] = gids
        stages.append(({q: s[0] for q, s in sends.items()}, recv))
    local = np.array(list(held), dtype=np.int64)       # local index -> global id
    index = {int(g): a for a, g in enumerate(local)}
    pos = np.array([held[int(g)] for g in local])
    n_own = own.shape[0]
    model = Allegro64(hp, 42)
    terms = model.centre_terms(pos, full.Z[local], full.box, full.pbc, list(range(n_own)))
    nl_full = neighbors.neighbor_list(full.pos, full.box, full.pbc, hp["rc"], 0.0,
                                      centres=own.tolist())
    for a, g_id in enumerate(own):
        assert terms[a][1].shape[0] == nl_full[int(g_id)][0].shape[0]
    F = np.zeros((local.shape[0], 3))
    E = 0.0
    for a, (Ei, col, _sh, g) in terms.items():
        E += Ei
        if g.shape[0]:
            F[a] += g.sum(axis=0)
            np.add.at(F, col, -g)
    # reverse exchange in the opposite order: the forces on the ghosts received in a stage
    # go back to the rank that sent them, which adds them to its own rows (its atoms, or
    # ghosts of an earlier stage that it passes on in that stage's reverse step)
    for sent, recv in reversed(stages):
        back = {q: (ids, F[[index[int(i)] for i in ids]].reshape(-1, 3))
                for q, ids in recv.items()}
        ret = _exchange(back)
        for q, (ids, rows) in ret.items():
            assert np.array_equal(np.sort(ids), np.sort(sent[q]))
            for i, r in zip(ids, rows):
                F[index[int(i)]] += r
    Ft = torch.zeros(full.n, 3, dtype=torch.float64)
    Ft[torch.tensor(own)] = torch.tensor(F[:n_own])
    Et = torch.tensor([E], dtype=torch.float64)
    relayed = torch.tensor([float(sum(len(v) for v in stages[-1][1].values()))],
                           dtype=torch.float64)
    dist.all_reduce(Ft)
    dist.all_reduce(Et)
    dist.all_reduce(relayed)
    if rank == 0:
        np.savez(out_path, F=Ft.numpy(), E=Et.numpy(), relayed=relayed.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("dims", [(2, 2, 1), (3, 1, 2), (2, 2, 2)])
def test_brick_grid_with_staged_halo_matches_whole_box(tmp_path, dims):
    """Grids of bricks over two or three axes (2 x 2 along x, y: the same peer on both
    sides of each axis; 3 x 2 along x, z: distinct peers along x; 2 x 2 x 2), halo
    rc + skin = 6 A.  The halo exchange runs one axis at a time and forwards the ghosts of
    earlier axes, so atoms of edge- and corner-adjacent bricks reach a rank through one or
    two intermediate ranks; the ghost forces return in the reverse order through the same
    ranks.  Owned energies and forces equal the single-process evaluation."""
    import synth
    from oracle import Allegro64
    world = int(np.prod(dims))
    out = str(tmp_path / "grid.npz")
    mp.start_processes(_grid_worker, args=(world, _free_port(), dims, out), nprocs=world,
                       join=True, start_method="spawn")
    res = np.load(out)
    s = synth.water_system(310, L=21.0, seed=1001)
    E, _, F = Allegro64(synth.preset("small", skin=1.0), 42).evaluate(s.pos, s.Z, s.box,
                                                                       s.pbc)
    assert res["relayed"][0] > 0
    np.testing.assert_allclose(res["F"], F, rtol=0, atol=1e-12 * max(1.0, np.abs(F).max()))
    assert abs(res["E"][0] - E[0]) <= 1e-12 * abs(E[0])
