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
