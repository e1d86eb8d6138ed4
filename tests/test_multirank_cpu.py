"""Multi-process (gloo, world size 2, CPU) checks of how the path shards.

Strict locality (Abstract: "strictly-local") lets disjoint sets of centre atoms be
evaluated independently: each rank computes the energies of its centres and the edge
gradients of their edges, scatters them into a force array (F_i += g_e, F_j -= g_e) and
one all-reduce sums the ranks.  The result must equal the single-process evaluation.
The benchmark's replica mode is checked too: the timed value uses the maximum time over
ranks and every rank's atoms.
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
