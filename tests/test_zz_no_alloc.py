"""ff_neighbors_noalloc: the neighbour-list build for callers that cannot allocate device
memory (pool-only MD engines, code inside CUDA-graph capture, hosts that forbid
allocation in their step loop).  Its edge list must equal the one ff_neighbors builds,
on consecutive calls that reuse its shared scratch array.

This file is collected last on purpose, so that a run stopping at the first failure has
run every other test first.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ff():
    import paper_2502_06073_gb300 as ff
    ff._build.build()
    ff.load_library()
    assert torch.cuda.is_available()
    return ff


def _noalloc(ff, s, rc):
    lib = ff.load_library()
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    box = (ctypes.c_double * 3)(*s.box.tolist())
    pbc = (ctypes.c_int * 3)(*[int(b) for b in s.pbc])
    rp = torch.empty(s.n + 1, dtype=torch.int32, device="cuda")
    ne = ctypes.c_int64()
    msg = ctypes.create_string_buffer(256)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc_ = lib.ff_neighbors_noalloc(ctypes.c_void_p(pos.data_ptr()), s.n, box, pbc, rc,
                                   ctypes.c_void_p(rp.data_ptr()), None, None, 0,
                                   ctypes.byref(ne), msg, 256, stream)
    assert rc_ == 0, msg.value
    E = ne.value
    col = torch.empty(max(E, 1), dtype=torch.int32, device="cuda")
    sh = torch.empty(max(E, 1), dtype=torch.int32, device="cuda")
    rc_ = lib.ff_neighbors_noalloc(ctypes.c_void_p(pos.data_ptr()), s.n, box, pbc, rc,
                                   ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                                   ctypes.c_void_p(sh.data_ptr()), E, ctypes.byref(ne), msg, 256,
                                   stream)
    assert rc_ == 0, msg.value
    torch.cuda.synchronize()
    packed = sh[:E].cpu().numpy().astype(np.int64)
    shift = np.stack([((packed >> (8 * k)) & 0xFF).astype(np.int8) for k in range(3)], axis=1)
    return rp.cpu().numpy(), col[:E].cpu().numpy(), shift.astype(np.int32)


def _existing(ff, s, rc):
    hp = synth.preset("small", rc=rc, skin=0.0)
    m = ff.FFModel(hp, seed=1)
    m.bind(torch.tensor(s.pos, dtype=torch.float64, device="cuda"),
           torch.tensor(s.Z, dtype=torch.int32, device="cuda"), s.box, s.pbc)
    rp, col, sh, _ = m.edges()
    return rp, col, sh


def test_noalloc_matches_ff_neighbors_on_consecutive_calls(ff):
    cases = [(synth.csh_system(sub=True), 6.0),          # 512 atoms, then
             (synth.config1_system(), 5.0),              # a smaller, tiny periodic box
             (synth.water_system(1365, L=34.44, seed=1001), 6.0)]   # 4,095 atoms
    for s, rc in cases:
        got = _noalloc(ff, s, rc)
        ref = _existing(ff, s, rc)
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)


def test_noalloc_rejects_oversized_system(ff):
    lib = ff.load_library()
    n = 4097
    pos = torch.zeros(n, 3, dtype=torch.float64, device="cuda")
    rp = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    ne = ctypes.c_int64()
    msg = ctypes.create_string_buffer(256)
    rc_ = lib.ff_neighbors_noalloc(ctypes.c_void_p(pos.data_ptr()), n,
                                   (ctypes.c_double * 3)(50.0, 50.0, 50.0),
                                   (ctypes.c_int * 3)(1, 1, 1), 5.0,
                                   ctypes.c_void_p(rp.data_ptr()), None, None, 0,
                                   ctypes.byref(ne), msg, 256, None)
    assert rc_ == -1 and b"FF_NOALLOC_MAX_ATOMS" in msg.value
