"""ff_neighbors_noalloc: the neighbour-list build for callers that cannot allocate device
memory -- an MD engine whose pool allocator has reserved the device memory up front (a
cudaMalloc would fail or fragment its pool), or a host that forbids allocation inside its
time-step loop (cudaMalloc can synchronise the device and takes unbounded time).  Its edge
list must equal the one ff_neighbors builds, on consecutive calls that reuse its shared
scratch array, and the calls must leave the device's free memory unchanged.

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


def _noalloc(ff, s, rc, pos=None):
    lib = ff.load_library()
    if pos is None:
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


def _call(lib, pos, n, box, pbc, rc, rp, col=None, sh=None, cap=0):
    ne = ctypes.c_int64()
    msg = ctypes.create_string_buffer(256)
    rc_ = lib.ff_neighbors_noalloc(ctypes.c_void_p(pos.data_ptr()), n,
                                   (ctypes.c_double * 3)(*box), (ctypes.c_int * 3)(*pbc), rc,
                                   ctypes.c_void_p(rp.data_ptr()),
                                   ctypes.c_void_p(col.data_ptr()) if col is not None else None,
                                   ctypes.c_void_p(sh.data_ptr()) if sh is not None else None,
                                   cap, ctypes.byref(ne), msg, 256,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc_, ne.value, msg.value


def test_noalloc_coarsened_cell_grid_matches_ff_neighbors(ff):
    """4,095 atoms with rc = 2 A in a 34.44 A box: 17^3 = 4,913 cells of at least rc would
    exceed the 4,096-cell cap, so the call coarsens the grid (fewer, wider cells); the list
    must still equal ff_neighbors'."""
    s = synth.water_system(1365, L=34.44, seed=1001)
    assert int(np.floor(34.44 / 2.0)) ** 3 > 4096
    got = _noalloc(ff, s, 2.0)
    ref = _existing(ff, s, 2.0)
    assert got[1].shape[0] > 0
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_noalloc_errors_capacity_short_buffer_nonfinite(ff):
    """More than 256 neighbours -> FF_ERR_CAPACITY; edge buffers one short of the edge
    count -> FF_ERR_ARG; a NaN coordinate -> FF_ERR_NONFINITE; then a valid call on the
    same scratch still returns the right list."""
    lib = ff.load_library()
    rng = np.random.default_rng(7)
    n = 300
    dense = torch.tensor(rng.uniform(0.0, 10.0, size=(n, 3)), dtype=torch.float64,
                         device="cuda")
    rp = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    rc_, _, msg = _call(lib, dense, n, (10.0, 10.0, 10.0), (1, 1, 1), 8.0, rp)
    assert rc_ == -5 and b"FF_NOALLOC_MAX_NEIGHBORS" in msg, (rc_, msg)

    s = synth.config1_system()
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    rp = torch.empty(s.n + 1, dtype=torch.int32, device="cuda")
    box, pbc = s.box.tolist(), [int(b) for b in s.pbc]
    rc_, E, msg = _call(lib, pos, s.n, box, pbc, 5.0, rp)
    assert rc_ == 0 and E > 0, msg
    col = torch.empty(E, dtype=torch.int32, device="cuda")
    sh = torch.empty(E, dtype=torch.int32, device="cuda")
    rc_, _, msg = _call(lib, pos, s.n, box, pbc, 5.0, rp, col, sh, E - 1)
    assert rc_ == -1 and b"smaller than the edge count" in msg, (rc_, msg)

    bad = pos.clone()
    bad[17, 1] = float("nan")
    rc_, _, msg = _call(lib, bad, s.n, box, pbc, 5.0, rp, col, sh, E)
    assert rc_ == -6 and b"non-finite" in msg, (rc_, msg)

    got = _noalloc(ff, s, 5.0)
    ref = _existing(ff, s, 5.0)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_noalloc_allocates_nothing(ff):
    """Once a first call has run (kernels loaded, scratch address looked up), further calls
    change neither the device's free memory nor the memory torch's allocator reserves."""
    lib = ff.load_library()
    s = synth.csh_system(sub=True)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    rp = torch.empty(s.n + 1, dtype=torch.int32, device="cuda")
    box, pbc = s.box.tolist(), [int(b) for b in s.pbc]
    rc_, E, msg = _call(lib, pos, s.n, box, pbc, 6.0, rp)
    assert rc_ == 0, msg
    col = torch.empty(E, dtype=torch.int32, device="cuda")
    sh = torch.empty(E, dtype=torch.int32, device="cuda")
    rc_, _, msg = _call(lib, pos, s.n, box, pbc, 6.0, rp, col, sh, E)
    assert rc_ == 0, msg
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    first = (rp.clone(), col.clone(), sh.clone())
    for _ in range(3):
        rc_, E2, msg = _call(lib, pos, s.n, box, pbc, 6.0, rp)
        assert rc_ == 0 and E2 == E, msg
        rc_, _, msg = _call(lib, pos, s.n, box, pbc, 6.0, rp, col, sh, E)
        assert rc_ == 0, msg
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    for a, b in zip(first, (rp, col, sh)):
        assert torch.equal(a, b)
