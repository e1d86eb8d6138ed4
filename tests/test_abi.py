"""Host-side checks of the library: it builds for sm_103a, loads without a GPU, exports
every entry point declared in include/ff.h, validates hyperparameters and null or
out-of-range arguments before touching the device, and its generated tensor-product tables agree with the oracle's coupling tensors
(two independent constructions: Racah formula vs Wigner-matrix null space)."""
import ctypes
import importlib.util
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_06073_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    import paper_2502_06073_gb300 as ff
    ff._build.build()
    return ff.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "ff.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ff_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    import paper_2502_06073_gb300 as ff
    assert sorted(ff.ABI) == names


def test_build_compiles_every_cuda_source():
    """Every .cu file of csrc/ is one translation unit of libff.so, and only those."""
    from paper_2502_06073_gb300 import _build
    on_disk = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    assert sorted(_build.SOURCES) == on_disk
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _gen_module():
    spec = importlib.util.spec_from_file_location("gen_tp", os.path.join(CSRC, "gen_tp.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_hparams_rejected_before_device_use(lib):
    import synth
    import paper_2502_06073_gb300 as ff
    bad = [dict(lmax=3), dict(channels=24), dict(parity=0), dict(latent=[64]),
           dict(two_body=[30, 32]), dict(n_basis=12), dict(rc=-1.0), dict(n_layers=5)]
    for over in bad:
        hp = synth.preset("small", **over)
        h = ctypes.c_void_p()
        st = ff.hparams_struct(hp)
        rc = lib.ff_create(ctypes.byref(h), ctypes.byref(st), ctypes.c_uint64(1))
        assert rc == -1, over
        assert lib.ff_last_error(None)
        assert not h.value


def test_racah_tables_match_oracle_coupling():
    from oracle import so3
    gen = _gen_module()
    for l1 in range(3):
        for l2 in range(3):
            for l3 in range(abs(l1 - l2), min(l1 + l2, 2) + 1):
                A = np.zeros((2 * l1 + 1, 2 * l2 + 1, 2 * l3 + 1))
                for k, v in gen.coupling_real(l1, l2, l3).items():
                    A[k] = v
                np.testing.assert_allclose(A, so3.coupling(l1, l2, l3), atol=1e-12)


def test_generated_paths_match_oracle_paths():
    from oracle import so3
    gen = _gen_module()
    for lmax in (1, 2):
        for n_layers in (1, 2, 3, 4):
            layers = so3.model_paths(lmax, n_layers)
            for L, (irr_in, paths, outs) in enumerate(layers, start=1):
                ink = min(L - 1, 2)
                irr = gen.in_irreps_of(lmax, ink)
                gp, gouts = gen.layer(irr, lmax, L == n_layers)
                assert irr == irr_in and gp == paths and gouts == outs


def test_pruned_layer_before_last_keeps_everything_the_energy_sees():
    """The layer before the last computes only natural-parity outputs (output kind 1) and
    the last layer reads only those: check against the oracle's full path lists that every
    path into a 0e output of the last layer starts from a natural-parity irrep, that the
    pruned kind keeps exactly the paths into natural outputs with their full-list indices
    (path weights and the 1/sqrt(n) mixing are those of the full layer), and that every
    layer of a 1- to 4-layer model maps to a generated kind."""
    from oracle import so3
    gen = _gen_module()
    for lmax in (1, 2):
        for n_layers in (1, 2, 3, 4):
            layers = so3.model_paths(lmax, n_layers)
            irr_last, paths_last, _ = layers[-1]
            for (i_in, _l2, out) in paths_last:
                assert out == (0, 1) and gen.natural(irr_last[i_in])
            for L in range(1, n_layers + 1):
                ink, outk = gen.layer_kinds(L, n_layers)
                irr = 0 if ink == 3 else ink
                assert (irr, outk) in gen.KINDS
                _, _, info = gen.gen_kind(lmax, irr, outk)
                irr_in, paths, outs = layers[L - 1]
                if ink == 3:
                    assert info["irr_in"] == [ir for ir in irr_in if gen.natural(ir)]
                else:
                    assert info["irr_in"] == irr_in
                if outk == 1:
                    assert info["np"] == len(paths)
                    assert info["kept"] == sum(gen.natural(p[2]) for p in paths)
                    assert info["outs"] == [o for o in outs if gen.natural(o)]
                elif outk == 2:
                    assert info["outs"] == [(0, 1)] and info["kept"] == info["np"]
                else:
                    assert info["outs"] == outs and info["kept"] == len(paths)


def test_committed_tp_header_is_current(tmp_path):
    gen = _gen_module()
    out = tmp_path / "tp_gen.cuh"
    gen.main(str(out))
    assert out.read_text() == open(os.path.join(CSRC, "tp_gen.cuh")).read()


def test_null_context_and_argument_errors(lib):
    """Every entry point that takes a context rejects a null one with FF_ERR_ARG before any
    device work; the argument checks that need no device answer the same way on a host
    without a GPU."""
    import synth
    import paper_2502_06073_gb300 as ff
    ERR_ARG = -1
    zeros = {ctypes.c_void_p: None, ctypes.c_int: 0, ctypes.c_int64: 0, ctypes.c_double: 0.0,
             ctypes.c_float: 0.0, ctypes.c_size_t: 0, ctypes.c_uint64: 0,
             ctypes.c_char_p: None}
    takes_ctx = ("ff_neighbors", "ff_energy_forces", "ff_forces", "ff_md_step",
                 "ff_export_params", "ff_get_edges", "ff_energy_forces_graph", "ff_set_graph",
                 "ff_autotune", "ff_virial", "ff_md_nvt")
    for name in takes_ctx:
        fn = getattr(lib, name)
        args = [zeros.get(t) for t in fn.argtypes]
        assert fn(*args) == ERR_ARG, name
    lib.ff_destroy(None)
    assert isinstance(lib.ff_last_error(None), bytes)
    # ff_create: null output or hyperparameters
    h = ctypes.c_void_p()
    st = ff.hparams_struct(synth.preset("small"))
    assert lib.ff_create(None, ctypes.byref(st), 1) == ERR_ARG
    assert lib.ff_create(ctypes.byref(h), None, 1) == ERR_ARG and not h.value
    # profiler: the class table and a too-small read buffer
    n = ctypes.c_int()
    one = (ctypes.c_int64 * 1)()
    onef = (ctypes.c_double * 1)()
    assert lib.ff_profile_read(one, onef, 1, ctypes.byref(n)) == ERR_ARG
    assert n.value >= 2
    names = [lib.ff_profile_class(k).decode() for k in range(n.value)]
    assert all(names) and len(set(names)) == n.value
    assert lib.ff_profile_class(-1) == b"" and lib.ff_profile_class(n.value) == b""
    # ff_neighbors_noalloc validates its arguments before it asks for a device
    dummy = ctypes.c_void_p(16)           # never dereferenced on these paths
    ne = ctypes.c_int64()
    msg = ctypes.create_string_buffer(256)
    box = (ctypes.c_double * 3)(20.0, 20.0, 20.0)
    pbc = (ctypes.c_int * 3)(1, 1, 1)

    def noalloc(pos=dummy, n_atoms=10, box_=box, pbc_=pbc, rc=5.0, row_ptr=dummy):
        msg.value = b""
        return lib.ff_neighbors_noalloc(pos, n_atoms, box_, pbc_, rc, row_ptr, None, None, 0,
                                        ctypes.byref(ne), msg, 256, None)

    assert noalloc(pos=None) == ERR_ARG and msg.value
    assert noalloc(row_ptr=None) == ERR_ARG and msg.value
    assert noalloc(n_atoms=0) == ERR_ARG
    assert noalloc(n_atoms=4097) == ERR_ARG and b"FF_NOALLOC_MAX_ATOMS" in msg.value
    assert noalloc(rc=0.0) == ERR_ARG and b"rc" in msg.value
    assert noalloc(box_=(ctypes.c_double * 3)(20.0, -1.0, 20.0)) == ERR_ARG
    assert noalloc(pbc_=(ctypes.c_int * 3)(1, 2, 1)) == ERR_ARG


def test_error_word_decoding(tmp_path):
    """The mapping from the device error word to status codes (csrc/ff_flags.h), compiled
    on the host with gcc: each bit gives its code, a bad input wins over what it causes,
    a pipeline timeout is FF_ERR_TIMEOUT, an unknown bit FF_ERR_CUDA."""
    import subprocess
    shim = tmp_path / "shim.c"
    shim.write_text('#include "ff_flags.h"\n'
                    'int decode(int w) { const char* m = 0; int s = ff_flags_status(w, &m);'
                    ' return (w && !(m && m[0])) ? 99 : s; }\n')
    so = tmp_path / "libshim.so"
    subprocess.run(["gcc", "-shared", "-fPIC", "-std=c99", "-Wall", "-Werror", "-I", CSRC,
                    str(shim), "-o", str(so)], check=True)
    dec = ctypes.CDLL(str(so)).decode
    expect = {0: 0, 1: -5, 4: -8, 8: -7, 16: -2, 32: -6, 64: -9, 128: -6, 256: -4,
              16 | 64: -2, 128 | 1: -6, 4 | 1: -8, 64 | 32: -9, 1 | 64: -5}
    for word, code in expect.items():
        assert dec(word) == code, (word, dec(word), code)
    import paper_2502_06073_gb300 as ff
    assert ff.ERRORS[-9] == "FF_ERR_TIMEOUT"
    hdr = open(os.path.join(ROOT, "include", "ff.h")).read()
    assert "FF_ERR_TIMEOUT = -9" in hdr
