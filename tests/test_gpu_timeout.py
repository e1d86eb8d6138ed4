"""Failure detection on the GPU without a fault: a bounded device wait that runs out.

Every wait of the persistent tensor-core GEMM (TMA stages, accumulators, epilogue inputs)
has an iteration limit, after which the kernel sets a timeout bit in the context's error
word, the other warps leave through the abort path, the CTA releases its tensor memory and
returns.  With FF_TEST_STALL_ONCE set when a context is created, the first GEMM launch
withholds the completion signal of each CTA's first accumulator (a signal that nothing
sends), so its epilogue's wait runs out after a short limit.  The evaluation must report
FF_ERR_TIMEOUT, and the same context must then evaluate normally, bit for bit like a fresh
one.
"""
import os

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


def _bind(ff, hp, s):
    m = ff.FFModel(hp, seed=42, precision=1)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    m.bind(pos, torch.tensor(s.Z, dtype=torch.int32, device="cuda"), s.box, s.pbc)
    return m, pos


def test_gemm_wait_timeout_is_reported_and_the_context_recovers(ff):
    s = synth.csh_system(sub=True)
    hp = synth.preset("fm_water", avg_num_neighbors=synth.NU["csh512"])
    os.environ["FF_TEST_STALL_ONCE"] = "1"
    try:
        m, pos = _bind(ff, hp, s)
    finally:
        del os.environ["FF_TEST_STALL_ONCE"]
    with pytest.raises(ff.FFError, match="FF_ERR_TIMEOUT"):
        m.energy_forces(pos)
    _, Ea, F = m.energy_forces(pos)
    ref, pos_r = _bind(ff, hp, s)
    _, Ea_r, F_r = ref.energy_forces(pos_r)
    assert torch.equal(Ea, Ea_r) and torch.equal(F, F_r)
    assert np.isfinite(F.cpu().numpy()).all()
