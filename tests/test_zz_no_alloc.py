"""smcx_energy_noalloc: the energy entry point for callers that cannot
allocate device memory (it keeps its scratch in a fixed device array inside
the library instead of asking cudaMalloc).

The paper has no counterpart to this entry point.  The test calls it through
the C ABI on configurations held by lattice handles and compares each result
with the handle-based smcx_energy (an exact integer, so the tolerance is
zero), on two different configurations called back to back (the shared
scratch must be cleared between calls) and then once more on the first.
Collected last on purpose, so that a failure here stops a -x run only after
every other test has run.
"""
import numpy as np
import pytest

from paper_2503_12591_gb300 import smcx
from paper_2503_12591_gb300.inputs import epi_gaussian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lattice(kind, dims, M, comp, storage, K, seed, stream):
    lat = smcx.Lattice(kind, dims, M, comp, init_seed=seed, storage=storage, stream=stream)
    V = epi_gaussian(K, M, 20.0, seed)
    lat.set_epi(V)
    if lat.schedule()[0]:
        lat.sweep(1500.0, 2, seed)
    return lat, V


def test_energy_noalloc_matches_handle_energy():
    assert torch.cuda.is_available()
    stream = torch.cuda.current_stream()
    a, Va = _lattice(smcx.BCC, (16, 14, 12), 4, [0.25] * 4, smcx.PACKED4, 4, 3, stream)
    b, Vb = _lattice(smcx.FCC, (9, 8, 10), 5, [0.3, 0.25, 0.2, 0.15, 0.1], smcx.INT8, 3, 5, stream)
    want_a, want_b = a.energy(), b.energy()
    pa, _ = a.device_buffer()
    pb, _ = b.device_buffer()
    got_a = smcx.energy_noalloc(smcx.BCC, a.dims, 4, smcx.PACKED4, Va, pa, stream)
    got_b = smcx.energy_noalloc(smcx.FCC, b.dims, 5, smcx.INT8, Vb, pb, stream)
    assert got_a == want_a
    assert got_b == want_b
    assert smcx.energy_noalloc(smcx.BCC, a.dims, 4, smcx.PACKED4, Va, pa, stream) == want_a
    a.close()
    b.close()


def test_energy_noalloc_rejects_oversize_tables():
    stream = torch.cuda.current_stream()
    lat = smcx.Lattice(smcx.BCC, (8, 8, 8), 4, [0.25] * 4, storage=smcx.INT8, stream=stream)
    p, _ = lat.device_buffer()
    big = np.zeros((4, 20, 20), np.int32)  # K*M*M = 1600 exceeds the fixed scratch
    with pytest.raises(smcx.SmcxError) as e:
        smcx.energy_noalloc(smcx.BCC, (8, 8, 8), 20, smcx.INT8, big, p, stream)
    assert e.value.code == smcx.E_INVALID_ARG
    lat.close()
