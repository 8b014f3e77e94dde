"""smcx_energy_noalloc: the energy entry point for callers that cannot
allocate device memory (it keeps its scratch in a fixed device array inside
the library instead of asking cudaMalloc).

The paper has no counterpart to this entry point.  The tests call it through
the C ABI and compare each result with the oracle's energy of the same
configuration (an exact integer, so the tolerance is zero) and with the
handle-based smcx_energy: on two different configurations called back to
back (the shared scratch must be cleared between calls), then once more on
the first; at the scratch capacity (K*M*M up to 1296 of 1300 histogram
bins); and with ids outside 0..M-1 or a host pointer, which must be refused
without touching memory out of bounds.  Collected last on purpose, so that a
failure here stops a -x run only after every other test has run.
"""
import numpy as np
import pytest

import oracle as O
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


def test_energy_noalloc_matches_handle_and_oracle_energy():
    assert torch.cuda.is_available()
    stream = torch.cuda.current_stream()
    a, Va = _lattice(smcx.BCC, (16, 14, 12), 4, [0.25] * 4, smcx.PACKED4, 4, 3, stream)
    b, Vb = _lattice(smcx.FCC, (9, 8, 10), 5, [0.3, 0.25, 0.2, 0.15, 0.1], smcx.INT8, 3, 5, stream)
    want_a, want_b = a.energy(), b.energy()
    assert want_a == O.energy(O.BCC, a.dims, 4, 4, Va, a.get_config())
    assert want_b == O.energy(O.FCC, b.dims, 5, 3, Vb, b.get_config())
    pa, _ = a.device_buffer()
    pb, _ = b.device_buffer()
    got_a = smcx.energy_noalloc(smcx.BCC, a.dims, 4, smcx.PACKED4, Va, pa, stream)
    got_b = smcx.energy_noalloc(smcx.FCC, b.dims, 5, smcx.INT8, Vb, pb, stream)
    assert got_a == want_a
    assert got_b == want_b
    assert smcx.energy_noalloc(smcx.BCC, a.dims, 4, smcx.PACKED4, Va, pa, stream) == want_a
    a.close()
    b.close()


def _pack4(cfg):
    c = cfg.astype(np.uint8)
    if c.size % 2:
        c = np.concatenate([c, np.zeros(1, np.uint8)])
    return (c[0::2] | (c[1::2] << 4)).astype(np.uint8)


@pytest.mark.parametrize("kind,dims,M,K,storage", [
    (smcx.BCC, (6, 5, 7), 18, 4, smcx.INT8),    # 1296 bins: the layout at its limit
    (smcx.BCC, (5, 6, 4), 36, 1, smcx.INT8),    # 1296 bins, one shell
    (smcx.FCC, (5, 4, 3), 20, 3, smcx.INT8),    # 1200 bins
    (smcx.BCC, (7, 6, 5), 15, 4, smcx.PACKED4),  # 900 bins, packed store
])
def test_energy_noalloc_at_scratch_capacity(kind, dims, M, K, storage):
    stream = torch.cuda.current_stream()
    m = 2 if kind == smcx.BCC else 4
    N = int(np.prod(dims)) * m
    rng = np.random.default_rng(M * 100 + K)
    cfg = rng.integers(0, M, N).astype(np.int8)
    V = epi_gaussian(K, M, 20.0, M + K)
    want = O.energy(O.BCC if kind == smcx.BCC else O.FCC, dims, M, K, V, cfg)
    store = cfg.view(np.uint8) if storage == smcx.INT8 else _pack4(cfg)
    dev = torch.from_numpy(store.copy()).to("cuda")
    for _ in range(2):  # twice in a row: the scratch is cleared per call
        got = smcx.energy_noalloc(kind, dims, M, storage, V, dev.data_ptr(), stream)
        assert got == want


def test_energy_noalloc_refuses_bad_ids_and_host_pointers():
    stream = torch.cuda.current_stream()
    dims, M, K = (6, 6, 6), 4, 4
    rng = np.random.default_rng(7)
    cfg = rng.integers(0, M, 2 * 216).astype(np.int8)
    V = epi_gaussian(K, M, 20.0, 2)
    good = torch.from_numpy(cfg.copy()).to("cuda")
    want = O.energy(O.BCC, dims, M, K, V, cfg)
    bad_cfg = cfg.copy()
    bad_cfg[[5, 100]] = M  # ids outside 0..M-1
    bad = torch.from_numpy(bad_cfg).to("cuda")
    with pytest.raises(smcx.SmcxError) as e:
        smcx.energy_noalloc(smcx.BCC, dims, M, smcx.INT8, V, bad.data_ptr(), stream)
    assert e.value.code == smcx.E_INVALID_ARG
    host = np.ascontiguousarray(cfg.view(np.uint8))
    with pytest.raises(smcx.SmcxError) as e:
        smcx.energy_noalloc(smcx.BCC, dims, M, smcx.INT8, V, host.ctypes.data, stream)
    assert e.value.code == smcx.E_INVALID_ARG
    # the flag and histogram are cleared for the next call
    assert smcx.energy_noalloc(smcx.BCC, dims, M, smcx.INT8, V, good.data_ptr(), stream) == want


def test_energy_noalloc_rejects_oversize_tables():
    stream = torch.cuda.current_stream()
    lat = smcx.Lattice(smcx.BCC, (8, 8, 8), 4, [0.25] * 4, storage=smcx.INT8, stream=stream)
    p, _ = lat.device_buffer()
    big = np.zeros((4, 20, 20), np.int32)  # K*M*M = 1600 exceeds the fixed scratch
    with pytest.raises(smcx.SmcxError) as e:
        smcx.energy_noalloc(smcx.BCC, (8, 8, 8), 20, smcx.INT8, big, p, stream)
    assert e.value.code == smcx.E_INVALID_ARG
    lat.close()
