"""GPU parity: the CUDA path through the C ABI against the oracle.

Integer results (configurations, trial statistics, energies, pair counts) must
match bit for bit; the Warren-Cowley SRO (FP64 from integer counts) within
1e-12 relative.  Cases span several tiles, uneven tile sizes (ragged tails),
both storages, both lattices, the paper's link-cell schedule and the tiled
schedule.
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_12591_gb300 import smcx
from paper_2503_12591_gb300.inputs import epi_gaussian, ORACLE_BCC16

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def stream():
    assert torch.cuda.is_available()
    return torch.cuda.current_stream()


def _oracle_run(kind, dims, M, K, V, comp, init_seed, T, n, seed, sched):
    ref = O.init_config(kind, dims, M, comp, init_seed)
    st = O.sweep(kind, dims, M, K, V, ref, T, n, seed, L=sched[0], nt=sched[1])
    return ref, st


@pytest.mark.parametrize("kind,dims,M,comp,storage", [
    (smcx.BCC, (6, 7, 5), 4, [0.25] * 4, smcx.INT8),
    (smcx.BCC, (9, 4, 6), 4, [0.25] * 4, smcx.PACKED4),
    (smcx.FCC, (5, 6, 7), 5, [0.3, 0.25, 0.2, 0.15, 0.1], smcx.PACKED4),
    (smcx.FCC, (4, 4, 4), 3, [0.5, 0.3, 0.2], smcx.INT8),
])
def test_initial_configuration(stream, kind, dims, M, comp, storage):
    lat = smcx.Lattice(kind, dims, M, comp, init_seed=77, storage=storage, stream=stream)
    got = lat.get_config()
    ref = O.init_config(kind, dims, M, comp, 77)
    assert (got == ref).all()


@pytest.mark.parametrize("kernel", [smcx.KERNEL_AUTO, smcx.KERNEL_GENERIC], ids=["auto", "generic"])
@pytest.mark.parametrize("kind,K,dims,M,storage", [
    (smcx.BCC, 4, (8, 6, 10), 4, smcx.INT8),
    (smcx.BCC, 2, (6, 6, 6), 3, smcx.PACKED4),
    (smcx.BCC, 4, (45, 38, 41), 4, smcx.PACKED4),
    (smcx.BCC, 3, (21, 7, 26), 2, smcx.INT8),
    (smcx.FCC, 3, (6, 8, 6), 5, smcx.PACKED4),
])
def test_energy_pair_counts_sro(stream, kind, K, dims, M, storage, kernel):
    N = O.n_sites(kind, dims)
    cfg = np.random.default_rng(5).integers(0, M, N).astype(np.int8)
    V = epi_gaussian(K, M, 20.0, 3)
    lat = smcx.Lattice(kind, dims, M, [1.0 / M] * M, storage=storage, stream=stream)
    lat.set_kernel(kernel)
    lat.set_epi(V)
    lat.set_config(cfg)
    assert (lat.get_config() == cfg).all()
    C = lat.pair_counts()
    assert (C == O.pair_counts(kind, dims, M, K, cfg)).all()
    assert lat.energy() == O.energy(kind, dims, M, K, V, cfg)
    np.testing.assert_allclose(lat.sro(), O.sro(kind, dims, M, K, cfg), rtol=1e-12, atol=1e-15)


SWEEP_CASES = [
    # kind, K, dims, M, comp, storage, schedule (L, nt), T, sweeps
    (smcx.BCC, 4, (16, 16, 16), 4, [0.25] * 4, smcx.INT8, (3, (4, 4, 4)), 1000.0, 10),
    (smcx.BCC, 4, (16, 16, 16), 4, [0.25] * 4, smcx.PACKED4, (4, (2, 2, 2)), 1000.0, 10),
    (smcx.BCC, 4, (13, 14, 15), 4, [0.25] * 4, smcx.PACKED4, (3, (4, 2, 4)), 1500.0, 6),   # ragged tiles
    (smcx.BCC, 4, (12, 12, 12), 4, [0.25] * 4, smcx.INT8, (3, (1, 1, 1)), 800.0, 6),       # link-cell
    (smcx.BCC, 4, (12, 12, 16), 4, [0.25] * 4, smcx.PACKED4, (4, (1, 1, 1)), 2500.0, 4),   # link-cell
    (smcx.BCC, 2, (12, 10, 8), 3, [0.5, 0.3, 0.2], smcx.INT8, (3, (2, 2, 2)), 1200.0, 5),
    (smcx.BCC, 2, (40, 36, 32), 4, [0.25] * 4, smcx.PACKED4, (4, (2, 2, 2)), 1000.0, 2),  # 20-cell tiles
    (smcx.BCC, 3, (20, 18, 16), 4, [0.25] * 4, smcx.PACKED4, (4, (2, 2, 2)), 1300.0, 3),
    (smcx.BCC, 1, (10, 12, 8), 2, [0.5, 0.5], smcx.PACKED4, (3, (2, 2, 2)), 600.0, 5),
    (smcx.BCC, 3, (24, 20, 22), 6, [1 / 6] * 6, smcx.PACKED4, (4, (2, 2, 2)), 1500.0, 3),
    (smcx.BCC, 4, (40, 24, 26), 8, [0.125] * 8, smcx.INT8, (3, (2, 2, 2)), 2000.0, 2),
    (smcx.BCC, 4, (42, 40, 38), 4, [0.25] * 4, smcx.PACKED4, (4, (4, 2, 2)), 1000.0, 2),
    # staging from 32-bit words: tile origins at every x offset mod 4 (packed) and mod 2 (int8),
    # and an odd x extent that takes the per-column path
    (smcx.BCC, 4, (44, 20, 18), 4, [0.25] * 4, smcx.PACKED4, (3, (4, 2, 2)), 1000.0, 2),
    (smcx.BCC, 4, (22, 15, 14), 4, [0.25] * 4, smcx.INT8, (3, (2, 2, 2)), 1000.0, 3),
    (smcx.BCC, 4, (15, 12, 14), 4, [0.25] * 4, smcx.INT8, (3, (2, 2, 2)), 1000.0, 3),
    (smcx.FCC, 3, (12, 12, 12), 5, [0.3, 0.25, 0.2, 0.15, 0.1], smcx.PACKED4, (3, (4, 4, 4)), 1200.0, 5),
    (smcx.FCC, 3, (9, 10, 11), 5, [0.3, 0.25, 0.2, 0.15, 0.1], smcx.INT8, (3, (2, 4, 2)), 1200.0, 4),
    (smcx.FCC, 3, (9, 9, 9), 4, [0.25] * 4, smcx.PACKED4, (3, (1, 1, 1)), 1000.0, 4),      # link-cell
    # tiles of 15/14-15/14 cells: the largest box of the FCC tile kernel
    (smcx.FCC, 3, (30, 29, 28), 5, [0.3, 0.25, 0.2, 0.15, 0.1], smcx.PACKED4, (3, (2, 2, 2)), 1200.0, 3),
    # fewer shells on the FCC tile kernel (six-bit counters, M <= 5)
    (smcx.FCC, 2, (16, 14, 12), 3, [0.5, 0.3, 0.2], smcx.INT8, (3, (2, 2, 2)), 900.0, 4),
    (smcx.FCC, 1, (12, 12, 10), 2, [0.5, 0.5], smcx.PACKED4, (3, (2, 2, 2)), 700.0, 4),
    (smcx.FCC, 3, (18, 12, 12), 4, [0.25] * 4, smcx.PACKED4, (3, (2, 2, 2)), 1100.0, 3),
    (smcx.FCC, 3, (12, 12, 12), 6, [1 / 6] * 6, smcx.INT8, (3, (2, 2, 2)), 1300.0, 3),
    # FCC staging: 16-bit cells from words with an odd tile origin, and an odd x extent (per-column path)
    (smcx.FCC, 3, (22, 12, 12), 5, [0.3, 0.25, 0.2, 0.15, 0.1], smcx.PACKED4, (3, (2, 2, 2)), 1200.0, 3),
    (smcx.FCC, 3, (21, 12, 12), 4, [0.25] * 4, smcx.PACKED4, (3, (2, 2, 2)), 1200.0, 3),
]


@pytest.mark.parametrize("kernel", [smcx.KERNEL_AUTO, smcx.KERNEL_GENERIC], ids=["auto", "generic"])
@pytest.mark.parametrize("case", SWEEP_CASES, ids=lambda c: f"{'bcc' if c[0]==0 else 'fcc'}{c[2]}K{c[1]}L{c[6][0]}nt{c[6][1]}s{c[5]}")
def test_sweep_bit_exact(stream, case, kernel):
    kind, K, dims, M, comp, storage, sched, T, n = case
    V = epi_gaussian(K, M, 20.0, 11)
    lat = smcx.Lattice(kind, dims, M, comp, init_seed=3, storage=storage, sched=sched, stream=stream)
    lat.set_kernel(kernel)
    lat.set_epi(V)
    assert lat.schedule() == (sched[0], tuple(sched[1]))
    lat.sweep(T, n, 9)
    got = lat.get_config()
    sw, st = lat.state()
    ref, rst = _oracle_run(kind, dims, M, K, V, comp, 3, T, n, 9, sched)
    assert sw == n
    assert (got == ref).all(), f"{(got != ref).sum()} sites differ"
    assert st.tolist() == rst.tolist()
    assert lat.energy() == O.energy(kind, dims, M, K, V, ref)


@pytest.mark.parametrize("K", [2, 3])
def test_bcc_fewer_shells_large_epi_bit_exact(stream, K):
    """2 and 3 BCC shells with |V| >= 2^15: the tile kernel falls back from
    one counter word and two byte planes to two words and three planes."""
    kind, dims, M = smcx.BCC, (16, 14, 12), 4
    comp = [0.25] * 4
    V = epi_gaussian(K, M, 2000.0, 4)
    assert np.abs(V).max() >= 2**15
    lat = smcx.Lattice(kind, dims, M, comp, init_seed=3, storage=smcx.PACKED4, sched=(3, (2, 2, 2)), stream=stream)
    lat.set_epi(V)
    lat.sweep(5.0e4, 3, 9)
    ref, rst = _oracle_run(kind, dims, M, K, V, comp, 3, 5.0e4, 3, 9, (3, (2, 2, 2)))
    assert (lat.get_config() == ref).all()
    assert lat.state()[1].tolist() == rst.tolist()
    lat.close()


@pytest.mark.parametrize("M", [4, 5])
def test_fcc_large_epi_bit_exact(stream, M):
    """EPI entries near the 2^23 limit of the FCC tile kernel: the kernel's
    intermediate sums leave int32 and must wrap back to the exact dE."""
    kind, K, dims = smcx.FCC, 3, (15, 12, 12)
    comp = [1.0 / M] * M
    V = epi_gaussian(K, M, 20000.0, 4)
    assert np.abs(V).max() < 2**23
    lat = smcx.Lattice(kind, dims, M, comp, init_seed=3, storage=smcx.PACKED4, sched=(3, (2, 2, 2)), stream=stream)
    lat.set_epi(V)
    lat.sweep(2.0e5, 3, 9)
    ref, rst = _oracle_run(kind, dims, M, K, V, comp, 3, 2.0e5, 3, 9, (3, (2, 2, 2)))
    assert (lat.get_config() == ref).all()
    assert lat.state()[1].tolist() == rst.tolist()
    assert lat.energy() == O.energy(kind, dims, M, K, V, ref)
    lat.close()


def test_oracle_sized_workload(stream):
    """BCC 16^3 quaternary, 4 shells, 1000 K, 100 sweeps, seed 1 (the
    oracle-sized workload), library-chosen schedule."""
    w = ORACLE_BCC16
    V = w.epi()
    lat = smcx.Lattice(w.kind, w.dims, w.M, w.comp, init_seed=w.init_seed, storage=w.storage, stream=stream)
    lat.set_epi(V)
    L, nt = lat.schedule()
    lat.sweep(w.temperatures[0], w.sweeps, w.seed)
    got = lat.get_config()
    ref, rst = _oracle_run(w.kind, w.dims, w.M, w.K, V, w.comp, w.init_seed, w.temperatures[0], w.sweeps,
                           w.seed, (L, nt))
    assert (got == ref).all()
    assert lat.state()[1].tolist() == rst.tolist()
    assert lat.energy() == O.energy(w.kind, w.dims, w.M, w.K, V, ref)


def test_split_sweeps_and_resume(stream):
    dims, M, K = (12, 12, 12), 4, 4
    V = epi_gaussian(K, M, 20.0, 2)
    a = smcx.Lattice(smcx.BCC, dims, M, [0.25] * 4, storage=smcx.PACKED4, sched=(3, (2, 2, 2)), stream=stream)
    a.set_epi(V)
    a.sweep(1200.0, 3, 5)
    mid = a.get_config()
    a.sweep(1200.0, 4, 5)
    b = smcx.Lattice(smcx.BCC, dims, M, [0.25] * 4, storage=smcx.PACKED4, sched=(3, (2, 2, 2)), stream=stream)
    b.set_epi(V)
    b.sweep(1200.0, 7, 5)
    assert (a.get_config() == b.get_config()).all()
    # checkpoint / resume: configuration + cumulative sweep counter
    c = smcx.Lattice(smcx.BCC, dims, M, [0.25] * 4, storage=smcx.INT8, sched=(3, (2, 2, 2)), stream=stream)
    c.set_epi(V)
    c.set_config(mid)
    c.set_sweep_counter(3)
    c.sweep(1200.0, 4, 5)
    assert (c.get_config() == b.get_config()).all()


def test_error_codes(stream):
    with pytest.raises(smcx.SmcxError) as e:
        smcx.Lattice(smcx.BCC, (12, 12, 12), 4, [0.25] * 4, sched=(2, (1, 1, 1)), stream=stream)
    assert e.value.code == smcx.E_SCHEDULE
    with pytest.raises(smcx.SmcxError) as e:
        smcx.Lattice(smcx.BCC, (12, 12, 12), 4, [0.25] * 4, sched=(3, (3, 2, 2)), stream=stream)
    assert e.value.code == smcx.E_SCHEDULE
    with pytest.raises(smcx.SmcxError) as e:
        smcx.Lattice(smcx.BCC, (12, 12, 12), 4, [0.5, 0.6, 0.0, 0.0], stream=stream)
    assert e.value.code == smcx.E_INVALID_ARG
    with pytest.raises(smcx.SmcxError) as e:
        smcx.Lattice(smcx.BCC, (12, 12, 12), 16, [1 / 16] * 16, storage=smcx.PACKED4, stream=stream)
    assert e.value.code == smcx.E_INVALID_ARG
    lat = smcx.Lattice(smcx.BCC, (12, 12, 12), 4, [0.25] * 4, stream=stream)
    with pytest.raises(smcx.SmcxError) as e:
        lat.sweep(1000.0, 1, 1)
    assert e.value.code == smcx.E_NO_EPI
    V = epi_gaussian(4, 4, 20.0, 1)
    bad = V.copy()
    bad[0, 0, 1] += 1
    with pytest.raises(smcx.SmcxError) as e:
        lat.set_epi(bad)
    assert e.value.code == smcx.E_INVALID_ARG
    with pytest.raises(smcx.SmcxError) as e:
        lat.set_epi(V * 100000)
    assert e.value.code == smcx.E_RANGE
    lat.set_epi(V)
    for T in (0.0, -5.0, float("nan")):
        with pytest.raises(smcx.SmcxError) as e:
            lat.sweep(T, 1, 1)
        assert e.value.code == smcx.E_INVALID_ARG
    with pytest.raises(smcx.SmcxError) as e:
        lat.set_config(np.full(lat.N, 7, np.int8))
    assert e.value.code == smcx.E_INVALID_ARG
    lat.sweep(1000.0, 0, 1)  # zero sweeps is a no-op
    assert lat.state()[0] == 0


@pytest.mark.parametrize("sigma_mev", [0.4, 20.0, 500.0], ids=["1plane", "2planes", "3planes"])
def test_epi_scale_byte_planes(stream, sigma_mev):
    """The shared-memory BCC kernel splits V into 1, 2 or 3 byte planes by its
    largest entry; every split must give the oracle's trajectory."""
    dims, M, K, sched = (20, 18, 16), 4, 4, (3, (2, 2, 2))
    V = epi_gaussian(K, M, sigma_mev, 21)
    T = 3000.0 if sigma_mev > 100 else 900.0
    lat = smcx.Lattice(smcx.BCC, dims, M, [0.25] * 4, init_seed=4, storage=smcx.PACKED4, sched=sched,
                       stream=stream)
    lat.set_epi(V)
    lat.sweep(T, 3, 2)
    ref, rst = _oracle_run(smcx.BCC, dims, M, K, V, [0.25] * 4, 4, T, 3, 2, sched)
    assert (lat.get_config() == ref).all()
    assert lat.state()[1].tolist() == rst.tolist()


@pytest.mark.parametrize("mode", [smcx.PROPOSAL_TILE, smcx.PROPOSAL_BLOCK], ids=["tile", "block"])
@pytest.mark.parametrize("kernel", [smcx.KERNEL_AUTO, smcx.KERNEL_GENERIC], ids=["auto", "generic"])
@pytest.mark.parametrize("case", [
    (smcx.BCC, 4, (20, 20, 20), 4, [0.25] * 4, smcx.PACKED4, (4, (2, 2, 2)), 1200.0, 4),
    (smcx.BCC, 4, (37, 22, 40), 4, [0.25] * 4, smcx.INT8, (4, (2, 2, 2)), 900.0, 3),     # ragged
    (smcx.BCC, 4, (18, 16, 20), 3, [0.5, 0.3, 0.2], smcx.PACKED4, (3, (2, 2, 2)), 2000.0, 3),  # L=3: generic
    (smcx.BCC, 2, (12, 12, 12), 4, [0.25] * 4, smcx.INT8, (3, (1, 1, 1)), 1000.0, 3),     # link-cell
    (smcx.FCC, 3, (12, 12, 12), 5, [0.3, 0.25, 0.2, 0.15, 0.1], smcx.PACKED4, (3, (4, 4, 4)), 1200.0, 3),
    (smcx.BCC, 4, (36, 24, 20), 4, [0.25] * 4, smcx.PACKED4, (4, (6, 4, 2)), 1200.0, 3),  # 3 blocks per colour
    (smcx.BCC, 4, (29, 18, 18), 4, [0.25] * 4, smcx.INT8, (3, (6, 2, 2)), 900.0, 3),      # odd: last block 1 tile
    (smcx.BCC, 4, (72, 36, 36), 4, [0.25] * 4, smcx.PACKED4, (3, (4, 2, 2)), 1200.0, 3),  # 18-cell tiles, 6^3 slots
    (smcx.BCC, 4, (70, 70, 34), 4, [0.25] * 4, smcx.INT8, (3, (4, 4, 2)), 900.0, 2),      # 17-18 cells, 2 blocks
    (smcx.BCC, 4, (54, 36, 36), 3, [0.5, 0.3, 0.2], smcx.PACKED4, (3, (6, 2, 2)), 1500.0, 2),  # M = 3, odd
    (smcx.BCC, 4, (52, 20, 20), 4, [0.25] * 4, smcx.PACKED4, (4, (4, 2, 2)), 1200.0, 2),  # x origins mod 4: 2, 3, 0, 1
    # FCC shared-direction kernel: byte counters (M = 4), 15/14/13-cell tiles
    (smcx.FCC, 3, (30, 28, 26), 4, [0.25] * 4, smcx.INT8, (3, (2, 2, 2)), 1000.0, 2),
    # six-bit counters (M = 5), ragged tiles, link cells of 4
    (smcx.FCC, 3, (22, 19, 18), 5, [0.3, 0.25, 0.2, 0.15, 0.1], smcx.PACKED4, (4, (2, 2, 2)), 1500.0, 2),
    # M = 2 (one counter word), 3 blocks per colour on x
    (smcx.FCC, 3, (36, 12, 12), 2, [0.6, 0.4], smcx.PACKED4, (3, (6, 2, 2)), 800.0, 2),
], ids=["bcc20", "bcc_ragged", "bcc_L3", "bcc_linkcell", "fcc", "bcc_blocks", "bcc_odd_blocks", "bcc_pair18",
        "bcc_pair_ragged", "bcc_pair_m3", "bcc_word_offsets", "fcc_m4", "fcc_ragged_L4", "fcc_m2_blocks"])
def test_shared_direction_proposals(stream, case, kernel, mode):
    """SMCX_PROPOSAL_TILE: one direction per (sweep, tile, intra colour);
    SMCX_PROPOSAL_BLOCK: one per (sweep, tile colour, block of two tiles,
    intra colour)."""
    kind, K, dims, M, comp, storage, sched, T, n = case
    V = epi_gaussian(K, M, 20.0, 12)
    lat = smcx.Lattice(kind, dims, M, comp, init_seed=5, storage=storage, sched=sched, stream=stream)
    lat.set_kernel(kernel)
    lat.set_proposal(mode)
    lat.set_replica(3)
    lat.set_epi(V)
    lat.sweep(T, n, 4)
    ref = O.init_config(kind, dims, M, comp, 5)
    rst = O.sweep(kind, dims, M, K, V, ref, T, n, 4, replica=3, L=sched[0], nt=sched[1], proposal=mode)
    assert (lat.get_config() == ref).all()
    assert lat.state()[1].tolist() == rst.tolist()


@pytest.mark.parametrize("storage", [smcx.INT8, smcx.PACKED4], ids=["int8", "packed4"])
def test_wrap_caller_store_in_place(stream, storage):
    """smcx_lattice_wrap sweeps a caller-held device buffer in place; the
    buffer then holds the oracle's configuration."""
    kind, K, dims, M = smcx.BCC, 4, (12, 12, 12), 4
    V = epi_gaussian(K, M, 20.0, 3)
    cfg = O.init_config(kind, dims, M, [0.25] * 4, 9)
    if storage == smcx.INT8:
        buf = torch.from_numpy(cfg.copy()).to("cuda")
    else:
        u = cfg.astype(np.uint8)
        buf = torch.from_numpy((u[0::2] | (u[1::2] << 4)).astype(np.uint8)).to("cuda")
    torch.cuda.synchronize()
    lat = smcx.Lattice.wrap(kind, dims, M, buf.data_ptr(), buf.numel(), storage=storage,
                            sched=(3, (4, 4, 4)), stream=stream, owner=buf)
    lat.set_epi(V)
    lat.sweep(1000.0, 2, 5)
    lat.synchronize()
    ref = cfg.copy()
    st = O.sweep(kind, dims, M, K, V, ref, 1000.0, 2, 5, L=3, nt=(4, 4, 4))
    host = buf.cpu().numpy()
    if storage == smcx.INT8:
        got = host.view(np.int8)
    else:
        got = np.empty(cfg.size, np.int8)
        got[0::2] = host & 15
        got[1::2] = host >> 4
    assert (got == ref).all()
    assert (lat.get_config() == ref).all()
    assert lat.state()[1].tolist() == st.tolist()
    assert lat.energy() == O.energy(kind, dims, M, K, V, ref)
    lat.close()
    assert buf.numel() > 0  # the caller's buffer survives the handle


def test_wrap_rejects_bad_store(stream):
    dims, M = (8, 8, 8), 4
    N = 2 * 8 * 8 * 8
    bad = torch.zeros(N, dtype=torch.int8, device="cuda")
    bad[N - 1] = 4  # species id >= M
    with pytest.raises(smcx.SmcxError) as e:
        smcx.Lattice.wrap(smcx.BCC, dims, M, bad.data_ptr(), bad.numel(), stream=stream)
    assert e.value.code == smcx.E_INVALID_ARG
    ok = torch.zeros(N, dtype=torch.int8, device="cuda")
    with pytest.raises(smcx.SmcxError) as e:
        smcx.Lattice.wrap(smcx.BCC, dims, M, ok.data_ptr(), N - 1, stream=stream)
    assert e.value.code == smcx.E_INVALID_ARG
    host = np.zeros(N, np.int8)
    with pytest.raises(smcx.SmcxError) as e:
        smcx.Lattice.wrap(smcx.BCC, dims, M, host.ctypes.data, N, stream=stream)
    assert e.value.code == smcx.E_INVALID_ARG


def test_edge_shorter_than_reach_rejected(stream):
    """A 4-shell BCC table reaches two cells along an axis: an edge of one
    cell is refused before any kernel runs (the gathers wrap once)."""
    lat = smcx.Lattice(smcx.BCC, (1, 8, 8), 4, [0.25] * 4, stream=stream)
    with pytest.raises(smcx.SmcxError) as e:
        lat.set_epi(epi_gaussian(4, 4, 20.0, 1))
    assert e.value.code == smcx.E_INVALID_ARG
    lat.set_epi(epi_gaussian(3, 4, 20.0, 1))  # 3 shells reach one cell: accepted
    cfg = lat.get_config()
    assert lat.energy() == O.energy(smcx.BCC, (1, 8, 8), 4, 3, epi_gaussian(3, 4, 20.0, 1), cfg)
    lat.close()
    d = torch.zeros(2 * 1 * 8 * 8, dtype=torch.int8, device="cuda")
    with pytest.raises(smcx.SmcxError) as e:
        smcx.energy_noalloc(smcx.BCC, (1, 8, 8), 4, smcx.INT8, epi_gaussian(4, 4, 20.0, 1), d.data_ptr(),
                            stream=stream)
    assert e.value.code == smcx.E_INVALID_ARG


@pytest.mark.parametrize("kind,K,dims,M,qsro", [
    (smcx.BCC, 4, (48, 40, 44), 4, False),
    (smcx.FCC, 3, (24, 24, 28), 5, False),
    (smcx.FCC, 3, (24, 24, 24), 4, True),
])
def test_autotune_restores_state_and_stays_exact(stream, kind, K, dims, M, qsro):
    V = epi_gaussian(K, M, 20.0, 2)
    lat = smcx.Lattice(kind, dims, M, [1.0 / M] * M, init_seed=3, storage=smcx.PACKED4, stream=stream)
    lat.set_epi(V)
    W = None
    if qsro:
        W = np.random.default_rng(1).integers(-200, 201, (K, M)).astype(np.int32)
        lat.set_qsro(W)
    lat.sweep(1200.0, 2, 9)
    cfg = lat.get_config()
    cum, st = lat.state()
    (L, nt), th = lat.autotune(1200.0, 1)
    assert lat.schedule() == (L, nt)
    assert (lat.get_config() == cfg).all()
    cum2, st2 = lat.state()
    assert cum2 == cum and st2.tolist() == st.tolist()
    lat.sweep(1200.0, 2, 9)
    ref = cfg.copy()
    if qsro:
        rst = O.sweep_qsro(kind, dims, M, K, V, W, ref, 1200.0, 2, 9, sweep0=2, L=L, nt=nt)
    else:
        rst = O.sweep(kind, dims, M, K, V, ref, 1200.0, 2, 9, sweep0=2, L=L, nt=nt)
    assert (lat.get_config() == ref).all()
    assert (lat.state()[1] - st).tolist() == rst.tolist()
    lat.close()


@pytest.mark.parametrize("storage", [smcx.INT8, smcx.PACKED4], ids=["int8", "packed4"])
def test_config_store_layout_io(stream, storage):
    kind, dims, M = smcx.BCC, (10, 8, 12), 4
    N = O.n_sites(kind, dims)
    cfg = np.random.default_rng(4).integers(0, M, N).astype(np.int8)
    lat = smcx.Lattice(kind, dims, M, [0.25] * 4, storage=storage, stream=stream)
    lat.set_config(cfg)
    raw = lat.get_config_store()
    if storage == smcx.INT8:
        assert raw.size == N and (raw.view(np.int8) == cfg).all()
    else:
        u = cfg.astype(np.uint8)
        assert raw.size == N // 2 and (raw == (u[0::2] | (u[1::2] << 4))).all()
    other = smcx.Lattice(kind, dims, M, [0.25] * 4, init_seed=9, storage=storage, stream=stream)
    before = other.get_config()
    bad = raw.copy()
    bad[3] = 0xF7 if storage == smcx.PACKED4 else 9  # an id >= M
    with pytest.raises(smcx.SmcxError) as e:
        other.set_config_store(bad)
    assert e.value.code == smcx.E_INVALID_ARG
    assert (other.get_config() == before).all()
    with pytest.raises(smcx.SmcxError):
        other.set_config_store(raw[:-1])
    other.set_config_store(raw)
    assert (other.get_config() == cfg).all()
    lat.close()
    other.close()


def test_lds_probe_near_nominal_peak(stream):
    """The measured shared-memory load rate is within a plausible band of the
    nominal one (SMs x 32 lanes x SM clock)."""
    rate = smcx.probe_lds_rate(stream)
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 32 * 2.07e9
    assert 0.3 * nominal < rate < 1.2 * nominal, (rate, nominal)
