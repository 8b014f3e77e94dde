"""qSRO-model sweeps on the GPU against the oracle (Method "The EPI and qSRO
model", Eq. quadratic_local_SRO, integer form): configuration, trial
statistics and energy bit-exact after several sweeps, for FCC (the paper's
qSRO system, 4x4x4 link cells) and BCC, both storages, explicit and
automatic schedules; the energy change equals the sum of accepted dE."""
import numpy as np
import pytest

import oracle as O
from paper_2503_12591_gb300 import smcx
from paper_2503_12591_gb300.inputs import epi_gaussian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def stream():
    return torch.cuda.current_stream()


def _w(K, M, seed, scale=300):
    return np.random.default_rng(seed).integers(-scale, scale + 1, (K, M)).astype(np.int32)


CASES = [
    # kind, K, dims, M, storage, schedule (None = library choice), T, sweeps
    (smcx.FCC, 3, (12, 8, 8), 4, smcx.INT8, (4, (4, 2, 2)), 1000.0, 3),
    (smcx.FCC, 3, (16, 12, 14), 5, smcx.PACKED4, None, 1200.0, 2),
    (smcx.FCC, 2, (10, 12, 8), 3, smcx.PACKED4, (4, (2, 2, 2)), 800.0, 3),
    # tiles of 20/19/18 cells (the largest the even-point FCC kernel takes,
    # 5^3 trial slots) and tiles of 22 cells (the generic kernel)
    (smcx.FCC, 3, (40, 38, 36), 4, smcx.INT8, (4, (2, 2, 2)), 1000.0, 1),
    (smcx.FCC, 2, (40, 38, 36), 5, smcx.PACKED4, (5, (2, 2, 2)), 900.0, 1),
    (smcx.FCC, 3, (44, 8, 8), 4, smcx.PACKED4, (4, (2, 2, 2)), 1000.0, 2),
    # 8 species: the largest pair and quadratic tables
    (smcx.FCC, 3, (12, 16, 8), 8, smcx.INT8, (4, (2, 2, 2)), 1100.0, 2),
    (smcx.BCC, 2, (12, 12, 12), 4, smcx.INT8, (4, (4, 4, 4)), 1000.0, 3),
    (smcx.BCC, 4, (20, 16, 16), 4, smcx.PACKED4, None, 1500.0, 2),
]


@pytest.mark.parametrize("kind,K,dims,M,storage,sched,T,n", CASES)
def test_qsro_sweep_bit_exact(stream, kind, K, dims, M, storage, sched, T, n):
    V = epi_gaussian(K, M, 20.0, 11)
    W = _w(K, M, 12)
    lat = smcx.Lattice(kind, dims, M, [1.0 / M] * M, init_seed=5, storage=storage, sched=sched, stream=stream)
    lat.set_epi(V)
    lat.set_qsro(W)
    L, nt = lat.schedule()
    assert O.schedule_check_model(kind, dims, K, L, nt, 1) == 0
    cfg = lat.get_config()
    E0 = lat.energy()
    assert E0 == O.energy_qsro(kind, dims, M, K, V, W, cfg)
    lat.sweep(T, n, 21)
    got = lat.get_config()
    _, st = lat.state()
    ref = cfg.copy()
    rst = O.sweep_qsro(kind, dims, M, K, V, W, ref, T, n, 21, L=L, nt=nt)
    assert (got == ref).all()
    assert st.tolist() == rst.tolist()
    assert lat.energy() == O.energy_qsro(kind, dims, M, K, V, W, ref) == E0 + st[3]
    lat.close()


def test_qsro_schedule_rules(stream):
    V = epi_gaussian(3, 4, 20.0, 1)
    # a link cell of 3 serves the pair model but not qSRO on FCC
    lat = smcx.Lattice(smcx.FCC, (12, 12, 12), 4, [0.25] * 4, sched=(3, (4, 4, 4)), stream=stream)
    lat.set_epi(V)
    with pytest.raises(smcx.SmcxError) as e:
        lat.set_qsro(_w(3, 4, 1))
    assert e.value.code == smcx.E_SCHEDULE
    lat.close()
    # automatic schedule grows to L = 4; W = None returns to the pair model
    lat = smcx.Lattice(smcx.FCC, (16, 16, 16), 4, [0.25] * 4, stream=stream)
    lat.set_epi(V)
    assert lat.schedule()[0] == 3
    lat.set_qsro(_w(3, 4, 1))
    assert lat.schedule()[0] == 4
    lat.set_qsro(None)
    assert lat.schedule()[0] == 3
    with pytest.raises(smcx.SmcxError) as e:
        lat.set_qsro(np.full((3, 4), 2_000_000, np.int32))
    assert e.value.code == smcx.E_RANGE
    lat.close()
    lat = smcx.Lattice(smcx.FCC, (8, 8, 8), 4, [0.25] * 4, stream=stream)
    with pytest.raises(smcx.SmcxError) as e:
        lat.set_qsro(np.zeros((3, 4), np.int32))
    assert e.value.code == smcx.E_NO_EPI
    lat.close()


def test_qsro_zero_weights_equal_pair_model(stream):
    """W = 0 gives the pair model's trajectory through the qSRO kernel."""
    kind, K, dims, M = smcx.FCC, 3, (12, 12, 12), 4
    V = epi_gaussian(K, M, 20.0, 3)
    a = smcx.Lattice(kind, dims, M, [0.25] * 4, init_seed=2, sched=(4, (2, 2, 2)), stream=stream)
    a.set_epi(V)
    a.set_qsro(np.zeros((K, M), np.int32))
    b = smcx.Lattice(kind, dims, M, [0.25] * 4, init_seed=2, sched=(4, (2, 2, 2)), stream=stream)
    b.set_epi(V)
    a.sweep(900.0, 2, 4)
    b.sweep(900.0, 2, 4)
    assert (a.get_config() == b.get_config()).all()
    assert a.state()[1].tolist() == b.state()[1].tolist()


def _tile_bounds(n, nt, i):
    base, rem = n // nt, n % nt
    return i * base + min(i, rem), base + (1 if i < rem else 0)


def _tile_ring_sites(dims, nt, tile, m):
    ranges = []
    for a in range(3):
        t0, ts = _tile_bounds(dims[a], nt[a], tile[a])
        ranges.append([(c % dims[a]) for c in range(t0 - 1, t0 + ts + 1)])
    idx = [((z * dims[1] + y) * dims[0] + x) * m + b
           for z in ranges[2] for y in ranges[1] for x in ranges[0] for b in range(m)]
    return np.array(idx, np.int64)


def test_qsro_full_size_fcc400_first_colour(stream):
    """FCC 400^3 (256M sites, the scale workload) under the qSRO model, in the
    launch configuration bench.py times: after the first tile colour, sampled
    tiles (tile + partner ring) bit-exact against the oracle's single-tile
    pass; energy change = sum of accepted dE; trial count."""
    from paper_2503_12591_gb300.inputs import SCALE_FCC400 as w
    V = w.epi()
    W = _w(w.K, w.M, 77)
    lat = smcx.Lattice(w.kind, w.dims, w.M, w.comp, init_seed=w.init_seed, storage=w.storage, stream=stream)
    lat.set_epi(V)
    lat.set_qsro(W)
    L, nt = lat.schedule()
    cfg0 = lat.get_config()
    E0 = lat.energy()
    lat.sweep_partial(1000.0, 31, 1)
    _, st = lat.state()
    cfg1 = lat.get_config()
    assert lat.energy() - E0 == st[3]
    colour0 = [(x, y, z) for z in range(0, nt[2], 2) for y in range(0, nt[1], 2) for x in range(0, nt[0], 2)]
    trials = sum(np.prod([_tile_bounds(w.dims[a], nt[a], t[a])[1] for a in range(3)]) * 4 for t in colour0)
    assert st[0] == trials
    rng = np.random.default_rng(8)
    for i in rng.choice(len(colour0), 2, replace=False):
        t = colour0[i]
        O.tile_pass_qsro(w.kind, w.dims, w.M, w.K, V, W, cfg0, 1000.0, 31, 0, 0, L, nt, t)
        sites = _tile_ring_sites(w.dims, nt, t, 4)
        assert (cfg1[sites] == cfg0[sites]).all(), f"tile {t}"
    lat.close()


@pytest.mark.parametrize("kind,K,dims,M", [(smcx.FCC, 3, (12, 8, 8), 4), (smcx.BCC, 2, (12, 12, 12), 3)])
def test_qsro_local_energy_and_clusters(stream, kind, K, dims, M):
    V = epi_gaussian(K, M, 20.0, 11)
    W = _w(K, M, 12)
    lat = smcx.Lattice(kind, dims, M, [1.0 / M] * M, init_seed=5, stream=stream)
    lat.set_epi(V)
    lat.set_qsro(W)
    lat.sweep(900.0, 2, 3)
    cfg = lat.get_config()
    N = cfg.size
    e2 = torch.empty(N, dtype=torch.int32, device="cuda")
    lat.local_energy(e2.data_ptr())
    lat.synchronize()
    want = O.local_energy2_qsro(kind, dims, M, K, V, W, cfg)
    got = e2.cpu().numpy().astype(np.int64)
    assert (got == want).all()
    assert got.sum() == 2 * lat.energy()
    lab = torch.empty(N, dtype=torch.int32, device="cuda")
    thr = int(np.quantile(want, 0.4))
    nc = lat.clusters(thr, lab.data_ptr())
    olab, onc = O.clusters_qsro(kind, dims, M, K, V, W, cfg, thr)
    assert nc == onc
    assert (lab.cpu().numpy().astype(np.int64) == olab).all()
    lat.close()


def test_qsro_sweep_energies_trace(stream):
    """smcx_sweep_energies under the qSRO model: the recorded energy after
    each sweep equals the oracle's qSRO energy of its configuration."""
    kind, K, dims, M, sched = smcx.FCC, 3, (12, 8, 8), 4, (4, (4, 2, 2))
    V = epi_gaussian(K, M, 20.0, 11)
    W = _w(K, M, 12)
    lat = smcx.Lattice(kind, dims, M, [0.25] * 4, init_seed=5, sched=sched, stream=stream)
    lat.set_epi(V)
    lat.set_qsro(W)
    ref = lat.get_config()
    E = lat.sweep_energies(900.0, 4, 13)
    for i in range(4):
        O.sweep_qsro(kind, dims, M, K, V, W, ref, 900.0, 1, 13, sweep0=i, L=sched[0], nt=sched[1])
        assert E[i] == O.energy_qsro(kind, dims, M, K, V, W, ref)
    assert (lat.get_config() == ref).all()
    assert lat.state()[0] == 4


@pytest.mark.parametrize("K,dims,M,storage,sched,calls", [
    # tiles of 3 cells on two axes (the smallest the count kernel takes)
    (3, (12, 6, 8), 5, smcx.PACKED4, (4, (4, 2, 2)), (1, 2, 1)),
    (3, (6, 6, 6), 4, smcx.INT8, (4, (2, 2, 2)), (2, 2)),
    # 17-cell tiles: the largest of the 66 KB box (three CTAs per SM)
    (3, (34, 34, 20), 4, smcx.INT8, (4, (2, 2, 2)), (1, 1)),
    # 18-cell tiles: the 101 KB box
    (3, (36, 34, 20), 5, smcx.PACKED4, (4, (2, 2, 2)), (1, 1)),
    # two shells, six species, 20-cell tiles
    (2, (40, 40, 40), 6, smcx.PACKED4, (4, (2, 2, 2)), (1,)),
])
def test_qsro_count_kernel_shapes_and_calls(stream, K, dims, M, storage, sched, calls):
    """The FCC maintained-count kernel at its tile-size limits, with several
    sweep calls in a row: the counts are recomputed at the start of each
    call and carried through its sweeps, so every call must continue the
    oracle's trajectory bit for bit."""
    V = epi_gaussian(K, M, 20.0, 41)
    W = _w(K, M, 42)
    lat = smcx.Lattice(smcx.FCC, dims, M, [1.0 / M] * M, init_seed=9, storage=storage, sched=sched, stream=stream)
    lat.set_epi(V)
    lat.set_qsro(W)
    ref = lat.get_config()
    done = 0
    for n in calls:
        lat.sweep(1000.0, n, 23)
        st = O.sweep_qsro(smcx.FCC, dims, M, K, V, W, ref, 1000.0, n, 23, sweep0=done, L=sched[0], nt=sched[1])
        done += n
        assert (lat.get_config() == ref).all(), f"after {done} sweeps"
    assert lat.state()[0] == done
    assert lat.energy() == O.energy_qsro(smcx.FCC, dims, M, K, V, W, ref)
    lat.close()
