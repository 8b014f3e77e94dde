"""Parity at the full workload sizes, in the launch configuration bench.py
times (library-chosen schedule and kernel).

- BCC 800^3 (1.024B sites, packed 4-bit) and FCC 400^3 (256M sites, 5
  species): sampled initial species against the oracle's one-pass rank count;
  exact composition; after the first tile colour of a sweep, sampled tiles
  (tile + partner ring) bit-exact against the oracle's single-tile pass; the
  energy change equals the sum of accepted dE; trial count.
- BCC 800^3 with shared-direction proposals (per tile, as bench.py times
  the headline; and per block of two tiles): the same first-colour checks
  against the oracle's single-tile pass in that proposal mode.
- BCC 256^3 (33.5M sites, int8): one whole sweep bit-exact against the
  oracle (configuration and statistics).
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_12591_gb300 import smcx
from paper_2503_12591_gb300.inputs import SCALE_BCC800, SCALE_FCC400, THROUGHPUT_BCC256

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tile_bounds(n, nt, i):
    base, rem = n // nt, n % nt
    return i * base + min(i, rem), base + (1 if i < rem else 0)


def _tile_ring_sites(dims, nt, tile, m):
    idx = []
    ranges = []
    for a in range(3):
        t0, ts = _tile_bounds(dims[a], nt[a], tile[a])
        ranges.append([(c % dims[a]) for c in range(t0 - 1, t0 + ts + 1)])
    for z in ranges[2]:
        for y in ranges[1]:
            for x in ranges[0]:
                cell = (z * dims[1] + y) * dims[0] + x
                idx.extend(cell * m + b for b in range(m))
    return np.array(idx, np.int64)


@pytest.mark.parametrize("work,mode", [(SCALE_BCC800, smcx.PROPOSAL_SITE), (SCALE_FCC400, smcx.PROPOSAL_SITE),
                                       (SCALE_BCC800, smcx.PROPOSAL_TILE), (SCALE_BCC800, smcx.PROPOSAL_BLOCK)],
                         ids=["bcc800", "fcc400", "bcc800_tile", "bcc800_block"])
def test_full_size_first_colour_and_invariants(work, mode):
    stream = torch.cuda.current_stream()
    kind, dims, M = work.kind, work.dims, work.M
    T, seed = work.temperatures[0], work.seed
    m = 2 if kind == smcx.BCC else 4
    lat = smcx.Lattice(kind, dims, M, work.comp, init_seed=work.init_seed, storage=work.storage, stream=stream)
    lat.set_proposal(mode)
    V = work.epi()
    lat.set_epi(V)
    L, nt = lat.schedule()
    cfg0 = lat.get_config()
    N = cfg0.size
    counts = O.species_counts(M, work.comp, N)
    assert (np.bincount(cfg0, minlength=M) == counts).all()
    ids = np.random.default_rng(3).choice(N, 8, replace=False)
    assert (cfg0[ids] == O.init_sample(kind, dims, M, work.comp, work.init_seed, ids)).all()

    E0 = lat.energy()
    lat.sweep_partial(T, seed, 1)
    _, st = lat.state()
    cfg1 = lat.get_config()
    assert lat.energy() - E0 == st[3]
    assert (np.bincount(cfg1, minlength=M) == counts).all()
    colour0 = [(x, y, z) for z in range(0, nt[2], 2) for y in range(0, nt[1], 2) for x in range(0, nt[0], 2)]
    trials = sum(np.prod([_tile_bounds(dims[a], nt[a], t[a])[1] for a in range(3)]) * m for t in colour0)
    assert st[0] == trials

    rng = np.random.default_rng(5)
    picks = [colour0[i] for i in rng.choice(len(colour0), 2, replace=False)]
    for t in picks:
        O.tile_pass(kind, dims, M, work.K, V, cfg0, T, seed, 0, 0, L, nt, t, proposal=mode)
        sites = _tile_ring_sites(dims, nt, t, m)
        assert (cfg1[sites] == cfg0[sites]).all(), f"tile {t}"
    lat.close()


def test_throughput_lattice_one_sweep_bit_exact():
    w = THROUGHPUT_BCC256
    stream = torch.cuda.current_stream()
    lat = smcx.Lattice(w.kind, w.dims, w.M, w.comp, init_seed=w.init_seed, storage=w.storage, stream=stream)
    V = w.epi()
    lat.set_epi(V)
    L, nt = lat.schedule()
    T = w.temperatures[0]
    lat.sweep(T, 1, w.seed)
    got = lat.get_config()
    _, st = lat.state()
    ref = O.init_config(w.kind, w.dims, w.M, w.comp, w.init_seed)
    rst = O.sweep(w.kind, w.dims, w.M, w.K, V, ref, T, 1, w.seed, L=L, nt=nt)
    assert (got == ref).all()
    assert st.tolist() == rst.tolist()
    lat.close()
