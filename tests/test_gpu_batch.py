"""Batched replicas in one persistent launch versus one-replica-per-launch
sweeps and the oracle (temperature parallelism: Supplementary
"Parallelization opportunities").  Configurations and trial statistics must
match bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2503_12591_gb300 import smcx
from paper_2503_12591_gb300.inputs import epi_gaussian, log_temperatures

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIMS = [(12, 12, 12), (24, 14, 16), (13, 20, 18), (30, 30, 26), (16, 24, 12), (40, 12, 20)]


def _sched(dims, L=3, target=20):
    nt = []
    for n in dims:
        t = 2
        while (n + t - 1) // t > target:
            t += 2
        nt.append(t)
    return (L, tuple(nt))


def _make(dims, r, V, stream, sched, storage=smcx.PACKED4):
    lat = smcx.Lattice(smcx.BCC, dims, 4, [0.25] * 4, init_seed=100 + r, storage=storage, sched=sched,
                       stream=stream)
    lat.set_replica(r)
    lat.set_epi(V)
    return lat


@pytest.fixture(scope="module")
def stream():
    return torch.cuda.current_stream()


def test_batch_equals_plain_and_oracle(stream):
    V = epi_gaussian(4, 4, 20.0, 1)
    T = log_temperatures(len(DIMS), 300.0, 3000.0)
    scheds = [_sched(d, L=3 + (i % 2)) for i, d in enumerate(DIMS)]
    batch_lat = [_make(d, r, V, stream, scheds[r]) for r, d in enumerate(DIMS)]
    b = smcx.Batch(batch_lat, stream)
    b.sweep(T, 3, 7)
    b.sweep(T, 2, 7)  # second call replays the captured graph
    info = b.info()
    assert info["grid"] > 0 and info["threads"] > 0
    for r, d in enumerate(DIMS):
        plain = _make(d, r, V, stream, scheds[r], storage=smcx.INT8)
        plain.sweep(T[r], 5, 7)
        got = batch_lat[r].get_config()
        assert (got == plain.get_config()).all(), f"replica {r} differs from its plain run"
        assert batch_lat[r].state()[1].tolist() == plain.state()[1].tolist()
        assert batch_lat[r].state()[0] == 5
        if r < 3:
            ref = O.init_config(O.BCC, d, 4, [0.25] * 4, 100 + r)
            st = O.sweep(O.BCC, d, 4, 4, V, ref, T[r], 5, 7, replica=r, L=scheds[r][0], nt=scheds[r][1])
            assert (got == ref).all()
            assert batch_lat[r].state()[1].tolist() == st.tolist()
    E = b.energy()
    assert E.tolist() == [l.energy() for l in batch_lat]
    b.close()


@pytest.mark.parametrize("threads", [128, 256])
def test_batch_block_sizes_equal_plain(stream, threads):
    """Tiles of 16-18 cells with link cells of 3 have up to 216 link-cell
    slots: two per thread on 128-thread CTAs, one on 256-thread CTAs.  Both
    block sizes give every replica its own plain trajectory."""
    dims = [(36, 34, 32), (18, 18, 18), (32, 36, 34)]
    V = epi_gaussian(4, 4, 20.0, 3)
    T = log_temperatures(len(dims), 500.0, 2500.0)
    scheds = [_sched(d, L=3, target=18) for d in dims]
    lats = [_make(d, r, V, stream, scheds[r]) for r, d in enumerate(dims)]
    b = smcx.Batch(lats, stream)
    b.set_block(threads)
    b.sweep(T, 3, 13)
    assert b.info()["threads"] == threads
    for r, d in enumerate(dims):
        plain = _make(d, r, V, stream, scheds[r])
        plain.sweep(T[r], 3, 13)
        assert (lats[r].get_config() == plain.get_config()).all(), f"replica {r} differs from its plain run"
        assert lats[r].state()[1].tolist() == plain.state()[1].tolist()
        plain.close()
    with pytest.raises(smcx.SmcxError):
        b.set_block(64)
    b.close()
    for l in lats:
        l.close()


def test_batch_multi_tile_replicas_equal_oracle(stream):
    """Replicas with several tiles per colour (4-6 per axis), so that tiles of
    one replica are swept by different CTAs on different SMs in every colour
    pass and read halo cells other SMs wrote in the previous pass; several
    launches in a row.  Every replica must follow its own oracle
    trajectory."""
    dims = [(24, 24, 24), (36, 20, 28), (30, 30, 18), (12, 12, 12)]
    V = epi_gaussian(4, 4, 20.0, 17)
    T = log_temperatures(len(dims), 600.0, 2400.0)
    scheds = [_sched(d, L=3, target=6) for d in dims]
    lats = [_make(d, r, V, stream, scheds[r]) for r, d in enumerate(dims)]
    b = smcx.Batch(lats, stream)
    for _ in range(3):
        b.sweep(T, 2, 19)
    for r, d in enumerate(dims):
        ref = O.init_config(O.BCC, d, 4, [0.25] * 4, 100 + r)
        st = O.sweep(O.BCC, d, 4, 4, V, ref, T[r], 6, 19, replica=r, L=scheds[r][0], nt=scheds[r][1])
        assert (lats[r].get_config() == ref).all(), f"replica {r} schedule {scheds[r]}"
        assert lats[r].state()[1].tolist() == st.tolist()
    b.close()
    for l in lats:
        l.close()


@pytest.mark.parametrize("mode", [smcx.PROPOSAL_TILE, smcx.PROPOSAL_BLOCK])
@pytest.mark.parametrize("threads", [0, 128, 256])
def test_batch_shared_direction_equals_plain_and_oracle(stream, mode, threads):
    """Shared-direction proposals in the persistent launch: one shell-1
    direction per (sweep, tile, phase), or per (sweep, colour, block of two
    tiles, phase).  Replicas of one and of several tiles per colour, link
    cells of 3 and 4, tiles of up to 216 link-cell slots (256-thread CTAs) or
    125 (either block size); two launches in a row, the second a graph
    replay.  Each replica must equal its plain run and its oracle
    trajectory."""
    dims = [(12, 12, 12), (36, 34, 32), (24, 24, 24), (13, 20, 18), (40, 12, 20)]
    V = epi_gaussian(4, 4, 20.0, 23)
    T = log_temperatures(len(dims), 400.0, 2800.0)
    target = 18 if threads != 128 else 15
    scheds = [_sched(d, L=3, target=target if i != 2 else 6) for i, d in enumerate(dims)]
    scheds[3] = _sched(dims[3], L=4, target=10)
    lats = [_make(d, r, V, stream, scheds[r]) for r, d in enumerate(dims)]
    for l in lats:
        l.set_proposal(mode)
    b = smcx.Batch(lats, stream)
    if threads:
        b.set_block(threads)
    b.sweep(T, 2, 31)
    b.sweep(T, 3, 31)
    if threads:
        assert b.info()["threads"] == threads
    for r, d in enumerate(dims):
        plain = _make(d, r, V, stream, scheds[r], storage=smcx.INT8)
        plain.set_proposal(mode)
        plain.sweep(T[r], 5, 31)
        got = lats[r].get_config()
        assert (got == plain.get_config()).all(), f"replica {r} differs from its plain run"
        assert lats[r].state()[1].tolist() == plain.state()[1].tolist()
        plain.close()
        if r in (0, 2, 3):
            ref = O.init_config(O.BCC, d, 4, [0.25] * 4, 100 + r)
            st = O.sweep(O.BCC, d, 4, 4, V, ref, T[r], 5, 31, replica=r, L=scheds[r][0], nt=scheds[r][1],
                         proposal=mode)
            assert (got == ref).all(), f"replica {r} schedule {scheds[r]}"
            assert lats[r].state()[1].tolist() == st.tolist()
    b.close()
    for l in lats:
        l.close()


def test_batch_mixed_proposal_modes_refused(stream):
    V = epi_gaussian(4, 4, 20.0, 1)
    dims = [(12, 12, 12), (16, 16, 16)]
    lats = [_make(d, r, V, stream, _sched(d)) for r, d in enumerate(dims)]
    lats[1].set_proposal(smcx.PROPOSAL_TILE)
    with pytest.raises(smcx.SmcxError):
        b = smcx.Batch(lats, stream)
        b.sweep(log_temperatures(2, 500.0, 1000.0), 1, 1)
    for l in lats:
        l.close()


def test_batch_autotune_then_oracle(stream):
    V = epi_gaussian(4, 4, 20.0, 2)
    dims = DIMS[:4]
    T = log_temperatures(len(dims), 500.0, 2500.0)
    lats = [_make(d, r, V, stream, _sched(d)) for r, d in enumerate(dims)]
    before = [l.get_config() for l in lats]
    b = smcx.Batch(lats, stream)
    threads = b.autotune(T, trial_sweeps=1)
    assert threads >= 0
    for l, c in zip(lats, before):  # the autotuner restores the configurations
        assert (l.get_config() == c).all()
        assert l.state()[0] == 0
    b.sweep(T, 3, 11)
    for r, (l, d) in enumerate(zip(lats, dims)):
        L, nt = l.schedule()
        ref = O.init_config(O.BCC, d, 4, [0.25] * 4, 100 + r)
        O.sweep(O.BCC, d, 4, 4, V, ref, T[r], 3, 11, replica=r, L=L, nt=nt)
        assert (l.get_config() == ref).all(), f"replica {r} schedule {(L, nt)}"
    b.close()


def test_batch_barrier_timeout_reports_and_recovers(stream):
    """A CTA that never arrives at the grid barrier: the other CTAs give up
    after the time limit, the call returns SMCX_E_TIMEOUT, and the context
    keeps working."""
    V = epi_gaussian(4, 4, 20.0, 3)
    lats = [_make(d, r, V, stream, _sched(d)) for r, d in enumerate(DIMS[:3])]
    b = smcx.Batch(lats, stream)
    b.set_fault(0, 200)
    with pytest.raises(smcx.SmcxError) as e:
        b.sweep([1000.0] * 3, 2, 1)
    assert e.value.code == smcx.E_TIMEOUT
    b.set_fault(-1, 2000)
    b.sweep([1000.0] * 3, 1, 1)
    torch.cuda.synchronize()
    assert lats[0].energy() == lats[0].energy()
    b.close()


def test_replica_exchange_matches_oracle(stream):
    """Batched sweeps with replica exchange against the oracle: per round,
    every replica sweeps at its slot's temperature, then the slot pairs of
    the round's parity exchange by the oracle's rule."""
    V = epi_gaussian(4, 4, 20.0, 1)
    dims, R, spr, n_rounds, seed = (12, 12, 12), 4, 2, 6, 21
    sched = _sched(dims, L=3)
    T_slot = np.array([1000.0, 1040.0, 1080.0, 1120.0])
    lats = [_make(dims, r, V, stream, sched) for r in range(R)]
    b = smcx.Batch(lats, stream)
    rep, ctr, acc = b.exchange(T_slot, np.arange(R), 3, spr, seed)
    rep, ctr, acc = b.exchange(T_slot, rep, n_rounds - 3, spr, seed, round_ctr=ctr, accepts=acc)
    assert ctr == n_rounds

    cfg = [O.init_config(O.BCC, dims, 4, [0.25] * 4, 100 + r) for r in range(R)]
    E = np.array([O.energy(O.BCC, dims, 4, 4, V, c) for c in cfg], np.int64)
    orep = np.arange(R, dtype=np.int32)
    oacc = np.zeros(R - 1, np.int64)
    for i in range(n_rounds):
        T_rep = np.empty(R)
        T_rep[orep] = T_slot
        for r in range(R):
            st = O.sweep(O.BCC, dims, 4, 4, V, cfg[r], T_rep[r], spr, seed, sweep0=i * spr, replica=r,
                         L=sched[0], nt=sched[1])
            E[r] += st[3]
        O.exchange_round(T_slot, E, orep, i, seed, oacc)
    assert rep.tolist() == orep.tolist()
    assert acc.tolist() == oacc.tolist()
    for r in range(R):
        assert (lats[r].get_config() == cfg[r]).all(), f"replica {r}"
        assert lats[r].energy() == E[r]
    assert acc.sum() > 0  # the chosen temperatures exchange now and then


def test_replica_exchange_rejects_bad_input(stream):
    V = epi_gaussian(4, 4, 20.0, 1)
    lats = [_make((12, 12, 12), 0, V, stream, _sched((12, 12, 12))),
            _make((14, 12, 12), 1, V, stream, _sched((14, 12, 12)))]
    b = smcx.Batch(lats, stream)
    with pytest.raises(smcx.SmcxError):
        b.exchange([1000.0, 1100.0], [0, 1], 1, 1, 3)  # shapes differ
    lats2 = [_make((12, 12, 12), r, V, stream, _sched((12, 12, 12))) for r in range(2)]
    b2 = smcx.Batch(lats2, stream)
    with pytest.raises(smcx.SmcxError):
        b2.exchange([1000.0, 1100.0], [0, 0], 1, 1, 3)  # not a permutation
    with pytest.raises(smcx.SmcxError):
        b2.exchange([1000.0, -1.0], [0, 1], 1, 1, 3)


def test_batch_fluct_accumulate_equals_per_lattice(stream):
    """smcx_batch_fluct_accumulate gives every replica the same FP64 sums as
    smcx_lattice_fluct_accumulate on that replica alone (same integer counts,
    same accumulation order)."""
    from paper_2503_12591_gb300 import diff
    V = epi_gaussian(4, 4, 20.0, 1)
    dims_list = [(12, 12, 12), (24, 14, 16), (13, 20, 18)]
    scheds = [_sched(d, L=3 + (i % 2)) for i, d in enumerate(dims_list)]
    lats = [_make(d, r, V, stream, scheds[r]) for r, d in enumerate(dims_list)]
    b = smcx.Batch(lats, stream)
    T = [900.0, 1100.0, 1300.0]
    est = diff.BatchFluctuationEstimator(b, 4, 4, 1)
    single = [diff.FluctuationEstimator(smcx.BCC, 4, 4, 1, l.N) for l in lats]
    for _ in range(3):
        b.sweep(T, 2, 5)
        est.add()
        for l, e in zip(lats, single):
            e.add_lattice(l)
    torch.cuda.synchronize()
    for r, e in enumerate(single):
        assert torch.equal(est.acc[r], e.acc), f"replica {r}"
    g = est.gradients(1000.0)
    assert torch.equal(g[1], single[1].gradient(1000.0))
