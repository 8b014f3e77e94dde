"""Oracle pins for the initial configuration and the checkerboard schedule.

Initial configuration: the paper starts from random configurations (Results,
FeCoNiAlTi section); the build's reading is an exact-composition placement by
rank of a per-site Philox key.  It is re-derived here with numpy's lexsort of
keys from the (ATen-pinned) Philox.

Schedule: the link-cell generalized checkerboard (Results "Performance of the
SMC-X algorithm"; Method "Implementation of SMC-GPU") is valid only if every
two trials that may run at the same time are independent: neither may change
a site the other reads (the LIZ rule).  The test enumerates, by brute force,
every pair of sites whose trials could interact for SOME choice of partners,
and checks that the schedule never runs such a pair concurrently.  Negative
controls (a link cell one smaller, tiles too thin) must show violations.
"""
import numpy as np
import pytest

import oracle as O


def test_species_counts_largest_remainder():
    assert O.species_counts(4, [0.25] * 4, 8192).tolist() == [2048] * 4
    # 2*25^3 = 31250 sites, 4 species: remainders 0.5 each -> ties go to the lower index
    assert O.species_counts(4, [0.25] * 4, 31250).tolist() == [7813, 7813, 7812, 7812]
    got = O.species_counts(5, [0.3, 0.25, 0.2, 0.15, 0.1], 256_000_000).tolist()
    assert got == [76_800_000, 64_000_000, 51_200_000, 38_400_000, 25_600_000]
    got = O.species_counts(3, [0.5, 0.3, 0.2], 7).tolist()  # 3.5, 2.1, 1.4 -> 4, 2, 1
    assert got == [4, 2, 1]


@pytest.mark.parametrize("kind,dims,M,comp,seed", [
    (O.BCC, (4, 5, 3), 4, [0.25] * 4, 1),
    (O.FCC, (3, 3, 3), 5, [0.3, 0.25, 0.2, 0.15, 0.1], 99),
])
def test_init_matches_lexsort(kind, dims, M, comp, seed):
    N = O.n_sites(kind, dims)
    keys = np.zeros(N, np.uint64)
    for i in range(N):
        o = O.philox([i & 0xFFFFFFFF, i >> 32, 0, 0x80000000], [seed & 0xFFFFFFFF, seed >> 32])
        keys[i] = (int(o[0]) << 32) | int(o[1])
    order = np.lexsort((np.arange(N), keys))
    counts = O.species_counts(M, comp, N)
    want = np.zeros(N, np.int8)
    want[order] = np.repeat(np.arange(M), counts).astype(np.int8)
    got = O.init_config(kind, dims, M, comp, seed)
    assert (got == want).all()


def test_schedule_check_rules():
    # BCC, 4 shells: link cell >= 3, tiles >= 3 cells, tile counts even (or 1 with n % L == 0)
    assert O.schedule_check(O.BCC, (12, 12, 12), 4, 3, (4, 4, 4)) == 0
    assert O.schedule_check(O.BCC, (12, 12, 12), 4, 3, (1, 1, 1)) == 0
    assert O.schedule_check(O.BCC, (12, 12, 12), 4, 2, (1, 1, 1)) != 0
    assert O.schedule_check(O.BCC, (12, 12, 12), 4, 3, (6, 6, 6)) != 0  # tiles of 2
    assert O.schedule_check(O.BCC, (12, 12, 12), 4, 3, (3, 4, 4)) != 0  # odd tile count
    assert O.schedule_check(O.BCC, (10, 12, 12), 4, 3, (1, 4, 4)) != 0  # 10 % 3
    assert O.schedule_check(O.BCC, (12, 12, 12), 2, 2, (1, 1, 1)) != 0  # 2 shells need L >= 3
    assert O.schedule_check(O.BCC, (12, 12, 12), 1, 2, (1, 1, 1)) == 0
    assert O.schedule_check(O.FCC, (12, 12, 12), 3, 3, (4, 4, 4)) == 0
    assert O.schedule_check(O.FCC, (12, 12, 12), 3, 3, (6, 6, 6)) == 0  # FCC gap of 2 suffices
    assert O.schedule_check(O.FCC, (12, 12, 12), 3, 2, (1, 1, 1)) != 0


def _neighbour_table(kind, dims, K):
    z, v = O.shells(kind, K)
    N = O.n_sites(kind, dims)
    nb = np.array([[O.neighbour(kind, dims, s, vec) for vec in v] for s in range(N)], np.int64)
    return z, nb


def _violations(kind, dims, K, L, nt):
    """Pairs of sites that may interact but can run concurrently."""
    z, nb = _neighbour_table(kind, dims, K)
    N = nb.shape[0]
    n1 = nb[:, :z[0]]
    ph = np.zeros(N, np.int64)
    tile = np.zeros((N, 3), np.int64)
    for s in range(N):
        p, t = O.phase_of(kind, dims, L, nt, s)
        ph[s] = p
        tile[s] = t
    m = O.sites_per_cell(kind)
    nA = L ** 3 * m
    tc, ic = ph // nA, ph % nA
    bad = 0
    for s2 in range(N):
        # sites a trial at s2 may read, for any partner choice
        R = np.unique(np.concatenate([[s2], n1[s2], nb[s2], nb[n1[s2]].ravel()]))
        # sites whose trial may write into R: R itself and its shell-1 neighbours
        X = np.unique(np.concatenate([R, n1[R].ravel()]))
        X = X[X != s2]
        same_tc = tc[X] == tc[s2]
        diff_tile = (tile[X] != tile[s2]).any(1)
        conc = same_tc & (diff_tile | (ic[X] == ic[s2]))
        bad += int(conc.sum())
    return bad


@pytest.mark.parametrize("kind,K,dims,L,nt", [
    (O.BCC, 4, (12, 12, 12), 3, (4, 4, 4)),   # thinnest tiles allowed
    (O.BCC, 4, (12, 12, 12), 3, (1, 1, 1)),   # paper link-cell schedule, 3^3 cells
    (O.BCC, 4, (12, 14, 12), 4, (2, 4, 2)),   # uneven-free, L = 4
    (O.BCC, 4, (13, 12, 14), 3, (4, 2, 4)),   # uneven tile sizes (4/3 split)
    (O.FCC, 3, (12, 12, 12), 3, (6, 4, 4)),   # FCC tiles of 2 cells
])
def test_schedule_independence_brute_force(kind, K, dims, L, nt):
    assert O.schedule_check(kind, dims, K, L, nt) == 0
    assert _violations(kind, dims, K, L, nt) == 0


@pytest.mark.parametrize("kind,K,dims,L,nt", [
    (O.BCC, 4, (12, 12, 12), 2, (1, 1, 1)),   # link cell too small
    (O.BCC, 4, (12, 12, 12), 3, (6, 6, 6)),   # tiles of 2 cells: too thin
    (O.FCC, 3, (12, 12, 12), 2, (1, 1, 1)),
])
def test_schedule_checker_finds_violations(kind, K, dims, L, nt):
    assert O.schedule_check(kind, dims, K, L, nt) != 0
    assert _violations(kind, dims, K, L, nt) > 0


@pytest.mark.parametrize("kind,K,dims,L,nt", [
    (O.BCC, 4, (12, 14, 13), 3, (4, 2, 4)),
    (O.FCC, 3, (9, 8, 10), 3, (2, 2, 2)),
])
def test_tile_passes_compose_to_sweep(kind, K, dims, L, nt):
    """Running every tile of colour 0, then colour 1, ... (tiles in a random
    order inside a colour) with the single-tile pass equals the oracle sweep:
    the single-tile pass is the sweep loop restricted to one tile."""
    from paper_2503_12591_gb300.inputs import epi_gaussian
    M = 4
    V = epi_gaussian(K, M, 20.0, 6)
    sig = O.init_config(kind, dims, M, [0.25] * 4, 8)
    a = sig.copy()
    st = O.sweep(kind, dims, M, K, V, a, 1100.0, 1, 3, sweep0=5, replica=2, L=L, nt=nt)
    b = sig.copy()
    rng = np.random.default_rng(1)
    tot = np.zeros(4, np.int64)
    for tc in range(8):
        tiles = [(x, y, z) for z in range(nt[2]) for y in range(nt[1]) for x in range(nt[0])
                 if (x & 1) | ((y & 1) << 1) | ((z & 1) << 2) == tc]
        rng.shuffle(tiles)
        for t in tiles:
            tot += O.tile_pass(kind, dims, M, K, V, b, 1100.0, 3, 5, 2, L, nt, t)
    assert (a == b).all()
    assert tot.tolist() == st.tolist()


def test_init_sample_matches_full_placement():
    dims = (5, 6, 7)
    comp = [0.4, 0.35, 0.25]
    full = O.init_config(O.FCC, dims, 3, comp, 21)
    ids = np.array([0, 1, 17, 333, 500, full.size - 1], np.int64)
    assert (O.init_sample(O.FCC, dims, 3, comp, 21, ids) == full[ids]).all()


@pytest.mark.parametrize("kind,K,dims,L,nt", [
    (O.BCC, 4, (12, 14, 13), 3, (4, 2, 4)),
    (O.BCC, 4, (16, 16, 16), 4, (1, 1, 1)),
    (O.FCC, 3, (9, 8, 10), 3, (2, 2, 2)),
])
def test_parallel_sweep_equals_serial(kind, K, dims, L, nt):
    """Sites of one phase are independent, so splitting every phase across
    threads reproduces the serial sweep exactly."""
    from paper_2503_12591_gb300.inputs import epi_gaussian
    M = 4
    V = epi_gaussian(K, M, 20.0, 6)
    sig = O.init_config(kind, dims, M, [0.25] * 4, 8)
    a, b = sig.copy(), sig.copy()
    st = O.sweep(kind, dims, M, K, V, a, 1300.0, 3, 4, sweep0=2, replica=1, L=L, nt=nt)
    st2, used = O.sweep_parallel(kind, dims, M, K, V, b, 1300.0, 3, 4, sweep0=2, replica=1, L=L, nt=nt,
                                 threads=4)
    assert used >= 1
    assert (a == b).all()
    assert st.tolist() == st2.tolist()
