"""ctypes wrapper of the C oracle (smcx_oracle.c).

TEST INFRASTRUCTURE ONLY.  Argument marshalling between numpy arrays and the
C functions; every computation happens in the C file, whose header cites the
paper's passages each function follows.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

BCC, FCC = 0, 1
KMAX = 8
NA_MAX = 4096
NB = 1024
KB_MEV = 8.617333262e-2

_lib = None


def lib():
    global _lib
    if _lib is None:
        # SMCX_ORACLE_SANITIZE=1: the AddressSanitizer / UBSan build (the
        # process must preload libasan; see tests/test_oracle_sanitize.py)
        path = _build.build(sanitize=os.environ.get("SMCX_ORACLE_SANITIZE") == "1")
        L = C.CDLL(path)
        i32, i64, u64, dbl, vp = C.c_int, C.c_int64, C.c_uint64, C.c_double, C.c_void_p
        L.orc_sites_per_cell.argtypes = [i32]
        L.orc_shells.argtypes = [i32, i32, vp, vp, i32]
        L.orc_neighbour.argtypes = [i32, i32, i32, i32, i64, vp]
        L.orc_neighbour.restype = i64
        L.orc_check_geometry.argtypes = [i32] * 5
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_philox4x32_10.restype = None
        L.orc_attempt_words.argtypes = [u64, u64, i32, i64, vp, vp]
        L.orc_attempt_words.restype = None
        L.orc_species_counts.argtypes = [i32, vp, i64, vp]
        L.orc_init_config.argtypes = [i32, i32, i32, i32, i32, vp, u64, vp]
        L.orc_pair_counts.argtypes = [i32] * 6 + [vp, vp]
        L.orc_energy.argtypes = [i32] * 6 + [vp, vp]
        L.orc_energy.restype = i64
        L.orc_delta_e.argtypes = [i32] * 6 + [vp, vp, i64, i32]
        L.orc_delta_e.restype = i64
        L.orc_sro.argtypes = [i32] * 6 + [vp, vp]
        L.orc_threshold_tables.argtypes = [dbl, vp, vp, vp]
        L.orc_threshold.argtypes = [vp, i32, vp, i64]
        L.orc_threshold.restype = C.c_uint32
        L.orc_schedule_check.argtypes = [i32] * 9
        L.orc_sweep.argtypes = ([i32] * 6 + [vp, vp, dbl, i64, u64, u64, i32, i32, i32, i32, i32, vp])
        L.orc_sweep_proposal.argtypes = ([i32] * 6 + [vp, vp, dbl, i64, u64, u64, i32, i32, i32, i32, i32, vp, i32])
        L.orc_local_energy2.argtypes = [i32] * 6 + [vp, vp, vp]
        L.orc_local_energy2_qsro.argtypes = [i32] * 6 + [vp, vp, vp, vp]
        L.orc_clusters_qsro.argtypes = [i32] * 6 + [vp, vp, vp, i64, vp, vp]
        L.orc_local_energy2_sample.argtypes = [i32] * 6 + [vp, vp, vp, i64, vp]
        L.orc_clusters.argtypes = [i32] * 6 + [vp, vp, i64, vp, vp]
        L.orc_energy_qsro.argtypes = [i32] * 6 + [vp, vp, vp]
        L.orc_energy_qsro.restype = i64
        L.orc_delta_e_qsro.argtypes = [i32] * 6 + [vp, vp, vp, i64, i32]
        L.orc_delta_e_qsro.restype = i64
        L.orc_schedule_check_model.argtypes = [i32] * 10
        L.orc_tile_pass_qsro.argtypes = ([i32] * 6 + [vp, vp, vp, dbl, u64, u64, i32, i32, i32, i32, i32, i32, i32,
                                                      i32, vp])
        L.orc_sweep_qsro.argtypes = ([i32] * 6 + [vp, vp, vp, dbl, i64, u64, u64, i32, i32, i32, i32, i32, vp])
        L.orc_exchange_round.argtypes = [i32, vp, vp, vp, u64, u64, vp]
        L.orc_sweep_parallel.argtypes = ([i32] * 6 + [vp, vp, dbl, i64, u64, u64, i32, i32, i32, i32, i32, vp,
                                                      i32, vp])
        L.orc_phase_direction.argtypes = [u64, u64, i32, i64, i32, i32]
        L.orc_tile_pass.argtypes = [i32] * 6 + [vp, vp, dbl, u64, u64, i32] + [i32] * 7 + [vp]
        L.orc_init_sample.argtypes = [i32] * 5 + [vp, u64, vp, i32, vp]
        L.orc_phase_of.argtypes = [i32] * 8 + [i64, vp]
        L.orc_phase_of.restype = i64
        L.orc_specific_heat.argtypes = [vp, vp, i64, i64, dbl, vp]
        L.orc_block_direction.argtypes = [u64, u64, i32, i32, i64, i32, i32]
        L.orc_tile_pass_proposal.argtypes = [i32] * 6 + [vp, vp, dbl, u64, u64, i32] + [i32] * 7 + [vp, i32]
        L.orc_sweep_parallel_proposal.argtypes = ([i32] * 6 + [vp, vp, dbl, i64, u64, u64, i32, i32, i32, i32, i32,
                                                               vp, i32, vp, i32])
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def sites_per_cell(kind):
    return lib().orc_sites_per_cell(kind)


def n_sites(kind, dims):
    nx, ny, nz = dims
    return nx * ny * nz * sites_per_cell(kind)


def shells(kind, K):
    """Shell sizes z[K] and vectors [sum z, 3] in half-lattice units."""
    z = np.zeros(KMAX, np.int32)
    v = np.zeros((512, 3), np.int32)
    n = lib().orc_shells(kind, K, _p(z), _p(v), 512)
    if n < 0:
        raise ValueError("bad shell request")
    return z[:K].copy(), v[:n].copy()


def neighbour(kind, dims, s, vec):
    v = np.ascontiguousarray(vec, np.int32)
    return lib().orc_neighbour(kind, *dims, int(s), _p(v))


def check_geometry(kind, dims, K):
    return lib().orc_check_geometry(kind, *dims, K)


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def attempt_words(seed, sweep, replica, site):
    rd = np.zeros(1, np.uint32)
    ru = np.zeros(1, np.uint32)
    lib().orc_attempt_words(seed, sweep, replica, site, _p(rd), _p(ru))
    return int(rd[0]), int(ru[0])


def species_counts(M, comp, N):
    c = np.ascontiguousarray(comp, np.float64)
    out = np.zeros(M, np.int64)
    if lib().orc_species_counts(M, _p(c), N, _p(out)):
        raise ValueError("bad composition")
    return out


def init_config(kind, dims, M, comp, seed):
    sig = np.zeros(n_sites(kind, dims), np.int8)
    c = np.ascontiguousarray(comp, np.float64)
    if lib().orc_init_config(kind, *dims, M, _p(c), seed, _p(sig)):
        raise ValueError("init failed")
    return sig


def pair_counts(kind, dims, M, K, sigma):
    Cc = np.zeros((K, M, M), np.int64)
    sig = np.ascontiguousarray(sigma, np.int8)
    if lib().orc_pair_counts(kind, *dims, M, K, _p(sig), _p(Cc)):
        raise ValueError("pair counts failed")
    return Cc


def energy(kind, dims, M, K, V, sigma):
    Vv = np.ascontiguousarray(V, np.int32)
    sig = np.ascontiguousarray(sigma, np.int8)
    return int(lib().orc_energy(kind, *dims, M, K, _p(Vv), _p(sig)))


def delta_e(kind, dims, M, K, V, sigma, s, d):
    Vv = np.ascontiguousarray(V, np.int32)
    sig = np.ascontiguousarray(sigma, np.int8)
    return int(lib().orc_delta_e(kind, *dims, M, K, _p(Vv), _p(sig), int(s), int(d)))


def sro(kind, dims, M, K, sigma):
    a = np.zeros((K, M, M), np.float64)
    sig = np.ascontiguousarray(sigma, np.int8)
    if lib().orc_sro(kind, *dims, M, K, _p(sig), _p(a)):
        raise ValueError("sro failed")
    return a


def threshold_tables(T):
    A = np.zeros(NA_MAX, np.uint32)
    B = np.zeros(NB, np.uint32)
    nA = np.zeros(1, np.int32)
    if lib().orc_threshold_tables(float(T), _p(A), _p(nA), _p(B)):
        raise ValueError("bad temperature")
    return A, int(nA[0]), B


def threshold(A, nA, B, dE):
    return int(lib().orc_threshold(_p(A), nA, _p(B), int(dE)))


def schedule_check(kind, dims, K, L, nt):
    return lib().orc_schedule_check(kind, *dims, K, L, *nt)


def sweep(kind, dims, M, K, V, sigma, T, n_sweeps, seed, sweep0=0, replica=0,
          L=0, nt=(1, 1, 1), proposal=0):
    """Run n_sweeps in place on sigma (int8, contiguous); returns stats
    (attempts, accepts, same-species proposals, sum of accepted dE).
    proposal: 0 = direction per trial, 1 = shared per (sweep, tile, phase),
    2 = shared per (sweep, tile colour, block of two tiles, phase)."""
    assert sigma.dtype == np.int8 and sigma.flags.c_contiguous
    Vv = np.ascontiguousarray(V, np.int32)
    st = np.zeros(4, np.int64)
    rc = lib().orc_sweep_proposal(kind, *dims, M, K, _p(Vv), _p(sigma), float(T), int(n_sweeps),
                                  int(seed), int(sweep0), int(replica), int(L), *[int(t) for t in nt],
                                  _p(st), int(proposal))
    if rc:
        raise ValueError(f"oracle sweep rejected the request ({rc})")
    return st


def sweep_parallel(kind, dims, M, K, V, sigma, T, n_sweeps, seed, sweep0=0, replica=0,
                   L=0, nt=(1, 1, 1), threads=0, proposal=0):
    """oracle sweep with every phase split across OpenMP threads (identical
    result to sweep()); returns (stats, threads used)."""
    assert sigma.dtype == np.int8 and sigma.flags.c_contiguous
    Vv = np.ascontiguousarray(V, np.int32)
    st = np.zeros(4, np.int64)
    used = np.zeros(1, np.int32)
    rc = lib().orc_sweep_parallel_proposal(kind, *dims, M, K, _p(Vv), _p(sigma), float(T), int(n_sweeps),
                                           int(seed), int(sweep0), int(replica), int(L), *[int(t) for t in nt],
                                           _p(st), int(threads), _p(used), int(proposal))
    if rc:
        raise ValueError(f"oracle sweep rejected the request ({rc})")
    return st, int(used[0])


def energy_qsro(kind, dims, M, K, V, W, sigma):
    """Energy of the qSRO model (pair part + sum_i sum_k W[k][s_i] n_k(i)^2)."""
    Vv, Wv = np.ascontiguousarray(V, np.int32), np.ascontiguousarray(W, np.int32)
    s = np.ascontiguousarray(sigma, np.int8)
    e = lib().orc_energy_qsro(kind, *dims, M, K, _p(Vv), _p(Wv), _p(s))
    if e == np.iinfo(np.int64).min:
        raise ValueError("oracle rejected the request")
    return int(e)


def delta_e_qsro(kind, dims, M, K, V, W, sigma, s, d):
    Vv, Wv = np.ascontiguousarray(V, np.int32), np.ascontiguousarray(W, np.int32)
    assert sigma.dtype == np.int8 and sigma.flags.c_contiguous
    e = lib().orc_delta_e_qsro(kind, *dims, M, K, _p(Vv), _p(Wv), _p(sigma), int(s), int(d))
    if e == np.iinfo(np.int64).min:
        raise ValueError("oracle rejected the request")
    return int(e)


def schedule_check_model(kind, dims, K, L, nt, model):
    return int(lib().orc_schedule_check_model(kind, *dims, K, L, *nt, model))


def sweep_qsro(kind, dims, M, K, V, W, sigma, T, n_sweeps, seed, sweep0=0, replica=0, L=0, nt=(1, 1, 1)):
    """qSRO-model sweeps in place on sigma; returns the statistics."""
    assert sigma.dtype == np.int8 and sigma.flags.c_contiguous
    Vv, Wv = np.ascontiguousarray(V, np.int32), np.ascontiguousarray(W, np.int32)
    st = np.zeros(4, np.int64)
    rc = lib().orc_sweep_qsro(kind, *dims, M, K, _p(Vv), _p(Wv), _p(sigma), float(T), int(n_sweeps), int(seed),
                              int(sweep0), int(replica), int(L), *[int(t) for t in nt], _p(st))
    if rc:
        raise ValueError(f"oracle sweep rejected the request ({rc})")
    return st


def tile_pass_qsro(kind, dims, M, K, V, W, sigma, T, seed, sweep, replica, L, nt, tile):
    """tile_pass for the qSRO model."""
    assert sigma.dtype == np.int8 and sigma.flags.c_contiguous
    Vv, Wv = np.ascontiguousarray(V, np.int32), np.ascontiguousarray(W, np.int32)
    st = np.zeros(4, np.int64)
    rc = lib().orc_tile_pass_qsro(kind, *dims, M, K, _p(Vv), _p(Wv), _p(sigma), float(T), int(seed), int(sweep),
                                  int(replica), int(L), *[int(t) for t in nt], *[int(t) for t in tile], _p(st))
    if rc:
        raise ValueError(f"oracle tile pass rejected the request ({rc})")
    return st


def local_energy2(kind, dims, M, K, V, sigma):
    """Twice the local energy of every site (int64 [N], 0.01 meV)."""
    N = n_sites(kind, dims)
    Vv = np.ascontiguousarray(V, np.int32)
    s = np.ascontiguousarray(sigma, np.int8)
    out = np.zeros(N, np.int64)
    if lib().orc_local_energy2(kind, *dims, M, K, _p(Vv), _p(s), _p(out)):
        raise ValueError("oracle local energy rejected the request")
    return out


def local_energy2_qsro(kind, dims, M, K, V, W, sigma):
    """2 E_i under the qSRO model (pair value + 2 sum_k W[k][s_i] n_k(i)^2)."""
    N = n_sites(kind, dims)
    Vv, Wv = np.ascontiguousarray(V, np.int32), np.ascontiguousarray(W, np.int32)
    s = np.ascontiguousarray(sigma, np.int8)
    out = np.zeros(N, np.int64)
    if lib().orc_local_energy2_qsro(kind, *dims, M, K, _p(Vv), _p(Wv), _p(s), _p(out)):
        raise ValueError("oracle local energy rejected the request")
    return out


def local_energy2_sample(kind, dims, M, K, V, sigma, ids):
    """2 E_i of the listed sites only."""
    Vv = np.ascontiguousarray(V, np.int32)
    s = np.ascontiguousarray(sigma, np.int8)
    idv = np.ascontiguousarray(ids, np.int64)
    out = np.zeros(idv.size, np.int64)
    if lib().orc_local_energy2_sample(kind, *dims, M, K, _p(Vv), _p(s), _p(idv), idv.size, _p(out)):
        raise ValueError("oracle local energy rejected the request")
    return out


def clusters(kind, dims, M, K, V, sigma, thr2):
    """Cluster labels (smallest site id of each cluster) and their count."""
    N = n_sites(kind, dims)
    Vv = np.ascontiguousarray(V, np.int32)
    s = np.ascontiguousarray(sigma, np.int8)
    lab = np.zeros(N, np.int64)
    nc = np.zeros(1, np.int64)
    if lib().orc_clusters(kind, *dims, M, K, _p(Vv), _p(s), int(thr2), _p(lab), _p(nc)):
        raise ValueError("oracle clusters rejected the request")
    return lab, int(nc[0])


def clusters_qsro(kind, dims, M, K, V, W, sigma, thr2):
    """clusters() with the qSRO local energies."""
    N = n_sites(kind, dims)
    Vv, Wv = np.ascontiguousarray(V, np.int32), np.ascontiguousarray(W, np.int32)
    s = np.ascontiguousarray(sigma, np.int8)
    lab = np.zeros(N, np.int64)
    nc = np.zeros(1, np.int64)
    if lib().orc_clusters_qsro(kind, *dims, M, K, _p(Vv), _p(Wv), _p(s), int(thr2), _p(lab), _p(nc)):
        raise ValueError("oracle clusters rejected the request")
    return lab, int(nc[0])


def cluster_summary(labels, sigma, M, min_size):
    """Clusters of at least min_size sites, largest first (ties: smaller
    label first): (labels, sizes, species counts [n][M])."""
    roots, size = np.unique(labels, return_counts=True)
    keep = size >= min_size
    roots, size = roots[keep], size[keep]
    order = np.lexsort((roots, -size))
    roots, size = roots[order], size[order]
    counts = np.zeros((roots.size, M), np.int64)
    for j, r in enumerate(roots):
        counts[j] = np.bincount(np.asarray(sigma)[labels == r], minlength=M)[:M]
    return roots, size, counts


def exchange_round(T_slot, E, slot_rep, rnd, seed, accepts=None):
    """One replica-exchange round (orc_exchange_round); slot_rep (int32) and
    accepts (int64, [R-1]) are updated in place."""
    T = np.ascontiguousarray(T_slot, np.float64)
    Ev = np.ascontiguousarray(E, np.int64)
    assert slot_rep.dtype == np.int32 and slot_rep.flags.c_contiguous
    R = T.size
    acc = accepts if accepts is not None else np.zeros(max(R - 1, 1), np.int64)
    assert acc.dtype == np.int64
    rc = lib().orc_exchange_round(R, _p(T), _p(Ev), _p(slot_rep), int(rnd), int(seed), _p(acc))
    if rc:
        raise ValueError(f"oracle exchange rejected the request ({rc})")
    return slot_rep


def phase_of(kind, dims, L, nt, s):
    t = np.zeros(3, np.int32)
    ph = lib().orc_phase_of(kind, *dims, L, *nt, int(s), _p(t))
    return int(ph), tuple(int(x) for x in t)


def tile_pass(kind, dims, M, K, V, sigma, T, seed, sweep, replica, L, nt, tile, proposal=0):
    """Run every phase of one tile in place (see orc_tile_pass)."""
    assert sigma.dtype == np.int8 and sigma.flags.c_contiguous
    Vv = np.ascontiguousarray(V, np.int32)
    st = np.zeros(4, np.int64)
    rc = lib().orc_tile_pass_proposal(kind, *dims, M, K, _p(Vv), _p(sigma), float(T), int(seed), int(sweep),
                                      int(replica), int(L), *[int(t) for t in nt], *[int(t) for t in tile], _p(st),
                                      int(proposal))
    if rc:
        raise ValueError(f"oracle tile pass rejected the request ({rc})")
    return st


def init_sample(kind, dims, M, comp, seed, ids):
    ids = np.ascontiguousarray(ids, np.int64)
    out = np.zeros(ids.size, np.int8)
    c = np.ascontiguousarray(comp, np.float64)
    if lib().orc_init_sample(kind, *dims, M, _p(c), int(seed), _p(ids), ids.size, _p(out)):
        raise ValueError("init sample failed")
    return out


def phase_direction(seed, sweep, replica, tile, ic, z1):
    return int(lib().orc_phase_direction(int(seed), int(sweep), int(replica), int(tile), int(ic), int(z1)))


def specific_heat(E, n_sites, T, w=None):
    """(mean E, Var E, C_V / (N k_B)) of energies E (int64, 0.01 meV) with
    optional weights w (see orc_specific_heat)."""
    Ev = np.ascontiguousarray(E, np.int64)
    wv = None if w is None else np.ascontiguousarray(w, np.float64)
    assert wv is None or wv.size == Ev.size
    out = np.zeros(3, np.float64)
    rc = lib().orc_specific_heat(_p(Ev), None if wv is None else _p(wv), Ev.size, int(n_sites), float(T), _p(out))
    if rc:
        raise ValueError("oracle specific heat rejected the request")
    return float(out[0]), float(out[1]), float(out[2])


def block_direction(seed, sweep, replica, tc, block, ic, z1):
    return int(lib().orc_block_direction(int(seed), int(sweep), int(replica), int(tc), int(block), int(ic),
                                         int(z1)))
