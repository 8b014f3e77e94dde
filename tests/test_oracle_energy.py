"""Oracle energy-model pins (Method "The EPI and qSRO model").

Closed forms of ordered structures the paper names (B2 in MoNbTaW, L1_2 in
FeCoNiAlTi), derived here from the shell geometry by hand; the pure-element
energy; the pair-count row-sum identity; and the swap energy change against
brute force E(after) - E(before), including tiny periodic boxes where shell
vectors alias onto the same site.
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_12591_gb300.inputs import epi_gaussian


def _b2(dims):
    N = O.n_sites(O.BCC, dims)
    sig = np.zeros(N, np.int8)
    sig[1::2] = 1  # A (0) on cube corners, B (1) on body centres
    return sig


def test_b2_energy_closed_form():
    dims = (4, 4, 4)
    V = epi_gaussian(4, 2, 20.0, 3).astype(np.int64)
    sig = _b2(dims)
    N = sig.size
    A, B = 0, 1
    # unordered pairs per site: shell1 AB 4, shell2 AA 3/4 & BB 3/4, shell3 AA 3/2 & BB 3/2, shell4 AB 12
    want4 = (16 * V[0, A, B] + 6 * (V[1, A, A] + V[1, B, B]) + 12 * (V[2, A, A] + V[2, B, B])
             + 48 * V[3, A, B])
    assert 4 * O.energy(O.BCC, dims, 2, 4, V, sig) == N * want4


def test_l12_energy_closed_form():
    dims = (4, 4, 4)
    V = epi_gaussian(3, 2, 20.0, 4).astype(np.int64)
    N = O.n_sites(O.FCC, dims)
    sig = np.zeros(N, np.int8)  # A = 0 on face centres
    sig[0::4] = 1  # B = 1 on cube corners (A3B)
    A, B = 0, 1
    want4 = (12 * V[0, A, B] + 12 * V[0, A, A] + 3 * V[1, B, B] + 9 * V[1, A, A]
             + 24 * V[2, A, B] + 24 * V[2, A, A])
    assert 4 * O.energy(O.FCC, dims, 2, 3, V, sig) == N * want4


@pytest.mark.parametrize("kind,K,z", [(O.BCC, 4, [8, 6, 12, 24]), (O.FCC, 3, [12, 6, 24])])
def test_pure_element(kind, K, z):
    dims = (3, 4, 5)
    V = epi_gaussian(K, 3, 20.0, 5).astype(np.int64)
    N = O.n_sites(kind, dims)
    for p in range(3):
        sig = np.full(N, p, np.int8)
        twice = N * sum(z[k] * V[k, p, p] for k in range(K))
        assert 2 * O.energy(kind, dims, 3, K, V, sig) == twice


@pytest.mark.parametrize("kind,K,dims", [(O.BCC, 4, (5, 4, 6)), (O.FCC, 3, (4, 5, 3))])
def test_pair_count_identities(kind, K, dims):
    M = 4
    z, _ = O.shells(kind, K)
    N = O.n_sites(kind, dims)
    sig = np.random.default_rng(9).integers(0, M, N).astype(np.int8)
    C = O.pair_counts(kind, dims, M, K, sig)
    Np = np.bincount(sig, minlength=M)
    for k in range(K):
        assert (C[k].sum(1) == z[k] * Np).all()
        assert (C[k] == C[k].T).all()
    V = epi_gaussian(K, M, 20.0, 2).astype(np.int64)
    assert 2 * O.energy(kind, dims, M, K, V, sig) == int((V * C).sum())


@pytest.mark.parametrize("kind,K,dims", [
    (O.BCC, 4, (2, 2, 2)),   # 16 sites: shell-4 vectors alias onto shell-1 sites
    (O.BCC, 4, (3, 2, 4)),
    (O.BCC, 4, (6, 6, 6)),
    (O.FCC, 3, (2, 2, 2)),
    (O.FCC, 3, (3, 4, 3)),
])
def test_delta_e_brute_force(kind, K, dims):
    M = 4
    z, v = O.shells(kind, K)
    N = O.n_sites(kind, dims)
    rng = np.random.default_rng(17)
    V = epi_gaussian(K, M, 20.0, 8)
    sig = rng.integers(0, M, N).astype(np.int8)
    E0 = O.energy(kind, dims, M, K, V, sig)
    sites = range(N) if N <= 64 else rng.choice(N, 40, replace=False)
    for s in sites:
        for d in range(z[0]):
            sp = O.neighbour(kind, dims, s, v[d])
            s2 = sig.copy()
            s2[s], s2[sp] = s2[sp], s2[s]
            assert O.delta_e(kind, dims, M, K, V, sig, s, d) == O.energy(kind, dims, M, K, V, s2) - E0


def test_b2_sro():
    dims = (4, 4, 4)
    a = O.sro(O.BCC, dims, 2, 4, _b2(dims))
    # shell 1: every neighbour of A is B -> alpha_AB = 1 - 1/(1/2) = -1, alpha_AA = +1
    assert a[0, 0, 1] == -1.0 and a[0, 1, 0] == -1.0
    assert a[0, 0, 0] == 1.0 and a[0, 1, 1] == 1.0
    # shell 2 (same sublattice): alpha_AA = 1 - 1/(1/2) = -1
    assert a[1, 0, 0] == -1.0 and a[1, 0, 1] == 1.0


def test_random_sro_near_zero():
    dims = (16, 16, 16)
    sig = O.init_config(O.BCC, dims, 4, [0.25] * 4, 5)
    a = O.sro(O.BCC, dims, 4, 4, sig)
    assert np.abs(a).max() < 0.05
