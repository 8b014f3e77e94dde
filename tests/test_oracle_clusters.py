"""Oracle pins for the local-energy field and the clusters (Results,
FeCoNiAlTi one-billion-atom section; Method "MC simulation": local energy
per site, an energy threshold, union-find over neighbouring sites).

e2[i] = 2 E_i = sum over the shells and their vectors of V_k[s_i][s_{i+v}].
Pinned against hand-counted environments of ordered structures (B2, L1_2,
pure elements) and the sum rule; clusters against scipy's
connected_components on the explicitly built neighbour graph.
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_12591_gb300.inputs import epi_gaussian

scipy_sparse = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


def test_pure_element_local_energy():
    V = epi_gaussian(4, 3, 20.0, 2)
    sig = np.full(O.n_sites(O.BCC, (4, 4, 4)), 2, np.int8)
    e2 = O.local_energy2(O.BCC, (4, 4, 4), 3, 4, V, sig)
    want = 8 * V[0, 2, 2] + 6 * V[1, 2, 2] + 12 * V[2, 2, 2] + 24 * V[3, 2, 2]
    assert (e2 == want).all()


def test_b2_local_energy_and_singletons():
    # B2: species 0 on the cube corners (b = 0), species 1 on the body centres
    dims = (4, 5, 3)
    V = epi_gaussian(4, 2, 20.0, 4)
    N = O.n_sites(O.BCC, dims)
    sig = np.tile(np.array([0, 1], np.int8), N // 2)
    e2 = O.local_energy2(O.BCC, dims, 2, 4, V, sig)
    eA = 8 * V[0, 0, 1] + 6 * V[1, 0, 0] + 12 * V[2, 0, 0] + 24 * V[3, 0, 1]
    eB = 8 * V[0, 1, 0] + 6 * V[1, 1, 1] + 12 * V[2, 1, 1] + 24 * V[3, 1, 0]
    assert (e2[0::2] == eA).all() and (e2[1::2] == eB).all()
    assert e2.sum() == 2 * O.energy(O.BCC, dims, 2, 4, V, sig)
    if eA != eB:
        # threshold between the two: every shell-1 neighbour is of the other
        # class, so every site is its own cluster
        thr = max(eA, eB)
        lab, nc = O.clusters(O.BCC, dims, 2, 4, V, sig, thr)
        assert nc == N and (lab == np.arange(N)).all()
    # threshold above both: one cluster, labelled 0
    lab, nc = O.clusters(O.BCC, dims, 2, 4, V, sig, max(eA, eB) + 1)
    assert nc == 1 and (lab == 0).all()


def test_l12_local_energy():
    # FCC A3B with B (species 1) on the cube corners (b = 0)
    dims = (3, 3, 4)
    V = epi_gaussian(3, 2, 30.0, 5)
    N = O.n_sites(O.FCC, dims)
    sig = np.tile(np.array([1, 0, 0, 0], np.int8), N // 4)
    e2 = O.local_energy2(O.FCC, dims, 2, 3, V, sig)
    eB = 12 * V[0, 1, 0] + 6 * V[1, 1, 1] + 24 * V[2, 1, 0]
    eA = 4 * V[0, 0, 1] + 8 * V[0, 0, 0] + 6 * V[1, 0, 0] + 8 * V[2, 0, 1] + 16 * V[2, 0, 0]
    assert (e2[0::4] == eB).all()
    for b in (1, 2, 3):
        assert (e2[b::4] == eA).all()
    assert e2.sum() == 2 * O.energy(O.FCC, dims, 2, 3, V, sig)


def _scipy_labels(kind, dims, cls):
    N = cls.size
    z, vecs = O.shells(kind, 1)
    rows, cols = [], []
    for s in range(N):
        for v in vecs[:z[0]]:
            t = O.neighbour(kind, dims, s, v)
            if cls[s] == cls[t]:
                rows.append(s)
                cols.append(t)
    g = scipy_sparse.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(N, N)).tocsr()
    nc, lab = csgraph.connected_components(g, directed=False)
    first = np.full(nc, N, np.int64)
    np.minimum.at(first, lab, np.arange(N))
    return first[lab], nc


@pytest.mark.parametrize("kind,dims,M,K,q", [
    (O.BCC, (5, 4, 6), 4, 4, 0.5),
    (O.BCC, (6, 6, 6), 3, 4, 0.2),
    (O.FCC, (4, 3, 5), 5, 3, 0.5),
    (O.FCC, (3, 4, 3), 2, 3, 0.8),
])
def test_clusters_match_connected_components(kind, dims, M, K, q):
    N = O.n_sites(kind, dims)
    sig = np.random.default_rng(7).integers(0, M, N).astype(np.int8)
    V = epi_gaussian(K, M, 20.0, 8)
    e2 = O.local_energy2(kind, dims, M, K, V, sig)
    assert e2.sum() == 2 * O.energy(kind, dims, M, K, V, sig)
    thr = int(np.quantile(e2, q))
    lab, nc = O.clusters(kind, dims, M, K, V, sig, thr)
    want, nc2 = _scipy_labels(kind, dims, e2 < thr)
    assert nc == nc2
    assert (lab == want).all()


def test_cluster_summary_by_hand():
    labels = np.array([0, 0, 2, 0, 2, 5, 5, 5, 5])
    sigma = np.array([1, 0, 2, 1, 2, 0, 0, 1, 2])
    roots, size, counts = O.cluster_summary(labels, sigma, 3, 2)
    assert roots.tolist() == [5, 0, 2]
    assert size.tolist() == [4, 3, 2]
    assert counts.tolist() == [[2, 1, 1], [1, 2, 0], [0, 0, 2]]


def test_sampled_local_energy_equals_full():
    dims = (5, 4, 3)
    N = O.n_sites(O.FCC, dims)
    sig = np.random.default_rng(2).integers(0, 3, N).astype(np.int8)
    V = epi_gaussian(3, 3, 20.0, 1)
    full = O.local_energy2(O.FCC, dims, 3, 3, V, sig)
    ids = np.array([0, 7, 100, N - 1], np.int64)
    assert (O.local_energy2_sample(O.FCC, dims, 3, 3, V, sig, ids) == full[ids]).all()
