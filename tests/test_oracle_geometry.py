"""Oracle geometry pins: coordination shells of the cubic lattices.

The shell radii and coordination numbers are textbook facts of the BCC and
FCC lattices (the paper names only "nx x ny x nz x m" cells, Tab.
models_summary, and neighbour lists from relative offsets, Method
"Implementation of SMC-GPU", neighbour-search item).
"""
import numpy as np
import pytest

import oracle as O


def test_bcc_shells_textbook():
    z, v = O.shells(O.BCC, 4)
    assert z.tolist() == [8, 6, 12, 24]
    d2 = (v ** 2).sum(1)
    # radii a*sqrt(3)/2, a, a*sqrt(2), a*sqrt(11)/2 -> squared half-units 3, 4, 8, 11
    start = np.concatenate([[0], np.cumsum(z)])
    for k, want in enumerate([3, 4, 8, 11]):
        assert set(d2[start[k]:start[k + 1]].tolist()) == {want}


def test_fcc_shells_textbook():
    z, v = O.shells(O.FCC, 3)
    assert z.tolist() == [12, 6, 24]
    d2 = (v ** 2).sum(1)
    start = np.concatenate([[0], np.cumsum(z)])
    for k, want in enumerate([2, 4, 6]):  # a/sqrt2, a, a*sqrt(3/2)
        assert set(d2[start[k]:start[k + 1]].tolist()) == {want}


@pytest.mark.parametrize("kind,K", [(O.BCC, 4), (O.FCC, 3)])
def test_shell_order_and_symmetry(kind, K):
    z, v = O.shells(kind, K)
    start = np.concatenate([[0], np.cumsum(z)])
    for k in range(K):
        sh = [tuple(x) for x in v[start[k]:start[k + 1]]]
        assert sh == sorted(sh), "canonical lexicographic order inside a shell"
        assert set(sh) == {tuple(-np.array(x)) for x in sh}, "closed under inversion"


@pytest.mark.parametrize("kind,dims", [(O.BCC, (3, 4, 5)), (O.FCC, (3, 3, 4)), (O.BCC, (2, 2, 2))])
def test_neighbour_round_trip(kind, dims):
    K = 4 if kind == O.BCC else 3
    _, v = O.shells(kind, K)
    N = O.n_sites(kind, dims)
    for s in range(N):
        for vec in v:
            t = O.neighbour(kind, dims, s, vec)
            assert 0 <= t < N
            assert O.neighbour(kind, dims, t, -vec) == s


def test_neighbour_explicit_bcc():
    # site (x=1,y=2,z=3,b=0) in a 4x5x6 box, vector (+1,+1,+1): body centre of the same cell
    dims = (4, 5, 6)
    s = ((3 * 5 + 2) * 4 + 1) * 2 + 0
    assert O.neighbour(O.BCC, dims, s, [1, 1, 1]) == s + 1
    # (-1,-1,-1) from b=0 of cell (1,2,3): body centre of cell (0,1,2)
    assert O.neighbour(O.BCC, dims, s, [-1, -1, -1]) == ((2 * 5 + 1) * 4 + 0) * 2 + 1
    # periodic wrap in x: cell x=3 + (2,0,0) -> cell x=0
    s2 = ((0 * 5 + 0) * 4 + 3) * 2
    assert O.neighbour(O.BCC, dims, s2, [2, 0, 0]) == 0


def test_geometry_rejects_self_images():
    assert O.check_geometry(O.BCC, (2, 2, 2), 4) == 0
    assert O.check_geometry(O.BCC, (1, 4, 4), 2) != 0  # (2,0,0) wraps onto itself
    assert O.check_geometry(O.FCC, (1, 1, 1), 1) == 0
    assert O.check_geometry(O.FCC, (1, 1, 1), 2) != 0  # (2,0,0) wraps onto itself
