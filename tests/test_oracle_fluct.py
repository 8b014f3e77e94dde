"""Pin of the thermal-derivative identity used by the fluctuation estimator.

For <A> = sum_s A(s) e^{-beta E(s)} / Z with E = 1/2 sum_i V_i C_i(s)
(Eq. Total_EPI pair form; Supplementary "Statistical mechanics"), the
derivative d<A>/dV_i equals -beta cov(A, C_i / 2).  On the 16-site BCC box
(binary 8/8, 12,870 states) both sides are computed exactly from the
oracle's pair counts: the covariance, and a central finite difference of the
enumerated <A>(V) itself.  A dropped 1/2, a sign error or a wrong beta unit
fails this test.
"""
import itertools

import numpy as np

import oracle as O
from paper_2503_12591_gb300.inputs import epi_gaussian

KB = 8.617333262e-2  # meV/K


def enumerate_states():
    dims = (2, 2, 2)
    states, C, A = [], [], []
    for ones in itertools.combinations(range(16), 8):
        s = np.zeros(16, np.int8)
        s[list(ones)] = 1
        states.append(s)
        C.append(O.pair_counts(O.BCC, dims, 2, 4, s))
        A.append(O.sro(O.BCC, dims, 2, 4, s)[0])  # shell-1 alpha [2, 2]
    return np.array(states), np.array(C, np.float64), np.array(A)


def thermal(Vmev, C, A, T):
    E = 0.5 * np.einsum("kpq,skpq->s", Vmev, C)  # meV
    beta = 1.0 / (KB * T)
    w = np.exp(-beta * (E - E.min()))
    w /= w.sum()
    return w, beta


def test_covariance_equals_finite_difference():
    _, C, A = enumerate_states()
    V = epi_gaussian(4, 2, 5.0, 3).astype(np.float64) / 100.0  # meV
    T = 1500.0
    w, beta = thermal(V, C, A, T)
    EA = np.einsum("s,spq->pq", w, A)
    EC = np.einsum("s,skpq->kpq", w, 0.5 * C)
    EAC = np.einsum("s,sab,skpq->abkpq", w, A, 0.5 * C)
    grad = -beta * (EAC - EA[:, :, None, None, None] * EC[None, None])
    h = 1e-3
    for (k, p, q) in [(0, 0, 1), (1, 1, 1), (3, 0, 0), (2, 1, 0)]:
        Vp, Vm = V.copy(), V.copy()
        Vp[k, p, q] += h
        Vm[k, p, q] -= h
        wp, _ = thermal(Vp, C, A, T)
        wm, _ = thermal(Vm, C, A, T)
        fd = (np.einsum("s,spq->pq", wp, A) - np.einsum("s,spq->pq", wm, A)) / (2 * h)
        np.testing.assert_allclose(grad[:, :, k, p, q], fd, rtol=1e-5, atol=1e-9)
    # the derivative along a null direction of V (the row-sum identity
    # sum_q C_k[p][q] = z_k N_p is fixed at fixed composition) vanishes
    null = np.zeros_like(V)
    null[2, 0, :] = 1.0
    null[2, :, 0] += 1.0
    assert abs(np.einsum("abkpq,kpq->ab", grad, null)).max() < 1e-12
