"""GPU differentiation path against the oracle.

- Batched pair counts == the oracle's counts (exact).
- EPIEnergy forward/backward == 1/2 V.C and 1/2 sum_b g_b C_b from the
  oracle's counts (FP64 sums rounded to FP32: rtol 1e-6).
- Fluctuation accumulator fed all 12,870 states of the 16-site binary BCC
  box with their Boltzmann weights == the exact derivative -beta cov(A, C/2)
  computed in numpy from the oracle's counts (rtol 1e-10, FP64 sums in a
  different order).
- Sampled fluctuation gradient from GPU sweeps agrees with a common-random-
  number central difference of <A> from GPU sweeps within 4 sigma.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2503_12591_gb300 import smcx
from paper_2503_12591_gb300.inputs import epi_gaussian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
KB = 8.617333262e-2


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    return torch.device("cuda")


@pytest.mark.parametrize("kind,dims,M,K", [(smcx.BCC, (8, 8, 8), 4, 4), (smcx.FCC, (4, 5, 3), 5, 3),
                                           (smcx.BCC, (2, 2, 2), 2, 4)])
def test_pair_counts_batch(dev, kind, dims, M, K):
    from paper_2503_12591_gb300 import diff
    N = O.n_sites(kind, dims)
    rng = np.random.default_rng(4)
    cfg = rng.integers(0, M, (7, N)).astype(np.int8)
    C = diff.pair_counts(torch.from_numpy(cfg).to(dev), kind, dims, M, K).cpu().numpy()
    for b in range(7):
        assert (C[b] == O.pair_counts(kind, dims, M, K, cfg[b])).all()


def test_epi_energy_autograd(dev):
    from paper_2503_12591_gb300 import diff
    dims, M, K, B = (8, 8, 8), 4, 4, 64
    N = O.n_sites(O.BCC, dims)
    cfg = np.stack([np.random.default_rng(b).permutation(np.repeat(np.arange(M), N // M)) for b in range(B)])
    cfg = cfg.astype(np.int8)
    Cref = np.stack([O.pair_counts(O.BCC, dims, M, K, c) for c in cfg]).astype(np.float64)
    Vint = epi_gaussian(K, M, 20.0, 5)
    V = torch.tensor(Vint, dtype=torch.float32, device=dev, requires_grad=True)
    C = diff.pair_counts(torch.from_numpy(cfg).to(dev), O.BCC, dims, M, K)
    E = diff.epi_energy(V, C)
    want = 0.5 * np.einsum("kpq,bkpq->b", Vint.astype(np.float64), Cref)
    np.testing.assert_allclose(E.detach().cpu().numpy(), want, rtol=1e-6)
    for b in range(3):  # integer V: the energy is exact and equals the oracle's
        assert int(round(want[b])) == O.energy(O.BCC, dims, M, K, Vint, cfg[b])
    g = torch.linspace(-1.0, 2.0, B, device=dev)
    (E * g).sum().backward()
    gref = 0.5 * np.einsum("b,bkpq->kpq", g.cpu().numpy().astype(np.float64), Cref)
    np.testing.assert_allclose(V.grad.cpu().numpy(), gref, rtol=1e-6)


def test_fluct_exact_enumeration(dev):
    from paper_2503_12591_gb300 import diff
    dims, M, K, T = (2, 2, 2), 2, 4, 1500.0
    states = []
    for ones in itertools.combinations(range(16), 8):
        s = np.zeros(16, np.int8)
        s[list(ones)] = 1
        states.append(s)
    states = np.array(states)
    Cref = np.array([O.pair_counts(O.BCC, dims, M, K, s) for s in states], np.float64)
    Aref = np.array([O.sro(O.BCC, dims, M, K, s)[0] for s in states])
    V = epi_gaussian(K, M, 5.0, 3).astype(np.float64) / 100.0
    E = 0.5 * np.einsum("kpq,skpq->s", V, Cref)
    beta = 1.0 / (KB * T)
    w = np.exp(-beta * (E - E.min()))
    w /= w.sum()
    EA = np.einsum("s,spq->pq", w, Aref)
    EC = np.einsum("s,skpq->kpq", w, 0.5 * Cref)
    EAC = np.einsum("s,sab,skpq->abkpq", w, Aref, 0.5 * Cref)
    exact = -beta * (EAC - EA[:, :, None, None, None] * EC[None]).reshape(M * M, K, M, M)

    C = diff.pair_counts(torch.from_numpy(states).to(dev), O.BCC, dims, M, K)
    est = diff.FluctuationEstimator(O.BCC, K, M, 0, 16)
    est.add_counts(C, torch.from_numpy(w).to(dev))
    got = est.gradient(T).cpu().numpy()
    scale = np.abs(exact).max()
    np.testing.assert_allclose(got, exact, rtol=1e-10, atol=1e-12 * scale)
    np.testing.assert_allclose(est.mean_A().cpu().numpy(), EA, rtol=1e-12, atol=1e-14)


def _chain(V, T, seed, n_burn, n_meas, dims, M, K, shell, comp):
    from paper_2503_12591_gb300 import diff
    stream = torch.cuda.current_stream()
    lat = smcx.Lattice(smcx.BCC, dims, M, comp, init_seed=11, storage=smcx.INT8, sched=(3, (2, 2, 2)), stream=stream)
    lat.set_epi(V)
    lat.sweep(T, n_burn, seed)
    est = diff.FluctuationEstimator(smcx.BCC, K, M, shell, lat.N)
    for _ in range(n_meas):
        lat.sweep(T, 1, seed)
        est.add_lattice(lat)
    return est


def test_fluct_sampled_vs_crn_difference(dev):
    """Sampled estimator -beta cov(A, C/2) on GPU sweeps against a central
    difference of the sampled <A> at V +- h with common random numbers, over
    8 independent chains (batch means for the error bars)."""
    dims, M, K, T = (6, 6, 6), 2, 4, 1200.0
    comp = [0.5, 0.5]
    V = epi_gaussian(K, M, 10.0, 9)
    i = (0, 0, 1)  # V_1[A][B] and its symmetric partner move together
    h = 100        # 1 meV
    grads, fds = [], []
    for seed in range(1, 9):
        est = _chain(V, T, seed, 200, 400, dims, M, K, 0, comp)
        g = est.gradient(T).cpu().numpy()
        gi = g[0 * M + 1, i[0], i[1], i[2]] + g[0 * M + 1, i[0], i[2], i[1]]  # d alpha_AB / dV (both entries)
        Vp, Vm = V.copy(), V.copy()
        Vp[i] += h
        Vp[i[0], i[2], i[1]] += h
        Vm[i] -= h
        Vm[i[0], i[2], i[1]] -= h
        ap = _chain(Vp, T, seed, 200, 400, dims, M, K, 0, comp).mean_A().cpu().numpy()[0, 1]
        am = _chain(Vm, T, seed, 200, 400, dims, M, K, 0, comp).mean_A().cpu().numpy()[0, 1]
        grads.append(gi)
        fds.append((ap - am) / (2 * h / 100.0))  # per meV
    grads, fds = np.array(grads), np.array(fds)
    sg = grads.std(ddof=1) / np.sqrt(len(grads))
    sf = fds.std(ddof=1) / np.sqrt(len(fds))
    assert abs(grads.mean() - fds.mean()) <= 4.0 * np.sqrt(sg ** 2 + sf ** 2), (grads, fds)
    assert abs(grads.mean()) > 2 * sg  # the derivative is resolved, not zero
