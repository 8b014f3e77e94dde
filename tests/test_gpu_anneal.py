"""Annealing driver and C_V (Results, Fig. C_V; Method "MC simulation").

The library records the exact energy after every sweep and reduces the trace
to <E>, Var(E) and C_V / (N k_B) on the device (smcx_sweep_cv).  The trace
must equal the oracle's energy after every sweep, bit for bit, and the
moments must equal the oracle's orc_specific_heat on that trace to 1e-12
relative (the oracle's specific heat is pinned by exact enumeration in
tests/test_oracle_cv.py).
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_12591_gb300 import anneal, smcx
from paper_2503_12591_gb300.inputs import epi_gaussian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _oracle_trace(dims, M, K, V, ref, T, discard, record, seed, sw, sched):
    O.sweep(O.BCC, dims, M, K, V, ref, T, discard, seed, sweep0=sw, L=sched[0], nt=sched[1])
    sw += discard
    trace = []
    for _ in range(record):
        O.sweep(O.BCC, dims, M, K, V, ref, T, 1, seed, sweep0=sw, L=sched[0], nt=sched[1])
        sw += 1
        trace.append(O.energy(O.BCC, dims, M, K, V, ref))
    return np.array(trace, np.int64), sw


def test_energy_trace_and_cv_match_oracle():
    dims, M, K, sched = (12, 12, 12), 4, 4, (3, (2, 2, 2))
    V = epi_gaussian(K, M, 20.0, 4)
    lat = smcx.Lattice(smcx.BCC, dims, M, [0.25] * 4, init_seed=6, storage=smcx.PACKED4, sched=sched,
                       stream=torch.cuda.current_stream())
    lat.set_epi(V)
    temps = [2000.0, 1950.0, 1900.0]
    steps = anneal.anneal(lat, temps, discard=3, record=6, seed=2, keep_energies=True)
    ref = O.init_config(O.BCC, dims, M, [0.25] * 4, 6)
    sw = 0
    for st in steps:
        trace, sw = _oracle_trace(dims, M, K, V, ref, st.T, 3, 6, 2, sw, sched)
        assert st.energies == trace.tolist()
        mean, var, cv = O.specific_heat(trace, ref.size, st.T)
        assert st.mean_E == pytest.approx(mean, rel=1e-12)
        assert st.var_E == pytest.approx(var, rel=1e-12)
        assert st.cv_per_site == pytest.approx(cv, rel=1e-12)
    assert (lat.get_config() == ref).all()


@pytest.mark.parametrize("record", [1, 37, 600])
def test_sweep_cv_long_trace(record):
    """Moments over traces shorter and longer than the reduction's 512
    threads; without the trace download (E = NULL)."""
    dims, M, K, sched, T = (12, 12, 12), 4, 4, (3, (2, 2, 2)), 2500.0
    V = epi_gaussian(K, M, 20.0, 9)
    lat = smcx.Lattice(smcx.BCC, dims, M, [0.25] * 4, init_seed=3, storage=smcx.INT8, sched=sched,
                       stream=torch.cuda.current_stream())
    lat.set_epi(V)
    _, mean, var, cv = lat.sweep_cv(T, record, 5, want_trace=False)
    ref = O.init_config(O.BCC, dims, M, [0.25] * 4, 3)
    trace, _ = _oracle_trace(dims, M, K, V, ref, T, 0, record, 5, 0, sched)
    om, ov, oc = O.specific_heat(trace, ref.size, T)
    assert mean == pytest.approx(om, rel=1e-12)
    if record == 1:
        assert var == 0.0 and cv == 0.0
    else:
        assert var == pytest.approx(ov, rel=1e-12)
        assert cv == pytest.approx(oc, rel=1e-12)
    with pytest.raises(smcx.SmcxError):
        lat.sweep_cv(T, 0, 5)
    lat.close()


def test_paper_schedule():
    s = anneal.paper_schedule()
    assert s[0] == 2000.0 and s[-1] == 1000.0 and len(s) == 21
