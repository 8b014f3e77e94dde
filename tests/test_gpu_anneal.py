"""Annealing driver and C_V (Method "MC simulation"): the energy trace read
from the accepted-dE sum must equal the oracle's energy after every sweep, and
the C_V it gives must equal the fluctuation formula applied to the oracle's
trace."""
import numpy as np
import pytest

import oracle as O
from paper_2503_12591_gb300 import anneal, smcx
from paper_2503_12591_gb300.inputs import epi_gaussian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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
        O.sweep(O.BCC, dims, M, K, V, ref, st.T, 3, 2, sweep0=sw, L=sched[0], nt=sched[1])
        sw += 3
        trace = []
        for _ in range(6):
            O.sweep(O.BCC, dims, M, K, V, ref, st.T, 1, 2, sweep0=sw, L=sched[0], nt=sched[1])
            sw += 1
            trace.append(O.energy(O.BCC, dims, M, K, V, ref))
        assert st.energies == trace
        e = np.array(trace, np.float64) * 0.01
        cv = e.var() / (ref.size * (anneal.KB_MEV * st.T) ** 2)
        assert st.cv_per_site == pytest.approx(cv, rel=1e-12)
    assert (lat.get_config() == ref).all()


def test_paper_schedule():
    s = anneal.paper_schedule()
    assert s[0] == 2000.0 and s[-1] == 1000.0 and len(s) == 21
