"""GPU post-processing of a snapshot sequence (section 2.3 source model, driver of
paper_1004_2503_b300.postprocess) against the oracle fed the same per-interval sources: parity
gates on the final state, and the photons emitted are those of the source model."""
import numpy as np
import pytest

import oracle as O
from oracle import sources_oracle as SO
from paper_1004_2503_b300 import aton as A
from paper_1004_2503_b300 import postprocess as PP
from paper_1004_2503_b300 import workloads as W

from parity_helpers import assert_gates, budget_closure, errors, oracle_params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [A.MODE_FUSED, A.MODE_UNFUSED])
def test_snapshot_sequence_matches_the_oracle(mode):
    st, snaps, run, interval, model = W.snapshot_workload()
    shape = st["nH"].shape
    a = A.from_workload(st, np.zeros(0, np.int64), np.zeros(0), run)
    a.set_exec(mode, 100)
    recs = PP.run_snapshots(a, snaps, shape, run["dx"], run["dt"], interval, model["f_esc"],
                            model["boost_a"], model["boost_k"], model["t0"], stats=True)
    assert a.synchronize() == 0
    f = a.get_fields()
    b = a.photon_budget()
    a.close()
    # the photons the model emits, from the reference source model
    model_photons = 0.0
    for p, r in enumerate(recs):
        t = model["t0"] + (p + 0.5) * interval
        _, rr = SO.star_sources(snaps[p + 1], shape, run["dx"], interval, f_esc=model["f_esc"],
                                a_b=model["boost_a"], k_b=model["boost_k"], t_universe=t)
        model_photons += sum(rr) * interval
        assert r["stars"] == len(snaps[p + 1])          # every star is young and active here
    # the kernels inject each source's rate dt / V rounded to float (and tally what they
    # injected), so the emission agrees with the model to that rounding, 2^-24
    assert b["emitted"] == pytest.approx(model_photons, rel=1e-7)
    assert abs(budget_closure(b)) <= 1e-6
    # oracle run with the same sources, interval by interval
    p = oracle_params(run)
    state, bud, sts = dict(st), None, None
    for r in recs:
        state, bud, sts = O.run(p, state, r["steps"], r["cell"], r["rate"], omp=True,
                                budget=bud, stats=sts)
    e = errors(f, state)
    print("snapshot sequence errors", mode, e, "x_v", recs[-1]["stats"]["x_volume"])
    assert_gates(e, f"mode {mode}")
    assert b["absorbed"] == pytest.approx(bud["absorbed"], rel=1e-3)
    assert recs[-1]["stats"]["x_volume"] > recs[0]["stats"]["x_volume"]
