"""GPU parity of the ionisation/radiation statistics pass (aton_ionisation_stats) with the FP64
reference evaluated on the same state: histogram and bin counts bit-exact (the bin decisions
compare the same float values with the same float edges), sums to 1e-6 relative (compensated
FP32 per thread, FP64 across)."""
import time

import numpy as np
import pytest

from oracle import stats_oracle as S
from paper_1004_2503_b300 import aton as A
from paper_1004_2503_b300 import workloads as W

pytestmark = pytest.mark.gpu

SCALARS = ("x_volume", "x_mass", "gamma12_volume", "J21_volume", "J21_plateau", "T_volume",
           "T_mass", "photons")


def _compare(a, st, run, **params):
    got = a.ionisation_stats(**params)
    f = a.get_fields()
    ref = S.stats(f["N"], f["y"], f["T"], st["nH"].astype(np.float32), run["c"],
                  run["sigma_n"], run["dx"] ** 3, **params)
    for k in ("hist_y", "hist_J", "bin_count"):
        assert np.array_equal(got[k], ref[k]), k
    assert got["cells"] == ref["cells"] and got["plateau_cells"] == ref["plateau_cells"]
    for k in SCALARS:
        assert got[k] == pytest.approx(ref[k], rel=1e-6, abs=1e-300), k
    for k in ("bin_mean_y", "bin_mean_J21"):
        assert np.allclose(got[k], ref[k], rtol=1e-6, atol=0), k
    return got, ref


# cell counts 17280, 105, 5049, 175 and 18: every remainder modulo the four cells a thread takes
@pytest.mark.parametrize("shape", [(20, 24, 36), (7, 5, 3), (33, 17, 9), (5, 5, 7), (3, 2, 3)])
def test_stats_match_the_reference_on_an_evolved_box(shape):
    st, idx, rate, run = W.workload_small(shape=shape, nsrc=3)
    a = A.from_workload(st, idx, rate, run)
    a.step(30)
    got, ref = _compare(a, st, run)
    # a narrower, finer binning with a different spectral reading and plateau
    _compare(a, st, run, nb_nH=64, nb_y=7, nb_J=33, nH_lo=1e-5, nH_hi=1e-2, y_lo=1e-5,
             J21_lo=1e-3, J21_hi=1e2, spectral_index=0.0, nH_plateau=1e-4)
    # the pass sums in a fixed order: a second call gives the same bits
    again = a.ionisation_stats()
    for k in SCALARS:
        assert again[k] == got[k], k
    a.close()
    assert got["hist_y"].sum() == np.prod(shape)


def test_stats_at_256_cubed_and_timing():
    st, idx, rate, run = W.cosmo_box(256, 2.0, 512, 3, 4)
    a = A.from_workload(st, idx, rate, run)
    a.step(40)
    _compare(a, st, run)
    a.ionisation_stats()
    t0 = time.perf_counter()
    for _ in range(5):
        a.ionisation_stats()
    dt = (time.perf_counter() - t0) / 5
    print(f"stats pass 256^3: {dt * 1e3:.3f} ms per call (host-timed, includes the copies)")
    a.close()


def test_degenerate_states_and_edges():
    shape = (4, 8, 8)
    st, idx, rate, run = W.workload_small(shape=shape, nsrc=1)
    # no radiation, fully ionised gas, densities exactly on bin edges
    E = S.edges(1e-6, 1.0, 48)
    nH = np.resize(E[::3], shape).astype(np.float32)
    st = dict(st, N=np.zeros(shape), Fx=np.zeros(shape), Fy=np.zeros(shape), Fz=np.zeros(shape),
              x=np.ones(shape), nH=nH)
    a = A.from_workload(st, idx[:0], rate[:0], run)
    got, ref = _compare(a, st, run)
    assert got["J21_volume"] == 0.0 and got["x_volume"] == 1.0
    a.close()


def test_stats_argument_errors():
    st, idx, rate, run = W.workload_small(shape=(4, 4, 4), nsrc=1)
    a = A.from_workload(st, idx, rate, run)
    for kw in (dict(nb_nH=0), dict(nb_y=65), dict(nH_lo=0.0), dict(J21_hi=1e-7),
               dict(spectral_index=-3.0)):
        with pytest.raises(A.AtonError):
            a.ionisation_stats(**kw)
    a.close()
