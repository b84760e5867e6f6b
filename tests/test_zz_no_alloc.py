"""aton_photon_sum_static: the photon count of a device field from an entry point that
allocates no device memory, for callers that cannot let a library allocate (a host code that
owns all device memory through its own fixed pool, or a hook run between time steps where an
allocation could block on queued work). Its scratch is a fixed device array inside the
library, shared by every call.

This file is collected last on purpose: run alone in a fresh process or after every other
test, it must pass either way."""
import ctypes as C

import numpy as np
import pytest

from paper_1004_2503_b300 import aton as A
from paper_1004_2503_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_sum_matches_the_budget_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    st, idx, rate, run = W.workload_small()
    V = run["dx"] ** 3
    a = A.from_workload(st, idx, rate, run)
    try:
        results = []
        for _ in range(2):
            a.step(7)
            ref = a.photon_budget()["stored"]     # the handle's own reduction
            N = a.get_fields(device=True)["N"]
            torch.cuda.synchronize()
            got = A.photon_sum_static(N, V)
            assert ref > 0
            assert got == pytest.approx(ref, rel=1e-12)
            again = A.photon_sum_static(N, V)     # same input, shared scratch reused
            assert again == got
            results.append(got)
        assert results[0] != results[1]           # the second call saw the new state
    finally:
        a.close()


def test_static_sum_of_a_large_field_and_its_size_limit():
    torch = pytest.importorskip("torch")
    n = 3 * 65536 + 123                           # several partial sums and a ragged tail
    x = torch.rand(n, device="cuda", dtype=torch.float32)
    got = A.photon_sum_static(x, 2.0)
    ref = 2.0 * float(x.double().sum())
    assert got == pytest.approx(ref, rel=1e-12)
    L = A.load()
    out = C.c_double()
    rc = L.aton_photon_sum_static(x.data_ptr(), (1 << 30) + 1, 1.0, C.byref(out), None)
    assert rc == A.ERR_BADARG
    assert "static scratch limit" in L.aton_last_message().decode()
    host = np.ones(16, np.float32)
    rc = L.aton_photon_sum_static(host.ctypes.data, 16, 1.0, C.byref(out), None)
    assert rc == A.ERR_BADARG
