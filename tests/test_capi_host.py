"""Host-side checks of the C ABI that need no GPU: the library loads, exports every entry
point the header declares, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

from paper_1004_2503_b300 import aton as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "aton.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(aton_[a-z_]+)\s*\(", src)))


def test_header_declarations_are_all_exported():
    L = A.load()
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(A.EXPORTS) == names


def test_strerror_covers_every_code():
    L = A.load()
    for code in (0, -1, -2, -3, -4, -5, -6):
        s = L.aton_strerror(code).decode()
        assert s and s != "unknown status"
    assert L.aton_strerror(-99).decode() == "unknown status"


def test_default_params_are_the_papers_single_group():
    p = A.default_params()
    assert p.sigma_n == 2.93e-18 and p.sigma_e == 2.49e-18 and p.e_gamma_eV == 20.27
    assert p.bc == A.BC_PERIODIC and p.max_sub == 10000 and p.sub_eps == 0.1


@pytest.mark.parametrize("args,msg", [
    ((0, 4, 4, 1.0, 1.0, 0.1), "grid sizes"),
    ((4, 4, -1, 1.0, 1.0, 0.1), "grid sizes"),
    ((2048, 2048, 1024, 1.0, 1.0, 0.1), "2^31"),
    ((4, 4, 4, 0.0, 1.0, 0.1), "positive"),
    ((4, 4, 4, 1.0, 1.0, float("nan")), "positive"),
    ((4, 4, 4, 1.0, 1.0, 0.34), "exceeds 1"),
])
def test_init_rejects_bad_arguments_without_touching_the_device(args, msg):
    L = A.load()
    h = C.c_void_p(123)
    rc = L.aton_init(*args, C.byref(h))
    assert rc == A.ERR_BADARG
    assert h.value is None
    assert msg in L.aton_last_message().decode()


def test_cfl_limit_is_inclusive():
    L = A.load()
    h = C.c_void_p()
    rc = L.aton_init(4, 4, 4, 3.0, 1.0, 1.0, C.byref(h))   # 3 c dt / dx = 1 exactly
    if rc == A.OK:
        L.aton_finalize(h)
    else:
        assert rc == A.ERR_CUDA   # no GPU here: it got past argument checks


def test_null_handle_is_rejected():
    L = A.load()
    assert L.aton_step(None, 1) == A.ERR_BADARG
    assert L.aton_synchronize(None) == A.ERR_BADARG
    p = A.default_params()
    assert L.aton_set_params(None, C.byref(p)) == A.ERR_BADARG
    L.aton_finalize(None)  # no-op


def test_binding_rejects_wrong_host_arrays():
    import numpy as np
    with pytest.raises(TypeError):
        A._ptr(np.zeros(4, np.float64), A.HOST)
    with pytest.raises(TypeError):
        A._ptr(np.zeros((4, 4), np.float32)[:, ::2], A.HOST)
