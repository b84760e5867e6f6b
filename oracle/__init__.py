"""FP64 CPU oracle of the ATON M1 radiative-transfer step -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. It wraps the plain C oracle (``aton_oracle.c``) with ctypes and adds the
FP64 NumPy reference of the chemistry-surrogate MLP (``mlp_oracle``). Nothing here is shared
with the GPU path.

Arrays are C-order (nz, ny, nx) with x fastest, float64, cgs units; F is the physical flux.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBS = {}

BC_PERIODIC = 0
BC_TRANSMISSIVE = 1
FLUX_GLF = 0
FLUX_HLL = 1


class Params(C.Structure):
    _fields_ = [
        ("c", C.c_double), ("dx", C.c_double), ("dt", C.c_double),
        ("sigma_n", C.c_double), ("sigma_e", C.c_double), ("e_gamma_eV", C.c_double),
        ("bc", C.c_int), ("fixed_T", C.c_int), ("coll_ion", C.c_int), ("cooling", C.c_int),
        ("max_sub", C.c_int),
        ("T_floor", C.c_double), ("sub_eps", C.c_double), ("y_floor", C.c_double),
        ("clump_R_A", C.c_double), ("clump_R_b", C.c_double),
        ("clump_I_A", C.c_double), ("clump_I_b", C.c_double),
        ("flux", C.c_int),
    ]


class Budget(C.Structure):
    _fields_ = [("emitted", C.c_double), ("absorbed", C.c_double),
                ("escaped", C.c_double), ("clipped", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("substeps_total", C.c_int64), ("substeps_max", C.c_int64),
                ("error_cells", C.c_int64)]


_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)


def lib(omp=False):
    """Load (building if needed) the single-threaded or the OpenMP oracle library."""
    key = "omp" if omp else "st"
    if key not in _LIBS:
        from . import build as _build
        _build.build()
        L = C.CDLL(os.path.join(_HERE, "liboracle_omp.so" if omp else "liboracle.so"))
        for f in ("orc_chi", "orc_alpha_B", "orc_beta_coll", "orc_cool_rec_B",
                  "orc_cool_coll_exc", "orc_cool_brems"):
            getattr(L, f).restype = C.c_double
            getattr(L, f).argtypes = [C.c_double]
        L.orc_default_params.argtypes = [C.POINTER(Params)]
        L.orc_eddington.argtypes = [C.c_double] * 5 + [_D]
        L.orc_cooling_rate.restype = C.c_double
        L.orc_cooling_rate.argtypes = [C.POINTER(Params), C.c_double, C.c_double, C.c_double]
        L.orc_heat_per_ionisation.restype = C.c_double
        L.orc_heat_per_ionisation.argtypes = [C.POINTER(Params)]
        L.orc_transport.argtypes = [C.POINTER(Params), C.c_int, C.c_int, C.c_int] + [_D] * 8 + [_D]
        L.orc_chem_cell.restype = C.c_int
        L.orc_chem_cell.argtypes = [C.POINTER(Params), C.c_double] + [_D] * 7 + [_I64]
        L.orc_step.restype = C.c_int
        L.orc_run.restype = C.c_int
        L.orc_run.argtypes = ([C.POINTER(Params), C.c_int, C.c_int, C.c_int, C.c_int] + [_D] * 7 +
                              [C.c_int64, _I64, _D, C.POINTER(Budget), C.POINTER(Stats)])
        L.orc_cell_step.restype = C.c_int
        L.orc_cell_step.argtypes = ([C.POINTER(Params)] + [_D] * 4 +
                                    [C.c_double] * 4 + [_D])
        L.orc_m1_speeds.argtypes = [_D, C.c_double, C.c_int, _D, _D]
        L.orc_m1_speeds.restype = None
        L.orc_stored.restype = C.c_double
        L.orc_stored.argtypes = [C.POINTER(Params), C.c_int64, _D]
        _LIBS[key] = L
    return _LIBS[key]


def params(**kw):
    """Default parameters (paper's single-group constants) with keyword overrides."""
    p = Params()
    lib().orc_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(a):
    return a.ctypes.data_as(_D)


def chi(f):
    return lib().orc_chi(float(f))


def eddington(N, F, c):
    D = np.zeros(9)
    lib().orc_eddington(float(N), float(F[0]), float(F[1]), float(F[2]), float(c), _ptr(D))
    return D.reshape(3, 3)


def m1_speeds(N, F, c, d):
    """(lo, hi): extreme eigenvalues of the M1 flux Jacobian along axis d."""
    u = np.array([N, F[0], F[1], F[2]], np.float64)
    lo, hi = C.c_double(), C.c_double()
    lib().orc_m1_speeds(_ptr(u), float(c), int(d), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def alpha_B(T):
    return lib().orc_alpha_B(float(T))


def beta_coll(T):
    return lib().orc_beta_coll(float(T))


def cool_rec_B(T):
    return lib().orc_cool_rec_B(float(T))


def cool_coll_exc(T):
    return lib().orc_cool_coll_exc(float(T))


def cool_brems(T):
    return lib().orc_cool_brems(float(T))


def cooling_rate(p, T, x, nH):
    return lib().orc_cooling_rate(C.byref(p), float(T), float(x), float(nH))


def heat_per_ionisation(p):
    return lib().orc_heat_per_ionisation(C.byref(p))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def transport(p, N, Fx, Fy, Fz):
    """Transport only (no clamp, sources or chemistry). Returns (N, Fx, Fy, Fz, escaped)."""
    N, Fx, Fy, Fz = (_f64(a) for a in (N, Fx, Fy, Fz))
    nz, ny, nx = N.shape
    out = [np.empty_like(N) for _ in range(4)]
    esc = C.c_double(0.0)
    lib().orc_transport(C.byref(p), nx, ny, nz, _ptr(N), _ptr(Fx), _ptr(Fy), _ptr(Fz),
                        *(_ptr(o) for o in out), C.byref(esc))
    return (*out, esc.value)


def chem_cell(p, nH, N, F, x, T):
    """Operator Phi on one cell over p.dt. Returns dict(N, F, x, T, absorbed, nsub, err)."""
    v = [C.c_double(float(a)) for a in (N, F[0], F[1], F[2], x, T)]
    ab = C.c_double(0.0)
    ns = C.c_int64(0)
    err = lib().orc_chem_cell(C.byref(p), float(nH), *(C.byref(a) for a in v), C.byref(ab),
                              C.byref(ns))
    return dict(N=v[0].value, F=np.array([v[1].value, v[2].value, v[3].value]), x=v[4].value,
                T=v[5].value, absorbed=ab.value, nsub=ns.value, err=err)


def run(p, state, nsteps, src_idx=None, src_rate=None, omp=False, budget=None, stats=None):
    """Advance ``state`` (dict of N, Fx, Fy, Fz, x, T, nH arrays) by ``nsteps`` steps.

    Returns (new_state, budget_dict, stats_dict). ``budget``/``stats`` continue a previous
    tally when given (as returned by an earlier call).
    """
    st = {k: _f64(state[k]).copy() for k in ("N", "Fx", "Fy", "Fz", "x", "T", "nH")}
    nz, ny, nx = st["N"].shape
    if src_idx is None:
        src_idx = np.zeros(0, np.int64)
        src_rate = np.zeros(0, np.float64)
    si = np.ascontiguousarray(src_idx, dtype=np.int64)
    sr = np.ascontiguousarray(src_rate, dtype=np.float64)
    b = Budget(**(budget or {}))
    s = Stats(**{k: v for k, v in (stats or {}).items()})
    rc = lib(omp).orc_run(C.byref(p), nx, ny, nz, int(nsteps), *(_ptr(st[k]) for k in
                          ("N", "Fx", "Fy", "Fz", "x", "T", "nH")), len(si),
                          si.ctypes.data_as(_I64), _ptr(sr), C.byref(b), C.byref(s))
    if rc < 0:
        raise MemoryError("oracle step failed to allocate")
    bud = dict(emitted=b.emitted, absorbed=b.absorbed, escaped=b.escaped, clipped=b.clipped)
    sts = dict(substeps_total=s.substeps_total, substeps_max=s.substeps_max,
               error_cells=s.error_cells)
    return st, bud, sts


def stored(p, N):
    N = _f64(N)
    return lib().orc_stored(C.byref(p), N.size, _ptr(N))


def cell_step(p, N27, Fx27, Fy27, Fz27, x, T, nH, src_rate=0.0):
    """One step of the centre of a 3x3x3 neighbourhood (ghosts pre-filled by the caller).
    Returns dict(N, Fx, Fy, Fz, x, T, absorbed, err)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (N27, Fx27, Fy27, Fz27)]
    out = np.zeros(7)
    err = lib().orc_cell_step(C.byref(p), *(_ptr(a) for a in arrs), float(x), float(T),
                              float(nH), float(src_rate), _ptr(out))
    return dict(zip(("N", "Fx", "Fy", "Fz", "x", "T", "absorbed"), out), err=err)
