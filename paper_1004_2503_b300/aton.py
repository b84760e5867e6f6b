"""Thin ctypes binding of libaton.so (include/aton.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels. Arrays are passed either as
NumPy float32 arrays (host) or as contiguous float32 torch CUDA tensors (device); nothing is
computed here. If the library is missing, loading raises instead of falling back to anything.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaton.so")

OK = 0
ERR_BADARG, ERR_NOMEM, ERR_CUDA, ERR_SUBCYCLE, ERR_NONFINITE, ERR_STATE = -1, -2, -3, -4, -5, -6
HOST, DEVICE = 0, 1
BC_PERIODIC, BC_TRANSMISSIVE = 0, 1
SRC_REPLACE, SRC_APPEND = 0, 1
MODE_FUSED, MODE_UNFUSED, MODE_FUSED_LDG = 0, 1, 2
FLUX_GLF, FLUX_HLL = 0, 1
B_EMITTED, B_STORED, B_ABSORBED, B_ESCAPED, B_CLIPPED, B_STORED0 = range(6)
BUDGET_LEN = 6
BUDGET_KEYS = ("emitted", "stored", "absorbed", "escaped", "clipped", "stored0")

# every entry point declared in include/aton.h
EXPORTS = (
    "aton_default_params", "aton_init", "aton_finalize", "aton_set_params", "aton_get_params",
    "aton_set_stream", "aton_set_exec", "aton_get_exec", "aton_set_tile", "aton_set_tile_rows",
    "aton_get_tile_rows", "aton_autotune", "aton_set_fields",
    "aton_get_fields", "aton_add_sources", "aton_step", "aton_synchronize",
    "aton_photon_budget", "aton_set_budget", "aton_get_diag", "aton_last_error_cells",
    "aton_launches_per_step", "aton_strerror", "aton_last_message", "aton_photon_sum_static",
    "aton_set_pair_sink", "aton_pair_count", "aton_default_surrogate_params", "aton_set_surrogate",
    "aton_mlp_create", "aton_mlp_destroy", "aton_mlp_num_params", "aton_mlp_set_params",
    "aton_mlp_get_params", "aton_mlp_fit_norm", "aton_mlp_get_norm", "aton_mlp_set_norm",
    "aton_mlp_features", "aton_mlp_forward", "aton_mlp_loss_grad", "aton_mlp_train_step",
    "aton_mlp_synchronize", "aton_default_stats_params", "aton_ionisation_stats",
    "aton_equilibrium_neutral_fraction", "aton_star_sources", "aton_budget_request",
    "aton_budget_collect",
)
# layout of aton_star: 7 doubles
STAR_DTYPE = np.dtype([("x", "<f8"), ("y", "<f8"), ("z", "<f8"), ("mass", "<f8"), ("age", "<f8"),
                       ("lifetime", "<f8"), ("photons_per_baryon", "<f8")])
STATS_MAX_BINS = 64


class aton_params(C.Structure):
    _fields_ = [
        ("sigma_n", C.c_double), ("sigma_e", C.c_double), ("e_gamma_eV", C.c_double),
        ("bc", C.c_int), ("fixed_T", C.c_int), ("coll_ion", C.c_int), ("cooling", C.c_int),
        ("max_sub", C.c_int),
        ("T_floor", C.c_double), ("sub_eps", C.c_double), ("y_floor", C.c_double),
        ("clump_R_A", C.c_double), ("clump_R_b", C.c_double),
        ("clump_I_A", C.c_double), ("clump_I_b", C.c_double),
        ("flux", C.c_int),
    ]


class aton_diag(C.Structure):
    _fields_ = [("steps", C.c_int64), ("substeps_total", C.c_int64),
                ("substeps_max", C.c_int64), ("error_cells", C.c_int64),
                ("nonfinite_cells", C.c_int64), ("surrogate_cells", C.c_int64),
                ("max_f", C.c_double)]


class aton_surrogate_params(C.Structure):
    _fields_ = [("enabled", C.c_int), ("gate_substeps", C.c_double), ("residual_max", C.c_double)]


class aton_stats_params(C.Structure):
    _fields_ = [("nb_nH", C.c_int), ("nb_y", C.c_int), ("nb_J", C.c_int),
                ("nH_lo", C.c_double), ("nH_hi", C.c_double), ("y_lo", C.c_double),
                ("y_hi", C.c_double), ("J21_lo", C.c_double), ("J21_hi", C.c_double),
                ("spectral_index", C.c_double), ("nH_plateau", C.c_double)]


class aton_stats(C.Structure):
    _fields_ = [("x_volume", C.c_double), ("x_mass", C.c_double),
                ("gamma12_volume", C.c_double), ("J21_volume", C.c_double),
                ("J21_plateau", C.c_double), ("T_volume", C.c_double), ("T_mass", C.c_double),
                ("photons", C.c_double), ("cells", C.c_int64), ("plateau_cells", C.c_int64)]


class aton_source_model(C.Structure):
    _fields_ = [("interval", C.c_double), ("f_esc", C.c_double), ("boost_a", C.c_double),
                ("boost_k", C.c_double), ("t_universe", C.c_double)]


class AtonError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


_lib = None
_VP = C.c_void_p


def load():
    """Load libaton.so (built by paper_1004_2503_b300.build); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_1004_2503_b300.build` "
            "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    L.aton_default_params.argtypes = [C.POINTER(aton_params)]
    L.aton_default_params.restype = None
    L.aton_init.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                            C.POINTER(_VP)]
    L.aton_finalize.argtypes = [_VP]
    L.aton_finalize.restype = None
    L.aton_set_params.argtypes = [_VP, C.POINTER(aton_params)]
    L.aton_get_params.argtypes = [_VP, C.POINTER(aton_params)]
    L.aton_set_stream.argtypes = [_VP, _VP]
    L.aton_set_exec.argtypes = [_VP, C.c_int, C.c_int]
    L.aton_set_tile.argtypes = [_VP, C.c_int, C.c_int]
    L.aton_set_tile_rows.argtypes = [_VP, C.c_int]
    L.aton_get_tile_rows.argtypes = [_VP, C.POINTER(C.c_int)]
    L.aton_get_exec.argtypes = [_VP] + [C.POINTER(C.c_int)] * 4
    L.aton_autotune.argtypes = [_VP, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_float)]
    L.aton_set_fields.argtypes = [_VP] + [_VP] * 8 + [C.c_int]
    L.aton_get_fields.argtypes = [_VP] + [_VP] * 7 + [C.c_int]
    L.aton_add_sources.argtypes = [_VP, _VP, _VP, C.c_int64, C.c_int]
    L.aton_step.argtypes = [_VP, C.c_int]
    L.aton_synchronize.argtypes = [_VP]
    L.aton_photon_budget.argtypes = [_VP, C.POINTER(C.c_double)]
    L.aton_set_budget.argtypes = [_VP, C.POINTER(C.c_double)]
    L.aton_budget_request.argtypes = [_VP]
    L.aton_budget_collect.argtypes = [_VP, C.POINTER(C.c_double)]
    L.aton_get_diag.argtypes = [_VP, C.POINTER(aton_diag)]
    L.aton_last_error_cells.argtypes = [_VP, C.POINTER(C.c_int64)]
    L.aton_launches_per_step.argtypes = [_VP, C.POINTER(C.c_int)]
    L.aton_strerror.argtypes = [C.c_int]
    L.aton_strerror.restype = C.c_char_p
    L.aton_photon_sum_static.argtypes = [_VP, C.c_int64, C.c_double, C.POINTER(C.c_double), _VP]
    L.aton_set_pair_sink.argtypes = [_VP, _VP, C.c_int64, C.c_int]
    L.aton_pair_count.argtypes = [_VP, C.POINTER(C.c_int64)]
    L.aton_default_surrogate_params.argtypes = [C.POINTER(aton_surrogate_params)]
    L.aton_default_surrogate_params.restype = None
    L.aton_set_surrogate.argtypes = [_VP, _VP, C.POINTER(aton_surrogate_params)]
    L.aton_mlp_create.argtypes = [C.POINTER(_VP), C.c_ulonglong]
    L.aton_mlp_destroy.argtypes = [_VP]
    L.aton_mlp_destroy.restype = None
    L.aton_mlp_num_params.argtypes = []
    L.aton_mlp_set_params.argtypes = [_VP, _VP, C.c_int]
    L.aton_mlp_get_params.argtypes = [_VP, _VP, C.c_int]
    L.aton_mlp_fit_norm.argtypes = [_VP, _VP, C.c_int64, C.c_double]
    L.aton_mlp_get_norm.argtypes = [_VP, _VP]
    L.aton_mlp_set_norm.argtypes = [_VP, _VP]
    L.aton_mlp_features.argtypes = [_VP, _VP, C.c_int64, C.c_double, _VP, _VP]
    L.aton_mlp_forward.argtypes = [_VP, _VP, C.c_int64, _VP]
    L.aton_mlp_loss_grad.argtypes = [_VP, _VP, _VP, C.c_int, _VP, C.POINTER(C.c_double)]
    L.aton_mlp_train_step.argtypes = [_VP, _VP, _VP, C.c_int, C.c_float, C.POINTER(C.c_double)]
    L.aton_mlp_synchronize.argtypes = [_VP]
    L.aton_default_stats_params.argtypes = [C.POINTER(aton_stats_params)]
    L.aton_ionisation_stats.argtypes = [_VP, C.POINTER(aton_stats_params), C.POINTER(aton_stats),
                                        _VP, _VP, _VP, _VP, _VP]
    L.aton_equilibrium_neutral_fraction.argtypes = [_VP, C.c_int, C.c_double, C.c_double,
                                                    C.c_int, C.c_double, C.c_double, _VP]
    L.aton_star_sources.argtypes = [_VP, C.c_int64, C.POINTER(aton_source_model), C.c_int,
                                    C.c_int, C.c_int, C.c_double, _VP, _VP]
    L.aton_last_message.argtypes = []
    L.aton_last_message.restype = C.c_char_p
    for name in EXPORTS:
        fn = getattr(L, name)
        if fn.restype is C.c_int or name in ("aton_init",):
            fn.restype = C.c_int
    _lib = L
    return L


def _check(code, where):
    if code != OK:
        L = load()
        raise AtonError(code, where, (L.aton_last_message() or b"").decode() or
                        L.aton_strerror(code).decode())
    return code


def default_params():
    p = aton_params()
    load().aton_default_params(C.byref(p))
    return p


def _ptr(a, where):
    """(pointer, where) of a float32 NumPy array or torch CUDA tensor; None passes NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise TypeError("host arrays must be C-contiguous float32")
        return a.ctypes.data
    # torch tensor
    if getattr(a, "is_cuda", False):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise TypeError("device tensors must be contiguous float32")
        return a.data_ptr()
    raise TypeError("expected a NumPy array or a torch CUDA tensor")


def _where(arrays):
    dev = [getattr(a, "is_cuda", False) for a in arrays if a is not None]
    if all(dev):
        return DEVICE
    if not any(dev):
        return HOST
    raise TypeError("mix of host and device arrays")


class Aton:
    """One simulation handle (aton_init ... aton_finalize)."""

    def __init__(self, nx, ny, nz, dx, c, dt):
        self.L = load()
        h = _VP()
        _check(self.L.aton_init(int(nx), int(ny), int(nz), float(dx), float(c), float(dt),
                                C.byref(h)), "aton_init")
        self.h = h
        self.shape = (int(nz), int(ny), int(nx))
        self.ncell = int(nx) * int(ny) * int(nz)

    def close(self):
        if getattr(self, "h", None):
            self.L.aton_finalize(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configuration
    def set_params(self, **kw):
        p = aton_params()
        _check(self.L.aton_get_params(self.h, C.byref(p)), "aton_get_params")
        for k, v in kw.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        _check(self.L.aton_set_params(self.h, C.byref(p)), "aton_set_params")

    def get_params(self):
        p = aton_params()
        _check(self.L.aton_get_params(self.h, C.byref(p)), "aton_get_params")
        return {k: getattr(p, k) for k, _ in aton_params._fields_}

    def set_stream(self, stream):
        ptr = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        _check(self.L.aton_set_stream(self.h, ptr), "aton_set_stream")

    def set_exec(self, mode=MODE_FUSED, graph_batch=100):
        _check(self.L.aton_set_exec(self.h, int(mode), int(graph_batch)), "aton_set_exec")

    def get_exec(self):
        v = [C.c_int() for _ in range(4)]
        _check(self.L.aton_get_exec(self.h, *(C.byref(x) for x in v)), "aton_get_exec")
        return dict(zip(("mode", "graph_batch", "ty", "tz"), (x.value for x in v)))

    def set_tile(self, ty, tz):
        _check(self.L.aton_set_tile(self.h, int(ty), int(tz)), "aton_set_tile")

    def set_tile_rows(self, rows):
        _check(self.L.aton_set_tile_rows(self.h, int(rows)), "aton_set_tile_rows")

    def get_tile_rows(self):
        r = C.c_int()
        _check(self.L.aton_get_tile_rows(self.h, C.byref(r)), "aton_get_tile_rows")
        return r.value

    def autotune(self, steps=3):
        ty, tz, ms = C.c_int(), C.c_int(), C.c_float()
        _check(self.L.aton_autotune(self.h, int(steps), C.byref(ty), C.byref(tz), C.byref(ms)),
               "aton_autotune")
        return ty.value, tz.value, ms.value

    # -- state
    def set_fields(self, N, Fx, Fy, Fz, T, nH, x=None, y=None):
        arrs = (N, Fx, Fy, Fz, x, y, T, nH)
        for a in arrs:
            if a is not None and int(np.prod(a.shape)) != self.ncell:
                raise ValueError("field size does not match the grid")
        w = _where(arrs)
        _check(self.L.aton_set_fields(self.h, *(_ptr(a, w) for a in arrs), w), "aton_set_fields")

    def get_fields(self, out=None, device=False):
        """Returns dict(N, Fx, Fy, Fz, x, y, T): host float32 arrays, or the given ``out`` dict
        of preallocated arrays/tensors, or new torch CUDA tensors when device=True."""
        keys = ("N", "Fx", "Fy", "Fz", "x", "y", "T")
        if out is None:
            if device:
                import torch
                out = {k: torch.empty(self.shape, dtype=torch.float32, device="cuda") for k in keys}
            else:
                out = {k: np.empty(self.shape, np.float32) for k in keys}
        arrs = [out.get(k) for k in keys]
        w = _where(arrs)
        _check(self.L.aton_get_fields(self.h, *(_ptr(a, w) for a in arrs), w), "aton_get_fields")
        return out

    def add_sources(self, cell_idx, rate, mode=SRC_REPLACE):
        i = np.ascontiguousarray(cell_idx, dtype=np.int64)
        r = np.ascontiguousarray(rate, dtype=np.float64)
        if i.shape != r.shape:
            raise ValueError("cell_idx and rate differ in length")
        _check(self.L.aton_add_sources(self.h, i.ctypes.data, r.ctypes.data, i.size, int(mode)),
               "aton_add_sources")

    # -- stepping
    def step(self, nsteps=1):
        _check(self.L.aton_step(self.h, int(nsteps)), "aton_step")

    def synchronize(self):
        return self.L.aton_synchronize(self.h)

    def photon_budget(self):
        b = (C.c_double * BUDGET_LEN)()
        _check(self.L.aton_photon_budget(self.h, b), "aton_photon_budget")
        return dict(zip(BUDGET_KEYS, list(b)))

    def budget_request(self):
        _check(self.L.aton_budget_request(self.h), "aton_budget_request")

    def budget_collect(self):
        b = (C.c_double * BUDGET_LEN)()
        _check(self.L.aton_budget_collect(self.h, b), "aton_budget_collect")
        return dict(zip(BUDGET_KEYS, list(b)))

    def set_budget(self, budget):
        b = (C.c_double * BUDGET_LEN)(*[float(budget[k]) for k in BUDGET_KEYS])
        _check(self.L.aton_set_budget(self.h, b), "aton_set_budget")

    def diag(self):
        d = aton_diag()
        _check(self.L.aton_get_diag(self.h, C.byref(d)), "aton_get_diag")
        return {k: getattr(d, k) for k, _ in aton_diag._fields_}

    def ionisation_stats(self, **params):
        """aton_ionisation_stats with the defaults overridden by ``params`` (fields of
        aton_stats_params). Returns the summary fields plus the arrays hist_y (nb_nH, nb_y),
        hist_J (nb_nH, nb_J), bin_count, bin_mean_y, bin_mean_J21 (nb_nH) and the params."""
        p = stats_params(**params)
        s = aton_stats()
        hy = np.zeros((p.nb_nH, p.nb_y), np.uint64)
        hj = np.zeros((p.nb_nH, p.nb_J), np.uint64)
        bc = np.zeros(p.nb_nH, np.uint64)
        my = np.zeros(p.nb_nH, np.float64)
        mj = np.zeros(p.nb_nH, np.float64)
        _check(self.L.aton_ionisation_stats(self.h, C.byref(p), C.byref(s), hy.ctypes.data,
                                            hj.ctypes.data, bc.ctypes.data, my.ctypes.data,
                                            mj.ctypes.data), "aton_ionisation_stats")
        out = {k: getattr(s, k) for k, _ in aton_stats._fields_}
        out.update(hist_y=hy, hist_J=hj, bin_count=bc, bin_mean_y=my, bin_mean_J21=mj,
                   params={k: getattr(p, k) for k, _ in aton_stats_params._fields_})
        return out

    def last_error_cells(self):
        n = C.c_int64()
        _check(self.L.aton_last_error_cells(self.h, C.byref(n)), "aton_last_error_cells")
        return n.value

    def set_pair_sink(self, records, stride=1):
        """records: a float32 torch CUDA tensor of shape (capacity, 8), or None to stop."""
        if records is None:
            _check(self.L.aton_set_pair_sink(self.h, None, 0, 1), "aton_set_pair_sink")
            return
        _check(self.L.aton_set_pair_sink(self.h, records.data_ptr(), int(records.shape[0]),
                                         int(stride)), "aton_set_pair_sink")

    def pair_count(self):
        n = C.c_int64()
        _check(self.L.aton_pair_count(self.h, C.byref(n)), "aton_pair_count")
        return n.value

    def set_surrogate(self, mlp, gate_substeps=8.0, residual_max=1e-4, enabled=True):
        p = aton_surrogate_params(int(bool(enabled)), float(gate_substeps), float(residual_max))
        _check(self.L.aton_set_surrogate(self.h, None if mlp is None else mlp.h,
                                         None if mlp is None else C.byref(p)), "aton_set_surrogate")
        self._sur = mlp   # keep the network alive while the handle may use it

    def launches_per_step(self):
        n = C.c_int()
        _check(self.L.aton_launches_per_step(self.h, C.byref(n)), "aton_launches_per_step")
        return n.value


def photon_sum_static(N, cell_volume, stream=None):
    """sum(N) * cell_volume of a float32 torch CUDA tensor through aton_photon_sum_static: the
    variant that allocates no device memory (for callers that cannot let a library allocate;
    see include/aton.h for the size limit and the shared scratch)."""
    ptr = _ptr(N, DEVICE)
    out = C.c_double()
    s = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(load().aton_photon_sum_static(ptr, int(N.numel()), float(cell_volume), C.byref(out), s),
           "aton_photon_sum_static")
    return out.value


def stats_params(**params):
    """aton_stats_params: the library defaults with ``params`` overriding fields."""
    p = aton_stats_params()
    _check(load().aton_default_stats_params(C.byref(p)), "aton_default_stats_params")
    for k, v in params.items():
        if k not in dict(aton_stats_params._fields_):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def equilibrium_neutral_fraction(nH, J21_0, n_star=1.0, power=0, T=1e4, spectral_index=1.0):
    """aton_equilibrium_neutral_fraction over the densities nH (any float array)."""
    n = np.ascontiguousarray(nH, dtype=np.float64).ravel()
    y = np.empty_like(n)
    _check(load().aton_equilibrium_neutral_fraction(n.ctypes.data, int(n.size), float(J21_0),
                                                    float(n_star), int(power), float(T),
                                                    float(spectral_index), y.ctypes.data),
           "aton_equilibrium_neutral_fraction")
    return y.reshape(np.shape(nH))


def star_sources(stars, shape, dx, interval, f_esc=1.0, boost_a=0.0, boost_k=0.0,
                 t_universe=1.0):
    """aton_star_sources: (cell, rate) of each star (a STAR_DTYPE array) on a grid of shape
    (nz, ny, nx) and cell size dx; cell -1 marks stars that do not emit in the interval."""
    st = np.ascontiguousarray(stars, dtype=STAR_DTYPE)
    nz, ny, nx = shape
    m = aton_source_model(float(interval), float(f_esc), float(boost_a), float(boost_k),
                          float(t_universe))
    cell = np.empty(st.size, np.int64)
    rate = np.empty(st.size, np.float64)
    _check(load().aton_star_sources(st.ctypes.data, int(st.size), C.byref(m), int(nx), int(ny),
                                    int(nz), float(dx), cell.ctypes.data, rate.ctypes.data),
           "aton_star_sources")
    return cell, rate


class Mlp:
    """The chemistry-surrogate network (aton_mlp_*). Arrays are float32 torch CUDA tensors."""
    NORM_LEN = 26

    def __init__(self, seed=0):
        self.L = load()
        h = _VP()
        _check(self.L.aton_mlp_create(C.byref(h), int(seed)), "aton_mlp_create")
        self.h = h
        self.n_params = self.L.aton_mlp_num_params()

    def close(self):
        if getattr(self, "h", None):
            self.L.aton_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, np.float32)
        _check(self.L.aton_mlp_set_params(self.h, t.ctypes.data, HOST), "aton_mlp_set_params")

    def get_params(self):
        t = np.empty(self.n_params, np.float32)
        _check(self.L.aton_mlp_get_params(self.h, t.ctypes.data, HOST), "aton_mlp_get_params")
        return t

    def fit_norm(self, records, dt):
        _check(self.L.aton_mlp_fit_norm(self.h, records.data_ptr(), int(records.shape[0]),
                                        float(dt)), "aton_mlp_fit_norm")

    def get_norm(self):
        v = np.empty(self.NORM_LEN, np.float32)
        _check(self.L.aton_mlp_get_norm(self.h, v.ctypes.data), "aton_mlp_get_norm")
        return v

    def set_norm(self, v):
        v = np.ascontiguousarray(v, np.float32)
        _check(self.L.aton_mlp_set_norm(self.h, v.ctypes.data), "aton_mlp_set_norm")

    def features(self, records, dt, targets=True):
        import torch
        n = int(records.shape[0])
        X = torch.empty((n, 5), dtype=torch.float32, device=records.device)
        T = torch.empty((n, 3), dtype=torch.float32, device=records.device) if targets else None
        _check(self.L.aton_mlp_features(self.h, records.data_ptr(), n, float(dt), X.data_ptr(),
                                        None if T is None else T.data_ptr()), "aton_mlp_features")
        return X, T

    def forward(self, X):
        import torch
        n = int(X.shape[0])
        Y = torch.empty((n, 3), dtype=torch.float32, device=X.device)
        _check(self.L.aton_mlp_forward(self.h, X.data_ptr(), n, Y.data_ptr()), "aton_mlp_forward")
        return Y

    def loss_grad(self, X, T):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device)
        loss = C.c_double()
        _check(self.L.aton_mlp_loss_grad(self.h, X.data_ptr(), T.data_ptr(), int(X.shape[0]),
                                         g.data_ptr(), C.byref(loss)), "aton_mlp_loss_grad")
        return loss.value, g

    def train_step(self, X, T, lr, want_loss=False):
        loss = C.c_double()
        _check(self.L.aton_mlp_train_step(self.h, X.data_ptr(), T.data_ptr(), int(X.shape[0]),
                                          float(lr), C.byref(loss) if want_loss else None),
               "aton_mlp_train_step")
        return loss.value if want_loss else None

    def synchronize(self):
        _check(self.L.aton_mlp_synchronize(self.h), "aton_mlp_synchronize")


def from_workload(state, src_idx, src_rate, run, **params):
    """Create a handle for a workload tuple of ``workloads`` and load its state (host)."""
    a = Aton(run["nx"], run["ny"], run["nz"], run["dx"], run["c"], run["dt"])
    bc = BC_TRANSMISSIVE if run["bc"] == "transmissive" else BC_PERIODIC
    kw = dict(bc=bc, sigma_n=run["sigma_n"], sigma_e=run["sigma_e"], e_gamma_eV=run["e_gamma_eV"])
    kw.update(params)
    a.set_params(**kw)
    f32 = {k: np.ascontiguousarray(v, dtype=np.float32) for k, v in state.items()}
    y = np.ascontiguousarray(1.0 - np.asarray(state["x"], np.float64), dtype=np.float32)
    a.set_fields(f32["N"], f32["Fx"], f32["Fy"], f32["Fz"], f32["T"], f32["nH"], y=y)
    a.add_sources(src_idx, src_rate)
    return a
