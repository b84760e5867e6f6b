"""Seeded synthetic inputs for the ATON step.

This module only makes inputs: density fields, initial states, source lists and the run
parameters of each workload. It holds none of the method's arithmetic, and both the GPU path
and the CPU oracle consume the same arrays from it.

The paper post-processes RAMSES cosmological snapshots (section 2.1), which are not available.
A seeded lognormal density field with a power-law spectrum stands in for them, with point
sources on its highest density peaks (section 2.3 assigns sources to cells, nearest grid point).

Arrays are C-order (nz, ny, nx) with x fastest; units are cgs.
"""
import numpy as np

KPC = 3.0856775814913673e21   # cm
C_LIGHT = 2.99792458e10       # cm/s
MYR = 3.15576e13              # s

# single-group constants of the workloads: sigma = 1.63e-18 cm^2, mean photon energy 29.6 eV
SIGMA = 1.63e-18
E_GAMMA_EV = 29.6


def cfl_dt(dx, c=C_LIGHT, courant=0.9):
    """Radiative step at ``courant`` times the unsplit 3-D limit dx / (3 c)."""
    return courant * dx / (3.0 * c)


def gaussian_field(n, slope=-2.5, seed=1, shape=None):
    """Zero-mean, unit-variance Gaussian random field with P(k) ~ k^slope on a periodic grid."""
    nz, ny, nx = shape if shape is not None else (n, n, n)
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((nz, ny, nx), dtype=np.float64)
    wk = np.fft.rfftn(white)
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    k2 = kz * kz + ky * ky + kx * kx
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)          # sqrt(P(k)) with P ~ k^slope
    amp[0, 0, 0] = 0.0
    wk *= amp
    del k2, amp
    g = np.fft.irfftn(wk, s=(nz, ny, nx), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def lognormal_density(n, sigma_ln, mean_nH, slope=-2.5, seed=1, shape=None):
    """n_H = mean * exp(sigma g - sigma^2/2) for the Gaussian field g above (float64)."""
    g = gaussian_field(n, slope=slope, seed=seed, shape=shape)
    return mean_nH * np.exp(sigma_ln * g - 0.5 * sigma_ln * sigma_ln)


def density_peaks(nH, k):
    """Linear indices of the ``k`` highest 26-neighbour periodic local maxima of ``nH``.

    Ties go to the lower linear index. If there are fewer maxima than ``k`` the list is
    filled with the next-highest remaining cells.
    """
    from scipy.ndimage import maximum_filter
    mx = maximum_filter(nH, size=3, mode="wrap")
    flat = nH.ravel()
    cand = np.flatnonzero((nH >= mx).ravel())
    order = np.lexsort((cand, -flat[cand]))
    chosen = cand[order[:k]]
    if chosen.size < k:
        rest = np.setdiff1d(np.arange(flat.size), chosen, assume_unique=False)
        order2 = np.lexsort((rest, -flat[rest]))
        chosen = np.concatenate([chosen, rest[order2[: k - chosen.size]]])
    return chosen.astype(np.int64)


def loguniform_rates(k, lo, hi, seed):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=k))


def initial_state(nH, T0, x0):
    """Empty radiation field over gas of density nH, temperature T0, ionised fraction x0."""
    z = np.zeros_like(nH)
    return dict(N=z.copy(), Fx=z.copy(), Fy=z.copy(), Fz=z.copy(),
                x=np.full_like(nH, x0), T=np.full_like(nH, T0), nH=nH.copy())


def stromgren_box(n=32, L_kpc=6.6, nH=1e-3, T0=1e4, x0=1.2e-3, rate=5e48, c=C_LIGHT,
                  center=None):
    """Uniform hydrogen box with one central point source (the 32^3 Stromgren workload)."""
    dx = L_kpc * KPC / n
    shape = (n, n, n)
    st = initial_state(np.full(shape, nH), T0, x0)
    cz = cy = cx = n // 2 if center is None else center
    idx = np.array([cx + n * (cy + n * cz)], np.int64)
    run = dict(nx=n, ny=n, nz=n, dx=dx, c=c, dt=cfl_dt(dx, c), bc="transmissive",
               sigma_n=SIGMA, sigma_e=SIGMA, e_gamma_eV=E_GAMMA_EV)
    return st, idx, np.array([rate], np.float64), run


def cosmo_box(n, sigma_ln, nsrc, seed_field, seed_src, mean_nH=2e-4, T0=100.0, x0=1e-4,
              dx_kpc=4.0, lum=(1e50, 1e52), shape=None, c=C_LIGHT):
    """Lognormal density with sources at the highest peaks (the 128^3 / 512^3 / 1024^3 recipe)."""
    nH = lognormal_density(n, sigma_ln, mean_nH, seed=seed_field, shape=shape)
    nz, ny, nx = nH.shape
    st = initial_state(nH, T0, x0)
    idx = density_peaks(nH, nsrc)
    rate = loguniform_rates(nsrc, lum[0], lum[1], seed_src)
    dx = dx_kpc * KPC
    run = dict(nx=nx, ny=ny, nz=nz, dx=dx, c=c, dt=cfl_dt(dx, c), bc="periodic",
               sigma_n=SIGMA, sigma_e=SIGMA, e_gamma_eV=E_GAMMA_EV)
    return st, idx, rate, run


def cosmo_box_f32(n, sigma_ln, nsrc, seed_field, seed_src, mean_nH=2e-4, T0=100.0, x0=1e-4,
                  dx_kpc=4.0, lum=(1e50, 1e52), c=C_LIGHT):
    """The lognormal recipe of cosmo_box with the state built in float32 and the field's
    intermediates released early (for 1024^3, where float64 copies of seven fields would take
    60 GB of host memory). The Gaussian field is the same one cosmo_box draws."""
    import os
    from scipy import fft as sfft
    workers = os.cpu_count() or 1
    nz = ny = nx = n
    rng = np.random.default_rng(seed_field)
    wk = sfft.rfftn(rng.standard_normal((nz, ny, nx), dtype=np.float64), workers=workers)
    for k in range(nz):   # P(k) ~ k^-2.5 amplitude, one plane at a time
        kz = np.fft.fftfreq(nz)[k]
        k2 = kz * kz + np.fft.fftfreq(ny)[:, None] ** 2 + np.fft.rfftfreq(nx)[None, :] ** 2
        if k == 0:
            k2[0, 0] = 1.0
        amp = k2 ** (-2.5 / 4.0)
        if k == 0:
            amp[0, 0] = 0.0
        wk[k] *= amp
    g = sfft.irfftn(wk, s=(nz, ny, nx), axes=(0, 1, 2), workers=workers)
    del wk
    g -= g.mean()
    g /= g.std()
    nH = (mean_nH * np.exp(sigma_ln * g - 0.5 * sigma_ln * sigma_ln)).astype(np.float32)
    del g
    z = np.zeros_like(nH)
    st = dict(N=z, Fx=np.zeros_like(nH), Fy=np.zeros_like(nH), Fz=np.zeros_like(nH),
              x=np.full_like(nH, x0), T=np.full_like(nH, T0), nH=nH)
    idx = density_peaks(nH, nsrc)
    rate = loguniform_rates(nsrc, lum[0], lum[1], seed_src)
    dx = dx_kpc * KPC
    run = dict(nx=nx, ny=ny, nz=nz, dx=dx, c=c, dt=cfl_dt(dx, c), bc="periodic",
               sigma_n=SIGMA, sigma_e=SIGMA, e_gamma_eV=E_GAMMA_EV)
    return st, idx, rate, run


# The workloads, by grid size. Each returns (state, src_idx, src_rate, run_params).
def workload_32():
    return stromgren_box()


def workload_128(seed_field=1, seed_src=2):
    return cosmo_box(128, 1.5, 64, seed_field, seed_src)


def workload_512(seed_field=3, seed_src=4):
    return cosmo_box(512, 2.0, 4096, seed_field, seed_src)


def workload_1024(seed_field=5, seed_src=6):
    return cosmo_box_f32(1024, 2.0, 32768, seed_field, seed_src)


def workload_256(seed_field=10, seed_src=11):
    return cosmo_box(256, 2.0, 1024, seed_field, seed_src)


def stromgren_256(nH=1e-5, rate=1e52, T0=100.0, x0=1e-4):
    """The uniform single-source 256^3 box of the surrogate evaluation: cold, nearly neutral
    gas (the lognormal recipe's T0 and x0) at 4 kpc cells around one bright source (the top of
    the recipe's luminosity range), transmissive; the front heats gas from 100 K to ~6e4 K,
    which the exact operator sub-cycles heavily."""
    return stromgren_box(n=256, L_kpc=4.0 * 256, nH=nH, T0=T0, x0=x0, rate=rate)


def workload_small(shape=(20, 24, 36), nsrc=6, sigma_ln=1.5, seed_field=7, seed_src=8,
                   dx_kpc=4.0):
    """Small ragged-shape lognormal box for parity tests (spans several tiles plus a tail)."""
    return cosmo_box(None, sigma_ln, nsrc, seed_field, seed_src, shape=shape, dx_kpc=dx_kpc)


def subsample_state(state, src_idx, src_rate, shape, origin=(0, 0, 0)):
    """Crop a periodic sub-box (nz, ny, nx) at ``origin`` and keep the sources inside it."""
    nz, ny, nx = state["N"].shape
    oz, oy, ox = origin
    sz, sy, sx = shape
    sl = (slice(oz, oz + sz), slice(oy, oy + sy), slice(ox, ox + sx))
    st = {k: np.ascontiguousarray(v[sl]) for k, v in state.items()}
    k = src_idx // (nx * ny)
    j = (src_idx // nx) % ny
    i = src_idx % nx
    m = (k >= oz) & (k < oz + sz) & (j >= oy) & (j < oy + sy) & (i >= ox) & (i < ox + sx)
    loc = (i[m] - ox) + sx * ((j[m] - oy) + sy * (k[m] - oz))
    return st, loc.astype(np.int64), src_rate[m].copy()


# ------------------------------------------------------------------------------------------
# Snapshot sequences of star particles (section 2.3 post-processing; the cosmological runs'
# star lists are not available). Stars form at the highest density peaks at uniformly random
# times, more of them in every interval; each snapshot lists every star born before it with its
# age then. Lifetimes are drawn uniformly in [5, 20] Myr and yields uniformly in [24 000,
# 98 000] ionising photons per stellar baryon, the ranges section 2.3 quotes; the star mass is
# the 12.5 Mpc/h run's minimum star particle mass of its parameter table.
# ------------------------------------------------------------------------------------------
MSUN = 1.98892e33             # g
STAR_FIELDS = [("x", "<f8"), ("y", "<f8"), ("z", "<f8"), ("mass", "<f8"), ("age", "<f8"),
               ("lifetime", "<f8"), ("photons_per_baryon", "<f8")]


def star_snapshots(nH, dx, n_snap, interval, seed, n_sites=16, first=4, growth=1.6,
                   m_star=5.81e4 * MSUN):
    """Star lists of snapshots 0..n_snap at times p * interval: a list of structured arrays
    (fields STAR_FIELDS, cgs). Interval k (between snapshots k and k+1) forms
    round(first * growth**k) stars at sites drawn among the n_sites highest peaks of nH."""
    rng = np.random.default_rng(seed)
    sites = density_peaks(nH, n_sites)
    nz, ny, nx = nH.shape
    born = []   # (birth time, x, y, z, lifetime, yield)
    snaps = []
    for p in range(n_snap + 1):
        t_p = p * interval
        rows = [(b[1], b[2], b[3], m_star, t_p - b[0], b[4], b[5]) for b in born]
        snaps.append(np.array(rows, dtype=STAR_FIELDS))
        if p == n_snap:
            break
        for _ in range(int(round(first * growth ** p))):
            c = int(sites[rng.integers(len(sites))])
            i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
            off = rng.random(3)
            born.append((t_p + rng.random() * interval, (i + off[0]) * dx, (j + off[1]) * dx,
                         (k + off[2]) * dx, rng.uniform(5.0, 20.0) * MYR,
                         rng.uniform(24000.0, 98000.0)))
    return snaps


def snapshot_workload(shape=(16, 20, 24), n_snap=3, steps_per_interval=40, seed_field=21,
                      seed_stars=22, sigma_ln=1.5, dx_kpc=4.0):
    """A small post-processing run: lognormal gas, a star-list sequence, the run parameters,
    and the source-model parameters (escape fraction and boost of the 12.5 Mpc/h run, boost
    evaluated at t = 500 Myr). The snapshot interval is steps_per_interval radiative steps."""
    st, _, _, run = cosmo_box(None, sigma_ln, 1, seed_field, seed_field + 1, shape=shape,
                              dx_kpc=dx_kpc)
    interval = steps_per_interval * run["dt"]
    snaps = star_snapshots(st["nH"], run["dx"], n_snap, interval, seed_stars)
    model = dict(f_esc=0.055, boost_a=0.7, boost_k=300.0 * MYR, t0=500.0 * MYR)
    return st, snaps, run, interval, model
