"""FP64 reference of the ionisation and radiation statistics -- TEST INFRASTRUCTURE ONLY.

Section 4 reports the volume-weighted ionised fraction x_v and the distribution of the neutral
fraction, the mean intensity J21 (or the photo-ionisation rate Gamma12) with its distribution,
and the density dependence (1-x)(nH), J21(nH) with the mean per density bin, set against
photo-ionisation equilibrium for a uniform field J0 and for the self-shielded fields
J1 = J0 exp(-nH/n1*) and J4 = J0 exp(-(nH/n4*)^4) (the exponent read as in the figure caption).

Readings (the paper defines none of the conversions):
- Gamma = c sigma_n N (the single-group rate, no sub-grid clumping), Gamma12 = Gamma / 1e-12 s^-1;
- J21 is the Lyman-limit mean intensity (1e-21 erg s^-1 cm^-2 Hz^-1 sr^-1) of a spectrum
  J_nu = J_0 (nu/nu_0)^-alpha with the same rate when sigma = sigma_0 (nu/nu_0)^-3:
  Gamma = int 4 pi J_nu sigma_nu / (h nu) dnu = 4 pi J_0 sigma_0 / (h (alpha + 3)),
  sigma_0 = 6.30e-18 cm^2;
- histogram bins are log-spaced float edges: edge k = float(10^(log10 lo + k (log10 hi -
  log10 lo) / nb)); a value v is in bin b when edge[b] <= v < edge[b+1], below edge[1] in bin 0,
  at or above edge[nb-1] in bin nb-1; J21 bins compare N with float(edge_J21 / kJ), kJ = J21 per
  unit N. The comparisons are made on the stored float32 values, as the kernels make them;
- equilibrium: (1-x) Gamma = alpha_B(T) nH x^2 (Eq. 14 at steady state, no collisions), solved
  without cancellation as x = 2G/(G + sqrt(G^2 + 4 a G)), y = a x^2 / G, a = alpha_B nH.

Sums are plain FP64 sums of the float32 state converted to FP64.
"""
import numpy as np

from . import alpha_B

H_PLANCK = 6.62607015e-27   # erg s
SIGMA_0 = 6.30e-18          # cm^2, HI photo-ionisation cross-section at 13.6 eV


def gamma_per_J21(alpha):
    """Photo-ionisation rate [s^-1] of J21 = 1 under the power-law reading."""
    return 4.0 * np.pi * SIGMA_0 * 1e-21 / (H_PLANCK * (alpha + 3.0))


def j21_per_N(c, sigma_n, alpha):
    """J21 of one photon per cm^3: Gamma = c sigma_n N, J21 = Gamma / gamma_per_J21."""
    return c * sigma_n / gamma_per_J21(alpha)


def edges(lo, hi, nb, div=1.0):
    """float32 log-spaced bin edges (nb + 1 of them), divided by div before rounding."""
    a, b = np.log10(lo), np.log10(hi)
    k = np.arange(nb + 1, dtype=np.float64)
    return (10.0 ** (a + (b - a) * k / nb) / div).astype(np.float32)


def bins(v, E):
    """Bin index of each float32 value of v against the float32 edges E (len nb + 1)."""
    nb = len(E) - 1
    b = np.searchsorted(E, np.asarray(v, np.float32), side="right") - 1
    return np.clip(b, 0, nb - 1)


DEFAULTS = dict(nb_nH=48, nb_y=48, nb_J=48, nH_lo=1e-6, nH_hi=1.0, y_lo=1e-7, y_hi=1.0,
                J21_lo=1e-6, J21_hi=1e4, spectral_index=1.0, nH_plateau=1e-3)


def stats(N, y, T, nH, c, sigma_n, cell_volume, **params):
    """Statistics of a state (float32 arrays of any shape, the layout the GPU stores)."""
    p = dict(DEFAULTS)
    p.update(params)
    N = np.asarray(N, np.float32).ravel()
    y = np.asarray(y, np.float32).ravel()
    T = np.asarray(T, np.float32).ravel()
    n = np.asarray(nH, np.float32).ravel()
    kJ = j21_per_N(c, sigma_n, p["spectral_index"])
    En = edges(p["nH_lo"], p["nH_hi"], p["nb_nH"])
    Ey = edges(p["y_lo"], p["y_hi"], p["nb_y"])
    EJ = edges(p["J21_lo"], p["J21_hi"], p["nb_J"], div=kJ)
    bn, by, bJ = bins(n, En), bins(y, Ey), bins(N, EJ)
    hist_y = np.zeros((p["nb_nH"], p["nb_y"]), np.uint64)
    np.add.at(hist_y, (bn, by), 1)
    hist_J = np.zeros((p["nb_nH"], p["nb_J"]), np.uint64)
    np.add.at(hist_J, (bn, bJ), 1)
    count = np.bincount(bn, minlength=p["nb_nH"]).astype(np.uint64)
    N64, y64, T64, n64 = (a.astype(np.float64) for a in (N, y, T, n))
    sy_b = np.bincount(bn, weights=y64, minlength=p["nb_nH"])
    sN_b = np.bincount(bn, weights=N64, minlength=p["nb_nH"])
    cnt = count.astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean_y = np.where(count > 0, sy_b / cnt, 0.0)
        mean_J = np.where(count > 0, kJ * sN_b / cnt, 0.0)
    ncell = N.size
    plateau = n < np.float32(p["nH_plateau"])
    npl = int(plateau.sum())
    return dict(
        x_volume=1.0 - y64.sum() / ncell,
        x_mass=1.0 - (n64 * y64).sum() / n64.sum(),
        gamma12_volume=c * sigma_n * N64.sum() / ncell / 1e-12,
        J21_volume=kJ * N64.sum() / ncell,
        J21_plateau=kJ * N64[plateau].sum() / npl if npl else 0.0,
        T_volume=T64.sum() / ncell,
        T_mass=(n64 * T64).sum() / n64.sum(),
        photons=N64.sum() * cell_volume,
        cells=ncell, plateau_cells=npl,
        hist_y=hist_y, hist_J=hist_J, bin_count=count, bin_mean_y=mean_y, bin_mean_J21=mean_J)


def equilibrium_y(nH, J21_0, n_star=1.0, power=0, T=1e4, spectral_index=1.0):
    """Neutral fraction in photo-ionisation equilibrium under Gamma(nH) = Gamma_0
    exp(-(nH/n_star)^power) (power 0: uniform J0; 1: J1; 4: J4)."""
    nH = np.asarray(nH, np.float64)
    G0 = J21_0 * gamma_per_J21(spectral_index)
    G = G0 * (np.ones_like(nH) if power == 0 else np.exp(-(nH / n_star) ** power))
    a = alpha_B(T) * nH
    with np.errstate(invalid="ignore", divide="ignore"):
        x = 2.0 * G / (G + np.sqrt(G * G + 4.0 * a * G))
        y = np.where(G > 0, a * x * x / G, 1.0)
    return y
