"""Pins of the oracle's M1 closure (section 2.2, Eqs. 5-6 and the chi paragraph)."""
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        if line.strip() and not line.startswith("#"):
            parts = line.split()
            out[parts[0]] = float(parts[1])
    return out


def test_chi_limits_match_paper():
    g = _golden("paper_constants.txt")
    assert O.chi(0.0) == pytest.approx(g["chi_diffusion"], abs=1e-15)
    assert O.chi(1.0) == pytest.approx(g["chi_transport"], abs=1e-15)


def test_chi_monotone_and_bounded():
    f = np.linspace(0.0, 1.0, 1001)
    c = np.array([O.chi(v) for v in f])
    assert np.all(np.diff(c) > 0)
    assert c.min() >= 1.0 / 3.0 - 1e-15 and c.max() <= 1.0 + 1e-15
    # reduced flux above 1 is clamped (|f| <= 1 kept)
    assert O.chi(1.7) == O.chi(1.0)
    assert O.chi(-0.3) == O.chi(0.0)


def _random_dirs(n, seed=0):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("f", [0.0, 0.1, 0.37, 0.5, 0.8, 0.99, 1.0])
def test_eddington_tensor_invariants(f):
    c = 2.99792458e10
    N = 3.7e-4
    for nvec in _random_dirs(8, seed=int(f * 100)):
        F = f * c * N * nvec
        D = O.eddington(N, F, c)
        chi = O.chi(f)
        assert np.allclose(D, D.T, atol=1e-15)
        assert np.trace(D) == pytest.approx(1.0, abs=1e-14)
        w, V = np.linalg.eigh(D)
        if f > 0:
            # eigenvalue chi along the flux, (1 - chi)/2 twice across it
            assert np.allclose(D @ nvec, chi * nvec, atol=1e-14)
            assert np.allclose(sorted(w), sorted([chi, (1 - chi) / 2, (1 - chi) / 2]), atol=1e-13)
        else:
            assert np.allclose(D, np.eye(3) / 3.0, atol=1e-15)


def test_free_streaming_tensor_is_projector():
    c = 1.0
    for nvec in _random_dirs(5, seed=3):
        D = O.eddington(2.0, 2.0 * nvec, c)
        assert np.allclose(D, np.outer(nvec, nvec), atol=1e-14)


def test_printed_coefficient_order_fails_diffusion_limit():
    """Documents the reading of Eq. 6: the coefficients as printed give tr D = 4chi - 1 and
    D = n(x)n/3 at chi = 1/3, contradicting the diffusion limit stated beside it; the swapped
    order used by the oracle gives D = I/3 there."""
    chi = 1.0 / 3.0
    n = np.array([1.0, 0, 0])
    printed = (3 * chi - 1) / 2 * np.eye(3) + (1 - chi) / 2 * np.outer(n, n)
    assert not np.allclose(printed, np.eye(3) / 3)
    assert np.allclose(O.eddington(1.0, [0, 0, 0], 1.0), np.eye(3) / 3)
