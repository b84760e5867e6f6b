"""Pins of the oracle's transport: the Lax-Friedrichs update of Appendix Eqs. A2/A5 with the
M1 closure of section 2.2."""
import numpy as np
import pytest
from scipy.special import comb

import oracle as O

C = 2.99792458e10


def _fields(shape, fill=0.0):
    return [np.full(shape, fill, dtype=np.float64) for _ in range(4)]


def test_uniform_state_is_invariant():
    shape = (5, 6, 7)
    p = O.params(dx=1e20, dt=0.3e20 / C, bc=O.BC_PERIODIC)
    N = np.full(shape, 2.5e-3)
    F = 0.6 * C * 2.5e-3 * np.array([0.48, -0.6, 0.64])
    Fx, Fy, Fz = (np.full(shape, v) for v in F)
    No, Fxo, Fyo, Fzo, esc = O.transport(p, N, Fx, Fy, Fz)
    assert np.allclose(No, N, rtol=1e-14, atol=0)
    assert np.allclose(Fxo, Fx, rtol=1e-13, atol=0)
    assert np.allclose(Fyo, Fy, rtol=1e-13, atol=0)
    assert np.allclose(Fzo, Fz, rtol=1e-13, atol=0)
    assert esc == 0.0


@pytest.mark.parametrize("lam", [0.3, 0.9])
def test_free_streaming_beam_is_exact_upwind(lam):
    """With F = cN along +x everywhere (f = 1), the global LF flux reduces to the upwind flux
    of N + F/c moving at c, so after s steps N_i = sum_k C(s,k) lam^k (1-lam)^(s-k) N_{i-k}."""
    nx, ny, nz = 64, 3, 2
    dx = 1e20
    p = O.params(dx=dx, dt=lam * dx / C, bc=O.BC_PERIODIC)
    prof = np.zeros(nx)
    prof[5:12] = np.linspace(1.0, 3.0, 7)
    prof[20] = 0.5
    N = np.broadcast_to(prof, (nz, ny, nx)).copy()
    Fx = C * N
    Fy = np.zeros_like(N)
    Fz = np.zeros_like(N)
    s = 17
    for _ in range(s):
        N, Fx, Fy, Fz, _e = O.transport(p, N, Fx, Fy, Fz)
    k = np.arange(s + 1)
    w = comb(s, k) * lam ** k * (1 - lam) ** (s - k)
    expect = np.zeros(nx)
    for kk, ww in zip(k, w):
        expect += ww * np.roll(prof, kk)
    assert np.allclose(N[1, 2], expect, rtol=1e-12, atol=1e-15)
    assert np.allclose(Fx / C, N, rtol=1e-12, atol=1e-14)
    assert np.abs(Fy).max() == 0.0 and np.abs(Fz).max() == 0.0


def test_mirror_and_axis_permutation_symmetry():
    """A central pulse in a cube evolves with the cube's symmetries (mirror and axis swaps)."""
    n = 11
    p = O.params(dx=1e20, dt=0.9e20 / (3 * C), bc=O.BC_TRANSMISSIVE)
    N, Fx, Fy, Fz = _fields((n, n, n))
    N[5, 5, 5] = 1.0
    N[5, 5, 6] = N[5, 5, 4] = N[5, 6, 5] = N[5, 4, 5] = N[6, 5, 5] = N[4, 5, 5] = 0.3
    for _ in range(12):
        N, Fx, Fy, Fz, _e = O.transport(p, N, Fx, Fy, Fz)
    scale = N.max()
    for ax in range(3):
        assert np.allclose(N, np.flip(N, axis=ax), atol=1e-13 * scale, rtol=0)
    assert np.allclose(N, N.transpose(0, 2, 1), atol=1e-13 * scale, rtol=0)
    assert np.allclose(N, N.transpose(2, 1, 0), atol=1e-13 * scale, rtol=0)
    assert np.allclose(Fx, -np.flip(Fx, axis=2), atol=1e-13 * scale * C, rtol=0)
    assert np.allclose(Fx, Fy.transpose(0, 2, 1), atol=1e-13 * scale * C, rtol=0)


def _random_realisable(shape, seed):
    rng = np.random.default_rng(seed)
    N = rng.uniform(0.1, 1.0, shape)
    d = rng.standard_normal((3,) + shape)
    d /= np.linalg.norm(d, axis=0)
    f = rng.uniform(0.0, 1.0, shape)
    F = C * N * f * d
    return N, F[0], F[1], F[2]


def test_positive_and_conservative_at_the_unsplit_limit():
    """At 3 c dt / dx = 1 a realisable state stays non-negative and sum(N) is conserved
    (periodic box, no sources, no absorption)."""
    shape = (8, 9, 10)
    p = O.params(dx=1.0, dt=1.0 / (3 * C), bc=O.BC_PERIODIC)
    N, Fx, Fy, Fz = _random_realisable(shape, 4)
    tot0 = N.sum()
    for _ in range(30):
        N, Fx, Fy, Fz, _e = O.transport(p, N, Fx, Fy, Fz)
        assert N.min() >= -1e-14
    assert N.sum() == pytest.approx(tot0, rel=1e-13)


def test_unstable_well_above_the_limit():
    """With 3 c dt / dx = 3 (dt = dx/c, the paper's Eq. 7 bound itself) a checkerboard
    perturbation grows without bound."""
    shape = (8, 8, 8)
    p = O.params(dx=1.0, dt=1.0 / C, bc=O.BC_PERIODIC)
    k, j, i = np.indices(shape)
    N = 1.0 + 1e-3 * (-1.0) ** (i + j + k)
    Fx, Fy, Fz = (np.zeros(shape) for _ in range(3))
    for _ in range(40):
        N, Fx, Fy, Fz, _e = O.transport(p, N, Fx, Fy, Fz)
    assert np.abs(N - N.mean()).max() > 1.0


def test_transmissive_escape_tally_is_the_boundary_flux():
    """Transport only: every photon that leaves the box is tallied as escaped."""
    shape = (6, 7, 8)
    p = O.params(dx=1.0, dt=0.9 / (3 * C), bc=O.BC_TRANSMISSIVE)
    N, Fx, Fy, Fz = _random_realisable(shape, 9)
    tot0 = N.sum()
    esc = 0.0
    for _ in range(10):
        N, Fx, Fy, Fz, e = O.transport(p, N, Fx, Fy, Fz)
        esc += e
    assert tot0 - N.sum() == pytest.approx(esc, rel=1e-12)
    assert esc > 0


def test_shadow_behind_an_absorber():
    """Section 2.2: the M1 scheme casts shadows behind absorbers. A plane-parallel beam from
    the -x side meets an opaque neutral clump; cells behind it stay far darker than cells at
    the same x beside it."""
    nx, ny, nz = 40, 21, 3
    dx = 3.0e20
    p = O.params(dx=dx, dt=0.9 * dx / (3 * C), bc=O.BC_TRANSMISSIVE, sigma_n=1.63e-18,
                 sigma_e=1.63e-18, e_gamma_eV=29.6, fixed_T=1, coll_ion=0)
    shape = (nz, ny, nx)
    nH = np.full(shape, 1e-8)
    nH[:, 8:13, 10:16] = 10.0   # optically thick clump
    st = dict(N=np.zeros(shape), Fx=np.zeros(shape), Fy=np.zeros(shape), Fz=np.zeros(shape),
              x=np.full(shape, 1.0 - 1e-8), T=np.full(shape, 1e4), nH=nH)
    st["x"][nH > 1] = 1e-4
    # a wall of sources in the first column
    k, j = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
    idx = (0 + nx * (j + ny * k)).ravel()
    rate = np.full(idx.size, 1e50)
    out, _b, _s = O.run(p, st, 250, idx, rate, omp=True)
    # right behind the clump (first-order LF diffusion refills the shadow further away)
    behind = out["N"][1, 10, 16]
    beside = out["N"][1, 2, 16]
    assert beside > 0
    assert behind < 0.1 * beside
    # and the shadow is still visible a clump-length further on
    assert out["N"][1, 10, 19] < 0.5 * out["N"][1, 2, 19]
