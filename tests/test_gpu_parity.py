"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on seeded inputs.

Gates (after 100 steps): |x_gpu - x_oracle| <= 1e-3; |T_gpu/T_oracle - 1| <= 1e-3;
|N_gpu/N_oracle - 1| <= 1e-3 on cells with N > 1e-6 max N. The photon budget closes to 1e-6.
"""
import itertools

import numpy as np
import pytest

from paper_1004_2503_b300 import aton as A
from paper_1004_2503_b300 import workloads as W

from parity_helpers import (assert_gates, budget_closure, errors, run_gpu, run_oracle)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    # 36 x 24 x 20: two 32-wide tiles in x (ragged tail of 4), three 8-row tiles in y, one slab
    return W.workload_small()


@pytest.fixture(scope="module")
def small_oracle(small):
    st, idx, rate, run = small
    return run_oracle(st, idx, rate, run, 100)


@pytest.mark.parametrize("mode", [A.MODE_FUSED, A.MODE_UNFUSED])
def test_lognormal_periodic_100_steps(small, small_oracle, mode):
    st, idx, rate, run = small
    f, b, d, rc = run_gpu(st, idx, rate, run, 100, mode=mode)
    assert rc == 0
    e = errors(f, small_oracle[0])
    print("errors", mode, e)
    assert_gates(e, f"mode {mode}")
    assert abs(budget_closure(b)) <= 1e-6
    assert d["error_cells"] == 0 and d["nonfinite_cells"] == 0
    assert d["substeps_total"] >= 100 * st["N"].size
    # the oracle's tallies agree with the GPU's
    ob = small_oracle[1]
    assert b["emitted"] == pytest.approx(ob["emitted"], rel=1e-6)
    assert b["absorbed"] == pytest.approx(ob["absorbed"], rel=1e-3)


@pytest.mark.parametrize("fixed_T", [0, 1])
def test_stromgren_32_transmissive(fixed_T):
    """Transmissive 32^3 box with one source, through the fused step and the plain three-kernel
    step (whose transport pass is the TMA-staged kernel's transport-only instance here)."""
    st, idx, rate, run = W.workload_32()
    kw = dict(fixed_T=fixed_T, coll_ion=0 if fixed_T else 1)
    orc, ob, _ = run_oracle(st, idx, rate, run, 100, **kw)
    for mode in (A.MODE_FUSED, A.MODE_UNFUSED):
        f, b, d, rc = run_gpu(st, idx, rate, run, 100, mode=mode, **kw)
        assert rc == 0
        e = errors(f, orc)
        print("errors", kw, mode, e)
        assert_gates(e, mode)
        assert abs(budget_closure(b)) <= 1e-6
        assert b["escaped"] == pytest.approx(ob["escaped"], rel=1e-3, abs=1e-6 * ob["emitted"])


@pytest.mark.parametrize("shape,tile", [((40, 1, 1), (4, 7)), ((2, 3, 5), (8, 1)),
                                        ((9, 17, 33), (4, 4)), ((3, 40, 70), (16, 2)),
                                        ((9, 17, 36), (4, 4)), ((3, 40, 68), (16, 2)),
                                        ((7, 5, 4), (8, 3))])
def test_ragged_and_degenerate_shapes(shape, tile):
    st, idx, rate, run = W.workload_small(shape=shape, nsrc=2, seed_field=11, seed_src=12)
    orc, _, _ = run_oracle(st, idx, rate, run, 30)
    for mode in (A.MODE_FUSED, A.MODE_UNFUSED):
        f, b, d, rc = run_gpu(st, idx, rate, run, 30, mode=mode, tile=tile)
        assert rc == 0
        assert_gates(errors(f, orc), (shape, tile, mode))
        assert abs(budget_closure(b)) <= 1e-6


@pytest.mark.parametrize("shape,tile", [((20, 24, 36), (8, 64)), ((9, 13, 44), (4, 3)),
                                        ((5, 7, 8), (16, 2)), ((12, 40, 96), (8, 5))])
def test_tma_staged_and_plain_load_fused_kernels_agree(shape, tile):
    """The TMA-staged fused kernel (nx a multiple of 4) and the plain-load fused kernel do the
    same arithmetic; separately compiled, they agree to 1e-5 (contraction may differ)."""
    st, idx, rate, run = W.workload_small(shape=shape, nsrc=3, seed_field=31, seed_src=32)
    for bc in ("periodic", "transmissive"):
        r = dict(run, bc=bc)
        f1, b1, d1, rc1 = run_gpu(st, idx, rate, r, 20, mode=A.MODE_FUSED, tile=tile)
        f2, b2, d2, rc2 = run_gpu(st, idx, rate, r, 20, mode=A.MODE_FUSED_LDG, tile=tile)
        assert rc1 == 0 and rc2 == 0
        for k in ("N", "Fx", "Fy", "Fz", "y", "T"):
            scale = np.abs(f2[k]).max()
            assert np.abs(f1[k] - f2[k]).max() <= 1e-5 * scale, (bc, k)
        assert b1["absorbed"] == pytest.approx(b2["absorbed"], rel=1e-5)
        assert b1["escaped"] == pytest.approx(b2["escaped"], rel=1e-5, abs=1e-9 * b2["emitted"])
        assert d1["substeps_total"] == pytest.approx(d2["substeps_total"], rel=1e-4)


def test_fused_equals_unfused_closely(small):
    st, idx, rate, run = small
    f1, b1, _, _ = run_gpu(st, idx, rate, run, 40, mode=A.MODE_FUSED)
    f2, b2, _, _ = run_gpu(st, idx, rate, run, 40, mode=A.MODE_UNFUSED)
    for k in ("N", "Fx", "Fy", "Fz", "y", "T"):
        scale = np.abs(f2[k]).max()
        assert np.abs(f1[k] - f2[k]).max() <= 1e-5 * scale, k


def test_tiles_and_graphs_give_identical_fields(small):
    """Per-cell arithmetic does not depend on the slab depth or on graph batching: bitwise
    equal for one tile height. Different tile heights are separate compiled kernels whose
    floating-point contraction may differ by an ulp: equal to 1e-5."""
    st, idx, rate, run = small
    refs = {}
    for ty in (4, 8, 16):
        refs[ty] = run_gpu(st, idx, rate, run, 25, graph_batch=0, tile=(ty, 64))
    for tile in [(4, 1), (8, 5), (16, 3), (8, 64)]:
        for gb in (0, 7, 100):
            f, b, _, _ = run_gpu(st, idx, rate, run, 25, graph_batch=gb, tile=tile)
            ref, bref, _, _ = refs[tile[0]]
            for k in ("N", "Fx", "Fy", "Fz", "y", "T"):
                assert np.array_equal(f[k], ref[k]), (tile, gb, k)
            # per-thread FP32 tally partitions differ with the slab depth
            assert b["absorbed"] == pytest.approx(bref["absorbed"], rel=1e-7)
    for ty in (4, 16):
        for k in ("N", "Fx", "Fy", "Fz", "y", "T"):
            a, r = refs[ty][0][k], refs[8][0][k]
            assert np.abs(a - r).max() <= 1e-5 * np.abs(r).max(), (ty, k)


@pytest.mark.parametrize("shape,tile", [((20, 24, 36), (8, 64)), ((24, 16, 64), (8, 7)),
                                        ((19, 22, 68), (8, 5)), ((40, 48, 32), (16, 16)),
                                        ((11, 9, 12), (16, 4))])
def test_two_rows_per_thread_match_one_row_and_the_oracle(shape, tile):
    """Two rows of the tile per thread (half the warps per CTA) do the same per-cell arithmetic
    as one row per thread, in a separately compiled kernel: within 1e-5 of it and within the
    oracle's gates, on full tiles, x- and y-ragged tiles and both boundaries, with the one-launch
    fused step running. Shapes are (nz, ny, nx) with nx a multiple of 4 (the TMA-staged kernel)."""
    st, idx, rate, run = W.workload_small(shape=shape, nsrc=5, seed_field=41, seed_src=42)
    for bc in ("periodic", "transmissive"):
        r = dict(run, bc=bc)
        orc, _, _ = run_oracle(st, idx, rate, r, 30)
        f1, b1, d1, rc1 = run_gpu(st, idx, rate, r, 30, tile=tile, rows=1)
        f2, b2, d2, rc2 = run_gpu(st, idx, rate, r, 30, tile=tile, rows=2)
        assert rc1 == 0 and rc2 == 0
        assert_gates(errors(f2, orc), (shape, tile, bc))
        assert abs(budget_closure(b2)) <= 1e-6
        for k in ("N", "Fx", "Fy", "Fz", "y", "T"):
            scale = np.abs(f1[k]).max()
            assert np.abs(f1[k] - f2[k]).max() <= 1e-5 * scale, (bc, k)
        assert b2["absorbed"] == pytest.approx(b1["absorbed"], rel=1e-5)
        assert b2["escaped"] == pytest.approx(b1["escaped"], rel=1e-5, abs=1e-9 * b1["emitted"])
        assert d2["substeps_total"] == pytest.approx(d1["substeps_total"], rel=1e-4)


def test_deterministic(small):
    st, idx, rate, run = small
    f1, b1, d1, _ = run_gpu(st, idx, rate, run, 20)
    f2, b2, d2, _ = run_gpu(st, idx, rate, run, 20)
    for k in f1:
        assert np.array_equal(f1[k], f2[k])
    assert b1 == b2 and d1 == d2


def test_checkpoint_restart_is_bitwise(small):
    st, idx, rate, run = small
    full, bfull, _, _ = run_gpu(st, idx, rate, run, 20)
    a = A.from_workload(st, idx, rate, run)
    a.step(10)
    mid = a.get_fields()
    bmid = a.photon_budget()
    a.close()
    b = A.Aton(run["nx"], run["ny"], run["nz"], run["dx"], run["c"], run["dt"])
    b.set_params(bc=A.BC_PERIODIC, sigma_n=run["sigma_n"], sigma_e=run["sigma_e"],
                 e_gamma_eV=run["e_gamma_eV"])
    b.set_fields(mid["N"], mid["Fx"], mid["Fy"], mid["Fz"], mid["T"],
                 np.ascontiguousarray(st["nH"], np.float32), y=mid["y"])
    b.set_budget(bmid)
    b.add_sources(idx, rate)
    b.step(10)
    end = b.get_fields()
    bend = b.photon_budget()
    b.close()
    for k in ("N", "Fx", "Fy", "Fz", "y", "T"):
        assert np.array_equal(end[k], full[k]), k
    assert bend["emitted"] == pytest.approx(bfull["emitted"], rel=1e-12)
    assert bend["absorbed"] == pytest.approx(bfull["absorbed"], rel=1e-6)


def test_device_pointers_and_stream():
    torch = pytest.importorskip("torch")
    st, idx, rate, run = W.workload_small(shape=(8, 16, 32), nsrc=3)
    host, _, _, _ = run_gpu(st, idx, rate, run, 10)
    a = A.Aton(run["nx"], run["ny"], run["nz"], run["dx"], run["c"], run["dt"])
    a.set_params(bc=A.BC_PERIODIC, sigma_n=run["sigma_n"], sigma_e=run["sigma_e"],
                 e_gamma_eV=run["e_gamma_eV"])
    s = torch.cuda.Stream()
    a.set_stream(s)
    dev = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda() for k, v in st.items()}
    yd = (1 - torch.from_numpy(np.asarray(st["x"], np.float64))).float().cuda()
    torch.cuda.synchronize()
    a.set_fields(dev["N"], dev["Fx"], dev["Fy"], dev["Fz"], dev["T"], dev["nH"], y=yd)
    a.add_sources(idx, rate)
    a.step(10)
    out = a.get_fields(device=True)
    a.set_stream(None)
    a.close()
    for k in ("N", "y", "T"):
        assert np.array_equal(out[k].cpu().numpy(), host[k]), k


def test_error_paths():
    st, idx, rate, run = W.workload_32()
    a = A.Aton(run["nx"], run["ny"], run["nz"], run["dx"], run["c"], run["dt"])
    with pytest.raises(A.AtonError) as e:
        a.step(1)
    assert e.value.code == A.ERR_STATE
    with pytest.raises(A.AtonError) as e:
        a.add_sources([32 ** 3], [1.0])
    assert e.value.code == A.ERR_BADARG
    with pytest.raises(A.AtonError) as e:
        a.add_sources([0], [-1.0])
    assert e.value.code == A.ERR_BADARG
    bad = np.ascontiguousarray(st["N"], np.float32)
    bad[3, 4, 5] = np.nan
    f32 = {k: np.ascontiguousarray(v, np.float32) for k, v in st.items()}
    with pytest.raises(A.AtonError) as e:
        a.set_fields(bad, f32["Fx"], f32["Fy"], f32["Fz"], f32["T"], f32["nH"], x=f32["x"])
    assert e.value.code == A.ERR_NONFINITE
    with pytest.raises(A.AtonError) as e:
        a.set_params(sub_eps=0.0)
    assert e.value.code == A.ERR_BADARG
    for rows in (0, 3):
        with pytest.raises(A.AtonError) as e:
            a.set_tile_rows(rows)
        assert e.value.code == A.ERR_BADARG
    assert a.get_tile_rows() == 2          # the default: two rows per thread
    a.set_tile_rows(1)
    assert a.get_tile_rows() == 1
    a.close()


def test_allocation_failure_in_init_releases_everything(monkeypatch):
    """Host-side failure injection: each of aton_init's device allocations is made to fail in
    turn (ATON_TEST_FAIL_ALLOC). Every attempt returns NOMEM, and no device memory is left
    behind: the 256^3 grid's field buffers are 64 MiB each, far above the tolerance. A handle
    made afterwards steps normally."""
    import torch
    torch.cuda.init()
    st, idx, rate, run = W.workload_32()
    n = 256
    A.Aton(32, 32, 32, run["dx"], run["c"], run["dt"]).close()   # (kernels loaded on the device)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(64):
        monkeypatch.setenv("ATON_TEST_FAIL_ALLOC", str(k))
        try:
            a = A.Aton(n, n, n, run["dx"], run["c"], run["dt"])
        except A.AtonError as e:
            assert e.code == A.ERR_NOMEM, (k, str(e))
            failures += 1
            continue
        a.close()          # k beyond the last allocation: the handle was built
        break
    assert failures == 15
    monkeypatch.delenv("ATON_TEST_FAIL_ALLOC")
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < 16 * 2 ** 20
    a = A.from_workload(st, idx, rate, run)
    a.step(2)
    assert a.synchronize() == 0
    a.close()


def test_subcycle_cap_is_reported():
    st, idx, rate, run = W.workload_small()
    a = A.from_workload(st, idx, rate, run, max_sub=2)
    a.step(5)
    rc = a.synchronize()
    assert rc == A.ERR_SUBCYCLE
    assert a.last_error_cells() > 0
    with pytest.raises(A.AtonError) as e:
        a.step(1)
    assert e.value.code == A.ERR_SUBCYCLE
    a.close()


def test_degenerate_values_stay_finite():
    """Denormal and zero photon densities (with and without flux), fully neutral and fully
    ionised cells and gas at the temperature floor: the step stays finite and on the oracle."""
    st, idx, rate, run = W.workload_small(shape=(8, 12, 16), nsrc=2, seed_field=21, seed_src=22)
    c = run["c"]
    N = st["N"]
    N[0, 0, :4] = 1e-40                # FP32 denormals
    st["Fx"][0, 0, :4] = 0.5 * c * 1e-40
    N[1, 1, 3] = 0.0
    st["Fy"][1, 1, 3] = 1e-12          # flux with no photons (clamped away)
    N[2, 2, 2] = 1e-3
    st["Fz"][2, 2, 2] = 3.0 * c * 1e-3  # |F| > cN: unrealisable, treated as f = 1
    st["x"][3, :, :] = 1.0
    st["x"][4, :, :] = 0.0
    st["T"][5, :, :] = 1.0
    orc, _, _ = run_oracle(st, idx, rate, run, 8)
    for mode in (A.MODE_FUSED, A.MODE_UNFUSED):
        f, b, d, rc = run_gpu(st, idx, rate, run, 8, mode=mode)
        assert rc == 0 and d["nonfinite_cells"] == 0
        for k in ("N", "Fx", "Fy", "Fz", "y", "T"):
            assert np.isfinite(f[k]).all(), k
        assert_gates(errors(f, orc), mode)


def _one_cell(run, N, F, y, T, n, **kw):
    """One step of a 1x1x1 periodic grid: transport is the identity, so this is the chemistry
    operator of one cell through the C ABI."""
    h = A.Aton(1, 1, 1, run["dx"], run["c"], run["dt"])
    h.set_params(sigma_n=run["sigma_n"], sigma_e=run["sigma_e"], e_gamma_eV=run["e_gamma_eV"], **kw)
    f = lambda v: np.array([v], np.float32)  # noqa: E731
    h.set_fields(f(N), f(F[0]), f(F[1]), f(F[2]), f(T), f(n), y=f(y))
    h.step(1)
    rc = h.synchronize()
    out = h.get_fields()
    d = h.diag()
    h.close()
    return rc, {k: float(v.ravel()[0]) for k, v in out.items()}, d


def test_chemistry_of_single_cells_matches_the_oracle():
    """Random cell states over the ranges the workloads reach (n_H 1e-9..10 cm^-3, 0..100
    photons per atom, neutral to fully ionised, 1 K..1e6 K), plus the dense cold cell hit by
    40 photons per atom that needs ~100 sub-steps."""
    import oracle as O
    from parity_helpers import oracle_params
    st, idx, rate, run = W.workload_small(shape=(2, 2, 2), nsrc=1)
    p = oracle_params(run)
    rng = np.random.default_rng(5)
    cases = [(2.407596854603867e-05, 0.0, 0.9998999834060669, 1.0, 5.894661180401288e-07)]
    for _ in range(150):
        n = 10 ** rng.uniform(-9, 1)
        N = n * 10 ** rng.uniform(-8, 2) * (rng.random() < 0.85)
        y = 10 ** rng.uniform(-7, 0) if rng.random() < 0.5 else 1 - 10 ** rng.uniform(-6, 0)
        T = 10 ** rng.uniform(0, 6)
        cases.append((N, 0.3 * run["c"] * N, y, T, n))
    # chemically inert cells (cold, a faint field: the whole-step shortcut) and gas colder than
    # the floor (T_floor = 1 K), which the shortcuts leave to the full sub-step loop
    for _ in range(60):
        n = 10 ** rng.uniform(-9, 1)
        N = n * 10 ** rng.uniform(-16, -8)
        y = 1 - 10 ** rng.uniform(-6, -2)
        T = 10 ** rng.uniform(-2, 3.1)
        cases.append((N, 0.3 * run["c"] * N, y, T, n))
    worst = dict(x=0.0, T=0.0, N=0.0)
    for N, Fx, y, T, n in cases:
        N32, y32, T32, n32 = (float(np.float32(v)) for v in (N, y, T, n))
        F32 = float(np.float32(Fx))
        rc, g, d = _one_cell(run, N32, (F32, 0.0, 0.0), y32, T32, n32)
        assert rc == 0, (N, y, T, n, d)
        r = O.chem_cell(p, n32, N32, [F32, 0, 0], 1 - y32, T32)
        worst["x"] = max(worst["x"], abs(g["x"] - r["x"]))
        worst["T"] = max(worst["T"], abs(g["T"] - r["T"]) / r["T"])
        # the remainder of a cell that absorbs nearly all its photons goes as exp(-tau):
        # compared where more than 1e-3 of them are left
        if r["N"] > 1e-3 * N32:
            worst["N"] = max(worst["N"], abs(g["N"] - r["N"]) / r["N"])
    print("single-cell worst", worst)
    assert worst["x"] <= 1e-3 and worst["T"] <= 1e-3 and worst["N"] <= 1e-3, worst


def test_autotune_leaves_the_state_untouched(small):
    st, idx, rate, run = small
    a = A.from_workload(st, idx, rate, run)
    a.step(3)
    before = a.get_fields()
    b0 = a.photon_budget()
    ty, tz, ms = a.autotune(1)
    assert ty in (4, 8, 16) and 1 <= tz <= run["nz"] and ms > 0
    assert a.get_exec()["mode"] in (A.MODE_FUSED, A.MODE_FUSED_LDG)
    after = a.get_fields()
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    assert a.photon_budget() == b0
    a.step(2)
    assert a.synchronize() == 0
    a.close()


# clumping factors C_R = max(1, 1e3 nH^0.7), C_I = max(1, 10 nH^0.2): 2.6 and 1.8 at the mean
# density of the lognormal box, up to ~40 and ~3 in its densest cells
CLUMP = dict(clump_R_A=1e3, clump_R_b=0.7, clump_I_A=10.0, clump_I_b=0.2)


@pytest.mark.parametrize("mode", [A.MODE_FUSED, A.MODE_UNFUSED])
def test_clumping_chemistry_matches_the_oracle(small, small_oracle, mode):
    """Section 3.2.1, Eq. 15 (read with the signs of Eq. 14): the clumping factors multiply the
    recombination and photo-ionisation terms; parity with the oracle under the same gates."""
    st, idx, rate, run = small
    orc, ob, _ = run_oracle(st, idx, rate, run, 100, **CLUMP)
    f, b, d, rc = run_gpu(st, idx, rate, run, 100, mode=mode, **CLUMP)
    assert rc == 0
    e = errors(f, orc)
    print("clumping errors", mode, e)
    assert_gates(e, f"clumping mode {mode}")
    assert abs(budget_closure(b)) <= 1e-6
    assert b["absorbed"] == pytest.approx(ob["absorbed"], rel=1e-3)
    # the factors change the answer far beyond the gates
    assert np.abs(orc["x"] - small_oracle[0]["x"]).max() > 1e-2


@pytest.mark.parametrize("mode", [A.MODE_FUSED, A.MODE_UNFUSED])
def test_hll_flux_matches_the_oracle(small, small_oracle, mode):
    """The HLL intercell flux (section 2.2) with the M1 wave-speed bounds: parity with the
    oracle's HLL step, in the TMA-staged fused kernel (one launch) and in the plain step; it
    differs from the Lax-Friedrichs result well beyond the gates."""
    st, idx, rate, run = small
    orc, ob, _ = run_oracle(st, idx, rate, run, 100, flux=1)
    a = A.from_workload(st, idx, rate, run, flux=A.FLUX_HLL)
    a.set_exec(mode, 100)
    assert a.launches_per_step() == (1 if mode == A.MODE_FUSED else 3)
    a.step(100)
    assert a.synchronize() == 0
    f = a.get_fields()
    b = a.photon_budget()
    a.close()
    e = errors(f, orc)
    print("hll errors", mode, e)
    assert_gates(e, f"hll mode {mode}")
    assert abs(budget_closure(b)) <= 1e-6
    assert b["absorbed"] == pytest.approx(ob["absorbed"], rel=1e-3)
    glf = small_oracle[0]
    m = glf["N"] > 1e-6 * glf["N"].max()
    assert np.max(np.abs(orc["N"][m] / glf["N"][m] - 1)) > 1e-2


# shapes are (nz, ny, nx): x-ragged tiles (nx a multiple of 4, not of 32) with ny not a
# multiple of the tile height, a full-width grid with ragged y, and nx = 30 (not a multiple of
# 4), where fused HLL falls back to the plain three-kernel step
@pytest.mark.parametrize("shape,tile,launches", [((20, 22, 36), (4, 64), 1),
                                                 ((9, 13, 44), (8, 5), 1),
                                                 ((12, 40, 96), (16, 7), 1),
                                                 ((8, 10, 30), (4, 3), 3)])
@pytest.mark.parametrize("bc", ["periodic", "transmissive"])
def test_hll_fused_equals_plain_hll_closely(shape, tile, launches, bc):
    """The fused HLL kernel (closure pair and speed bounds shared through the ring) and the
    plain HLL step (every neighbour's closure and speeds recomputed) do the same arithmetic up
    to rounding: equal to 1e-5 after 20 steps, tallies alike. Each case checks which path ran."""
    st, idx, rate, run = W.workload_small(shape=shape, nsrc=3, seed_field=51, seed_src=52)
    r = dict(run, bc=bc)
    a = A.from_workload(st, idx, rate, r, flux=A.FLUX_HLL)
    a.set_exec(A.MODE_FUSED, 100)
    a.set_tile(*tile)
    assert a.launches_per_step() == launches
    a.close()
    f1, b1, d1, rc1 = run_gpu(st, idx, rate, r, 20, mode=A.MODE_FUSED, tile=tile, flux=A.FLUX_HLL)
    f2, b2, d2, rc2 = run_gpu(st, idx, rate, r, 20, mode=A.MODE_UNFUSED, flux=A.FLUX_HLL)
    assert rc1 == 0 and rc2 == 0
    for k in ("N", "Fx", "Fy", "Fz", "y", "T"):
        scale = np.abs(f2[k]).max()
        assert np.abs(f1[k] - f2[k]).max() <= 1e-5 * scale, (bc, k)
    assert b1["absorbed"] == pytest.approx(b2["absorbed"], rel=1e-5)
    assert b1["escaped"] == pytest.approx(b2["escaped"], rel=1e-5, abs=1e-9 * b2["emitted"])
    assert abs(budget_closure(b1)) <= 1e-6


@pytest.mark.parametrize("n,tile", [(32, None), (20, (8, 7))])
def test_hll_stromgren_transmissive_escape(n, tile):
    """HLL in the one-launch fused kernel against the oracle's HLL step on the transmissive
    Stromgren box: the 32^3 box (full tiles) and a 20^3 box with tile height 8 (20 = 2 x 8 + 4:
    ragged x and y tiles, whose outside slots are patched from the boundary map)."""
    st, idx, rate, run = W.stromgren_box(n=n, L_kpc=6.6 * n / 32)
    kw = dict(fixed_T=1, coll_ion=0)
    orc, ob, _ = run_oracle(st, idx, rate, run, 100, flux=1, **kw)
    a = A.from_workload(st, idx, rate, run, flux=A.FLUX_HLL, **kw)
    a.set_exec(A.MODE_FUSED, 100)
    if tile is not None:
        a.set_tile(*tile)
    assert a.launches_per_step() == 1
    a.close()
    f, b, d, rc = run_gpu(st, idx, rate, run, 100, flux=A.FLUX_HLL, tile=tile, **kw)
    assert rc == 0
    assert_gates(errors(f, orc))
    assert abs(budget_closure(b)) <= 1e-6
    assert b["escaped"] == pytest.approx(ob["escaped"], rel=1e-3, abs=1e-6 * ob["emitted"])


@pytest.mark.parametrize("mode", [A.MODE_FUSED, A.MODE_UNFUSED])
def test_largest_reduced_flux_is_reported(mode):
    """aton_diag.max_f: the largest |F|/(cN) of the current state, the realisability bound
    f <= 1 of the M1 closure (section 2.2), on a state streaming at up to f = 0.97."""
    st, idx, rate, run = W.workload_small(shape=(12, 16, 20), nsrc=2)
    rng = np.random.default_rng(5)
    shape = st["N"].shape
    N = rng.uniform(1e-6, 1e-3, shape)
    f = rng.uniform(0.0, 0.97, shape)
    n = rng.normal(size=(3,) + shape)
    n /= np.linalg.norm(n, axis=0)
    c = run["c"]
    st = dict(st, N=N, Fx=c * N * f * n[0], Fy=c * N * f * n[1], Fz=c * N * f * n[2])
    a = A.from_workload(st, idx, rate, run)
    a.set_exec(mode, 0)
    d0 = a.diag()
    a.step(3)
    assert a.synchronize() == 0
    d = a.diag()
    g = a.get_fields()
    a.close()
    N32 = st["N"].astype(np.float32).astype(np.float64)
    F32 = [st[k].astype(np.float32).astype(np.float64) for k in ("Fx", "Fy", "Fz")]
    assert d0["max_f"] == pytest.approx((np.sqrt(sum(x * x for x in F32)) / (c * N32)).max(),
                                        rel=1e-5)
    Ng = g["N"].astype(np.float64)
    fg = np.sqrt(sum(g[k].astype(np.float64) ** 2 for k in ("Fx", "Fy", "Fz"))) / (c * Ng)
    assert d["max_f"] == pytest.approx(fg[Ng > 1e-30].max(), rel=1e-5)
    assert d["max_f"] <= 1.0 + 1e-6


def test_budget_request_and_collect_match_the_synchronous_budget():
    """aton_budget_request/collect return, without stalling the stream, the budget as of the
    request: here each step's budget, collected while the next step runs."""
    st, idx, rate, run = W.workload_small(shape=(12, 16, 20), nsrc=3)
    a = A.from_workload(st, idx, rate, run)
    ref = A.from_workload(st, idx, rate, run)
    with pytest.raises(A.AtonError):
        a.budget_collect()                     # nothing requested
    got, want = [], []
    for k in range(6):
        a.step(1)
        if k:
            got.append(a.budget_collect())
        a.budget_request()
        ref.step(1)
        want.append(ref.photon_budget())
    got.append(a.budget_collect())
    a.budget_request()
    a.budget_request()                         # replaces the one not collected
    last = a.budget_collect()
    now = a.photon_budget()
    a.close()
    ref.close()
    for g, w in zip(got, want):
        for key in g:
            assert g[key] == pytest.approx(w[key], rel=1e-12, abs=1e-300), key
    for key in last:
        assert last[key] == pytest.approx(now[key], rel=1e-12, abs=1e-300), key


def test_weakly_photo_ionised_cold_gas_matches_the_oracle():
    """Cold, nearly neutral gas (x = 1e-4, 100 K) under photo-ionisation rates from faint to
    30 per cent per step (Gam dt): a step may raise x by orders of magnitude, so the
    recombinations at the end of a sub-step can matter where those at its start are negligible. The GPU step
    must follow the oracle's implicit update to FP32 accuracy here (no shortcut may drop a term
    that the end state makes visible)."""
    import oracle as O
    from parity_helpers import oracle_params
    st, idx, rate, run = W.workload_small(shape=(2, 2, 2), nsrc=1)
    ksig_dt = run["c"] * run["sigma_n"] * run["dt"]
    worst = 0.0
    # with the temperature fixed no heating limit shortens the sub-step, so one sub-step can
    # take x from 1e-4 to a few per cent
    for fixed_T, n, gdt in itertools.product((0, 1), 10.0 ** np.arange(-4.0, 1.01, 0.25),
                                         (1e-9, 1e-6, 1e-4, 1e-3, 1e-2, 5e-2, 0.1, 0.3)):
        p = oracle_params(run, fixed_T=fixed_T)
        N32, y32, T32, n32 = (float(np.float32(v)) for v in (gdt / ksig_dt, 1 - 1e-4, 100.0, n))
        rc, g, d = _one_cell(run, N32, (0.0, 0.0, 0.0), y32, T32, n32, fixed_T=fixed_T)
        assert rc == 0
        r = O.chem_cell(p, n32, N32, [0, 0, 0], 1 - y32, T32)
        # x = 1 - y is resolved to ~6e-8 near x = 0 in FP32 (two ulps of y allowed)
        dx = r["x"] - (1 - y32)
        err = abs(g["x"] - r["x"])
        worst = max(worst, err / max(dx, 1e-12))
        assert err <= 1e-4 * dx + 1.2e-7, (fixed_T, n, gdt, g["x"], r["x"], dx)
        assert abs(g["T"] - r["T"]) <= 1e-5 * r["T"], (fixed_T, n, gdt, g["T"], r["T"])
    print("weak photo-ionisation worst relative error of the change in x", worst)


def test_source_lists_merge_and_append():
    """Sources given in pieces (a cell listed twice with half its rate each, the list split
    between a replacing and an appending call) step exactly like the merged list."""
    st, idx, rate, run = W.workload_small(shape=(8, 16, 32), nsrc=5, seed_field=41, seed_src=42)
    ref, bref, _, _ = run_gpu(st, idx, rate, run, 10)
    a = A.from_workload(st, idx[:0], rate[:0], run)
    try:
        half = len(idx) // 2
        dup_i = np.concatenate([idx[:half], idx[:half]])
        dup_r = np.concatenate([rate[:half] / 2, rate[:half] / 2])
        a.add_sources(dup_i, dup_r)                                   # replace
        a.add_sources(idx[half:][::-1], rate[half:][::-1], mode=A.SRC_APPEND)
        a.step(10)
        assert a.synchronize() == 0
        f = a.get_fields()
        b = a.photon_budget()
    finally:
        a.close()
    for k in ("N", "Fx", "Fy", "Fz", "y", "T"):
        assert np.array_equal(f[k], ref[k]), k
    assert b["emitted"] == pytest.approx(bref["emitted"], rel=1e-12)
