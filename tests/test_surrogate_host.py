"""Host logic of the surrogate driver that needs no GPU: the front-condition box built from
pair records of the exact operator."""
import numpy as np
import pytest


def test_front_cells_box_draws_only_heavy_records():
    """surrogate.front_cells_box: every cell's (nH, N, y, T) comes from a record with at least
    the requested sub-step count, F = 0, x = 1 - y, no sources, and the run is the given one
    resized; the draw is seeded."""
    import torch
    from paper_1004_2503_b300 import surrogate as S
    rng = np.random.default_rng(3)
    rec = np.zeros((50, 8), np.float32)
    rec[:, 0] = rng.uniform(1e-4, 1e-2, 50)          # nH
    rec[:, 1] = rng.uniform(1e-8, 1e-6, 50)          # N
    rec[:, 2] = rng.uniform(0.5, 1.0, 50)            # y
    rec[:, 3] = rng.uniform(100, 1e4, 50)            # T
    rec[:, 7] = np.arange(50) % 7                    # sub-steps 0..6
    run = dict(nx=64, ny=64, nz=64, dx=1.0, c=3e10, dt=1.0, bc="periodic")
    st, idx, rate, r = S.front_cells_box(torch.from_numpy(rec), 6, run, min_substeps=4)
    heavy = rec[rec[:, 7] >= 4]
    rows = {tuple(v) for v in heavy[:, :4]}
    got = np.stack([st["nH"].ravel(), st["N"].ravel(), st["y"].ravel(), st["T"].ravel()], 1)
    assert all(tuple(v) in rows for v in got)
    assert st["N"].shape == (6, 6, 6) and r["nx"] == r["ny"] == r["nz"] == 6 and r["dx"] == 1.0
    assert np.array_equal(st["x"], (1.0 - st["y"]).astype(np.float32))
    for k in ("Fx", "Fy", "Fz"):
        assert not st[k].any()
    assert idx.size == 0 and rate.size == 0
    st2, _, _, _ = S.front_cells_box(torch.from_numpy(rec), 6, run, min_substeps=4)
    assert np.array_equal(st["N"], st2["N"])
    with pytest.raises(ValueError):
        S.front_cells_box(torch.from_numpy(rec), 6, run, min_substeps=100)
