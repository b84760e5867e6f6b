"""GPU checks of the chemistry-surrogate MLP kernels against the FP64 reference, of the pair
sink against the exact operator, and of the surrogate inside the step."""
import numpy as np
import pytest

from paper_1004_2503_b300 import aton as A
from paper_1004_2503_b300 import surrogate as S
from paper_1004_2503_b300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rand_theta(seed=0, scale=1.0):
    from oracle import mlp_oracle as M
    return (M.init(seed) * scale).astype(np.float32)


def test_forward_matches_the_bf16_reference():
    from oracle import mlp_oracle as M
    m = A.Mlp(seed=1)
    theta = _rand_theta(2)
    m.set_params(theta)
    rng = np.random.default_rng(3)
    X = rng.normal(0, 1, (1000, 5)).astype(np.float32)
    Y = m.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = M.forward(theta.astype(np.float64), X.astype(np.float64), round_bf16=True)
    exact = M.forward(theta.astype(np.float64), X.astype(np.float64))
    scale = np.abs(exact).max()
    assert np.abs(Y - ref).max() <= 2e-2 * scale
    assert np.abs(Y - exact).max() <= 4e-2 * scale
    m.close()


def test_gradient_matches_the_fp64_backprop():
    from oracle import mlp_oracle as M
    m = A.Mlp(seed=1)
    theta = _rand_theta(4)
    m.set_params(theta)
    rng = np.random.default_rng(5)
    n = 1000   # several CTAs and a ragged tail
    X = rng.normal(0, 1, (n, 5)).astype(np.float32)
    T = rng.normal(0, 1, (n, 3)).astype(np.float32)
    loss, g = m.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    g = g.cpu().numpy().astype(np.float64)
    lref, gref = M.loss_and_grad(theta.astype(np.float64), X.astype(np.float64),
                                 T.astype(np.float64))
    assert loss == pytest.approx(lref, rel=1e-2)
    gp, rp = M.unpack(g), M.unpack(gref)
    for k in rp:
        err = np.linalg.norm(gp[k] - rp[k]) / np.linalg.norm(rp[k])
        assert err <= 1e-2, (k, err)
    m.close()


def test_adam_kernel_applies_the_reference_update():
    from oracle import mlp_oracle as M
    m = A.Mlp(seed=1)
    theta = _rand_theta(6)
    m.set_params(theta)
    rng = np.random.default_rng(7)
    X = torch.from_numpy(rng.normal(0, 1, (512, 5)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(0, 1, (512, 3)).astype(np.float32)).cuda()
    th = theta.astype(np.float64)
    mm = np.zeros_like(th)
    vv = np.zeros_like(th)
    for step in (1, 2, 3):
        _, g = m.loss_grad(X, T)          # the kernels' gradient at the current weights
        m.train_step(X, T, 1e-3)
        th, mm, vv = M.adam(th, g.cpu().numpy().astype(np.float64), mm, vv, step, lr=1e-3)
        got = m.get_params().astype(np.float64)
        assert np.abs(got - th).max() <= 1e-6, step
    m.close()


def test_training_reduces_the_loss():
    m = A.Mlp(seed=3)
    rng = np.random.default_rng(8)
    X = rng.uniform(-2, 2, (16384, 5)).astype(np.float32)
    T = np.stack([np.sin(X[:, 0]) + 0.5 * X[:, 1], X[:, 2] * X[:, 3], np.tanh(X[:, 4])], 1)
    Xg = torch.from_numpy(X).cuda()
    Tg = torch.from_numpy(T.astype(np.float32)).cuda()
    l0 = m.train_step(Xg, Tg, 3e-3, want_loss=True)
    for _ in range(300):
        m.train_step(Xg, Tg, 3e-3)
    l1 = m.train_step(Xg, Tg, 3e-3, want_loss=True)
    assert l1 < 0.1 * l0
    m.close()


def test_pair_sink_records_match_the_exact_operator():
    import oracle as O
    from parity_helpers import oracle_params
    st, idx, rate, run = W.workload_small(shape=(12, 16, 20), nsrc=3)
    rec = S.collect_pairs([(st, idx, rate, run)], steps=6, stride=7, capacity=10 ** 6)
    per = -(-st["N"].size // 7)
    assert 6 * (per - 1) <= rec.shape[0] <= 6 * per
    r = rec.cpu().numpy().astype(np.float64)
    p = oracle_params(run)
    pick = np.argsort(-r[:, 7])[:40]          # the most sub-cycled records and a random few
    pick = np.concatenate([pick, np.random.default_rng(0).choice(len(r), 40, replace=False)])
    for i in pick:
        n, N, y, T, N1, y1, T1, ns = r[i]
        o = O.chem_cell(p, n, N, [0, 0, 0], 1 - y, T)
        assert abs((1 - o["x"]) - y1) <= 1e-3 and abs(o["T"] - T1) <= 1e-3 * o["T"]
        if o["N"] > 1e-3 * N:
            assert abs(o["N"] - N1) <= 1e-3 * o["N"]
        assert abs(o["nsub"] - ns) <= max(2, 0.05 * o["nsub"])


def test_surrogate_in_the_plain_step_keeps_the_budget_and_tracks_the_oracle(trained_surrogate):
    """The plain step's gate and surrogate passes (the fused step's are checked in
    test_gpu_surrogate_step.py): at the residual threshold 1e-4 the accepted predictions keep the
    absorbed photons and the ionised atoms within 1e-3 of the oracle, the ionised-volume radius
    within one cell, and the photon budget closed."""
    from parity_helpers import run_oracle
    st, idx, rate, run = W.cosmo_box(64, 2.0, 64, 201, 202)
    orc, ob, _ = run_oracle(st, idx, rate, run, 40)
    a = A.from_workload(st, idx, rate, run)
    a.set_exec(A.MODE_UNFUSED, 0)
    a.set_surrogate(trained_surrogate, gate_substeps=4.0, residual_max=1e-4)
    assert a.launches_per_step() == 4
    a.step(40)
    assert a.synchronize() == 0
    f = a.get_fields()
    b = a.photon_budget()
    d = a.diag()
    a.close()
    clos = (b["stored0"] + b["emitted"] - b["stored"] - b["absorbed"] - b["escaped"] -
            b["clipped"]) / b["emitted"]
    assert abs(clos) <= 1e-6                   # the tally follows whichever path ran
    assert d["surrogate_cells"] > 0
    assert b["absorbed"] == pytest.approx(ob["absorbed"], rel=1e-3)
    ion_ref = float(np.sum(st["nH"] * orc["x"]))
    ion = float(np.sum(st["nH"] * f["x"]))
    vol_ref = float(np.sum(orc["x"]))
    vol = float(np.sum(f["x"]))
    # ionised-volume radius in cells
    r_ref, r = ((3 * vol_ref / (4 * np.pi)) ** (1 / 3), (3 * vol / (4 * np.pi)) ** (1 / 3))
    print("surrogate cells", d["surrogate_cells"], "ionised atoms rel", ion / ion_ref - 1,
          "radius cells", r - r_ref)
    assert abs(ion / ion_ref - 1) <= 1e-3
    assert abs(r - r_ref) < 1.0


def test_surrogate_off_or_rejecting_everything_matches_the_exact_path():
    st, idx, rate, run = W.workload_small(shape=(8, 16, 16), nsrc=2)
    m = A.Mlp(seed=2)
    ref = A.from_workload(st, idx, rate, run)
    ref.set_exec(A.MODE_UNFUSED, 0)
    ref.step(10)
    fr = ref.get_fields()
    ref.close()
    a = A.from_workload(st, idx, rate, run)
    a.set_exec(A.MODE_UNFUSED, 0)
    a.set_surrogate(m, gate_substeps=0.0, residual_max=0.0)   # every prediction rejected
    a.step(10)
    f = a.get_fields()
    assert a.diag()["surrogate_cells"] == 0
    a.close()
    for k in ("N", "y", "T"):
        assert np.allclose(f[k], fr[k], rtol=1e-5, atol=0), k
    m.close()
