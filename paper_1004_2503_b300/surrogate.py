"""Training driver of the chemistry surrogate: pair collection from the exact operator and the
training loop. Every computation runs in libaton.so's kernels; this module only orders the
calls and draws mini-batch indices.
"""
import numpy as np

from . import aton as A
from . import workloads as W


def collect_pairs(workloads, steps, stride, capacity, warmup=0, keep_light=1.0, seed=0):
    """Records of the exact chemistry operator from the plain step on each workload.

    workloads: iterable of (state, src_idx, src_rate, run). Every `stride`-th cell of every step
    (offset rotating) is recorded after `warmup` unrecorded steps. Records whose operator took a
    single sub-step are kept with probability keep_light (the heavily sub-cycled ones, which
    the surrogate serves, are all kept). Returns a (n, 8) float32 torch CUDA tensor: nH, N, y,
    T, N', y', T', sub-steps.
    """
    import torch
    out = []
    left = capacity
    for st, idx, rate, run in workloads:
        if left <= 0:
            break
        a = A.from_workload(st, idx, rate, run)
        try:
            a.set_exec(A.MODE_UNFUSED, 0)
            if warmup:
                a.step(warmup)
            per = -(-st["N"].size // stride)
            cap = min(left, per * steps)
            # slots whose sampled cell falls beyond the grid stay unwritten: mark them
            buf = torch.full((cap, 8), float("nan"), dtype=torch.float32, device="cuda")
            a.set_pair_sink(buf, stride)
            a.step(steps)
            if a.synchronize() != 0:
                raise RuntimeError("step failed while collecting pairs")
            n = a.pair_count()
            a.set_pair_sink(None)
        finally:
            a.close()
        buf = buf[:n]
        buf = buf[~torch.isnan(buf[:, 0])]
        if keep_light < 1.0:
            g = torch.Generator(device="cuda")
            g.manual_seed(seed + len(out))
            u = torch.rand(buf.shape[0], device="cuda", generator=g)
            buf = buf[(buf[:, 7] > 1) | (u < keep_light)]
        out.append(buf)
        left -= buf.shape[0]
    return torch.cat(out)


def training_boxes(seeds, n=64, sigma_ln=1.5, nsrc=8):
    """Lognormal boxes of the 128^3 recipe at a smaller size, seeds disjoint from evaluation."""
    for s in seeds:
        yield W.cosmo_box(n, sigma_ln, nsrc, s, s + 1000)


def train(mlp, records, dt, steps=2000, batch=8192, lr=1e-3, lr_end=5e-5, heavy_weight=1.0,
          seed=0, log_every=0):
    """Standardise on the records, then Adam on mini-batches. Records whose exact operator took
    more than one sub-step (the regime the surrogate serves) are drawn heavy_weight times as
    often. Returns the loss history (one value per logged step)."""
    import torch
    mlp.fit_norm(records, dt)
    X, T = mlp.features(records, dt)
    nsub = records[:, 7]
    w = torch.where(nsub > 1, torch.full_like(nsub, heavy_weight), torch.ones_like(nsub))
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    hist = []
    for k in range(steps):
        sel = torch.multinomial(w, batch, replacement=True, generator=g)
        lr_k = lr * (lr_end / lr) ** (k / max(1, steps - 1))
        want = log_every and (k % log_every == 0 or k == steps - 1)
        loss = mlp.train_step(X[sel].contiguous(), T[sel].contiguous(), lr_k, want_loss=bool(want))
        if want:
            hist.append((k, loss))
    mlp.synchronize()
    return hist


def train_on_lognormal_boxes(seeds=range(100, 112), n=64, sigma_ln=1.5, nsrc=8, steps=120,
                             keep_light=0.01, train_steps=3000, batch=16384, capacity=40_000_000,
                             net_seed=11):
    """The surrogate of the 256^3 evaluation: pairs of the exact operator from lognormal boxes
    of the 128^3 recipe (sigma_ln = 1.5, one source per 32^3 cells) at n^3, seeds disjoint from
    every evaluation box, every heavily sub-cycled record and a `keep_light` share of the
    others, then `train_steps` Adam steps. Returns (network, number of records, dt)."""
    wl = list(training_boxes(seeds, n=n, sigma_ln=sigma_ln, nsrc=nsrc))
    rec = collect_pairs(wl, steps=steps, stride=1, capacity=capacity, keep_light=keep_light)
    m = A.Mlp(seed=net_seed)
    dt = wl[0][3]["dt"]
    train(m, rec, dt, steps=train_steps, batch=batch)
    return m, int(rec.shape[0]), dt


def front_cells_box(records, n, run, min_substeps=4, seed=7):
    """A periodic n^3 box of front-condition cells: every cell's (nH, N, y, T) drawn (seeded,
    with replacement) from the pair records whose exact operator took at least `min_substeps`
    sub-steps; F = 0, no sources. Returns (state, src_idx, src_rate, run) like the workload
    builders; `run` gives the cell size and time step of the runs the records came from."""
    rec = records[records[:, 7] >= min_substeps].cpu().numpy()
    if rec.shape[0] == 0:
        raise ValueError("no record with that many sub-steps")
    pick = rec[np.random.default_rng(seed).integers(0, rec.shape[0], n ** 3)]
    st = {k: pick[:, j].reshape(n, n, n).astype(np.float32)
          for k, j in (("nH", 0), ("N", 1), ("y", 2), ("T", 3))}
    st["x"] = (1.0 - st["y"]).astype(np.float32)
    for k in ("Fx", "Fy", "Fz"):
        st[k] = np.zeros((n, n, n), np.float32)
    return st, np.zeros(0, np.int64), np.zeros(0, np.float64), dict(run, nx=n, ny=n, nz=n)
