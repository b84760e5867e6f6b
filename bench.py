"""Benchmark of the ATON step on the 512^3 lognormal workload (one JSON line on rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--grid 512]

A step is one full radiative step: M1 transport with the Lax-Friedrichs flux, source
injection, sub-cycled chemistry/cooling/absorption and the photon tallies, for every cell.
Metric: cell-updates per second (grid cells x steps / time). Inputs are resident in HBM when
the timed region starts; the state (7.0 GB read+write per 512^3 step) is far larger than L2,
so no flush is needed between steps.

N > 1 (torchrun): every rank advances its own replica of the workload (the method does not
shard here); value = all ranks' cell-updates / max-over-ranks time ("weak" scaling).
--impl reference times the FP64 CPU oracle on the host cores (bounded sample per step).
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M1+chemistry cell-updates/s at 512^3; % of HBM roofline; surrogate speedup"
UNIT = "cell-updates/s"
BYTES_PER_CELL = 52.0   # read N,Fx,Fy,Fz,y,T,nH (28 B) + write N,Fx,Fy,Fz,y,T (24 B)
PLAIN_BYTES_PER_CELL = 84.0   # the plain three-kernel step: 32 B transport + 52 B chemistry
E2E_MIN_STEPS = 1000  # the end-to-end leg runs at least ten 100-step graph batches (the 512^3
                      # workload is timed over at least ten batches)
HBM_FALLBACK_GBS = 6400.0
# DRAM bytes per cell-update of the fused kernel from an ncu capture, keyed by the hash of the
# kernel sources it was taken on (the figure is dropped when the kernel changes).
NCU_TRAFFIC = {
    # k_fused_tma, tile 32x4x64, lognormal 256^3: dram__bytes_read.sum 486.51 MB +
    # dram__bytes_write.sum 362.43 MB per launch over 16,777,216 cells
    "39f8acbedd89": (486.513920e6 + 362.430208e6) / 16777216,
    # the same kernel with the surrogate hook and instances added (the exact instance's fields
    # bitwise unchanged): 486.89 MB + 362.55 MB
    "ac0f3ed55d18": (486.887168e6 + 362.554368e6) / 16777216,
    # two rows per thread, tile 32x8x48 (k_fused_tma<8,1,1,1,0,0,2>), lognormal 256^3:
    # 494.62 MB + 360.54 MB per launch (the second key: the same kernel, host-side launch code
    # changed after the capture)
    "98eeb2517f5f": (494.624e6 + 360.544256e6) / 16777216,
    "42f4dc9ef256": (494.624e6 + 360.544256e6) / 16777216,
    # the same kernel with the transport-only instance added (k_fused_tma<8,1,1,1,0,0,2,0>,
    # 94 registers): 495.06 MB + 361.03 MB per launch
    "93e67ba67e3f": (495.059968e6 + 361.030144e6) / 16777216,
    # the same GLF kernel after the HLL carried z face and the surrogate tail's staged weights
    # (k_fused_tma<8,1,1,1,0,0,2,0>, 94 registers, 221.4 us): 494.22 MB + 360.03 MB per launch
    "e8a166fc6af2": (494.2208e6 + 360.033792e6) / 16777216,
    # the same code with the kernel's signature reflowed (its text without whitespace unchanged)
    "4f0cd4ebb515": (494.2208e6 + 360.033792e6) / 16777216,
    # the same kernel; host code only: the transport-only instances' shared-memory attribute set
    # per device with the others instead of on their first launch
    "8a7101e6a1b5": (494.2208e6 + 360.033792e6) / 16777216,
}


def _code_only(text):
    """Source text without comments and blank lines (a comment edit leaves the kernel as it was)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", ln).strip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def kernel_hash(read=None):
    """Hash of the step kernels' code (comments excluded): the key of the ncu traffic figures."""
    h = hashlib.sha1()
    for f in ("aton_kernels.cu", "aton_tma.cu", "aton_device.cuh", "aton_step_common.cuh"):
        path = os.path.join(ROOT, "paper_1004_2503_b300", "csrc", f)
        if read is None:
            with open(path, encoding="utf-8") as fh:
                text = fh.read()
        else:
            text = read(f)
        h.update(_code_only(text).encode())
    return h.hexdigest()[:12]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        # the raw samples (a CSV kept beside the run: ATON_CLOCKS_DIR, else the temp directory)
        folder = os.environ.get("ATON_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, f"clocks_bench_{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def replica_time(t_local, dist=None, device="cpu"):
    """Timed region of a replicas-only run: every rank steps its own full workload, so the job
    takes as long as the slowest rank (max over ranks; the only collective of the run)."""
    if dist is None:
        return t_local
    import torch
    x = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def replica_value(world, ncell, steps, t):
    """Whole-job cell-updates per second: all ranks' cells and steps over the max-rank time."""
    return world * ncell * steps / t


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(grid):
    from paper_1004_2503_b300 import workloads as W
    if grid == 512:
        return W.workload_512(), ("lognormal n_H (sigma_ln=2.0, P(k)~k^-2.5, seed 3), 4096 sources "
                                  "at the highest peaks (log-uniform 1e50-1e52 /s, seed 4), "
                                  "dx=4 kpc, periodic, T0=100 K, x0=1e-4")
    if grid == 1024:
        return W.workload_1024(), ("lognormal n_H (sigma_ln=2.0, P(k)~k^-2.5, seed 5), 32768 "
                                   "sources at the highest peaks (log-uniform 1e50-1e52 /s, seed "
                                   "6), dx=4 kpc, periodic, T0=100 K, x0=1e-4, float32 state")
    st = W.cosmo_box(grid, 2.0, max(1, 4096 * grid ** 3 // 512 ** 3), 3, 4)
    return st, f"lognormal {grid}^3 (sigma_ln=2.0), scaled source count"


def cpu_sample(st, idx, rate, run, budget_cells):
    """Crop a periodic cube of the workload with about ``budget_cells`` cells (the CPU sample)."""
    from paper_1004_2503_b300 import workloads as W
    n = run["nx"]
    side = int(max(16, min(n, round(budget_cells ** (1 / 3) / 8) * 8)))
    # centre the crop on the brightest source so it holds fronts as well as neutral gas
    k, j, i = np.unravel_index(int(idx[np.argmax(rate)]), st["N"].shape)
    org = tuple(int(min(max(v - side // 2, 0), n - side)) for v in (k, j, i))
    cst, cidx, crate = W.subsample_state(st, idx, rate, (side, side, side), org)
    crun = dict(run, nx=side, ny=side, nz=side)
    return cst, cidx, crate, crun, side, org


def time_oracle(cst, cidx, crate, crun, steps, omp=False):
    import oracle as O
    p = O.params(c=crun["c"], dx=crun["dx"], dt=crun["dt"], sigma_n=crun["sigma_n"],
                 sigma_e=crun["sigma_e"], e_gamma_eV=crun["e_gamma_eV"], bc=O.BC_PERIODIC)
    t0 = time.perf_counter()
    O.run(p, cst, steps, cidx, crate, omp=omp)
    dt = time.perf_counter() - t0
    return cst["N"].size * steps / dt, dt


def surrogate_leg(args):
    """Chemistry surrogate inside the fused step at 256^3. The network is trained on pairs of
    the exact operator from lognormal boxes of the 128^3 recipe (seeds disjoint from the
    evaluation boxes); then, from the same state, three runs of each evaluation workload: the
    exact fused step; the fused step with the surrogate (gate 8 sub-steps, residual 1e-4: the
    kernel lists the selected cells of each CTA and, after its z-loop, runs the network for them
    and the exact operator for the rejected ones, in the same launch); and the same with every
    prediction rejected. Exact vs rejected is the cost of listing the cells; rejected vs
    surrogate is what the network saves on them. Each run with CUDA graphs first steps k times untimed with its
    final settings (so that the CUDA graph of k steps is captured and loaded outside the timed
    region), then times the next k steps."""
    import torch
    from paper_1004_2503_b300 import aton as A
    from paper_1004_2503_b300 import surrogate as S
    from paper_1004_2503_b300 import workloads as W
    t0 = time.perf_counter()
    wl = list(S.training_boxes(range(100, 112), n=64, sigma_ln=1.5, nsrc=8))
    rec = S.collect_pairs(wl, steps=120, stride=1, capacity=40_000_000, keep_light=0.01)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    m = A.Mlp(seed=11)
    S.train(m, rec, wl[0][3]["dt"], steps=3000, batch=16384)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    # (workload, warm-up steps, timed steps, CUDA graphs). The first 40 steps of the Stromgren
    # box, where the ionising source switches on in neutral gas, are the sub-cycling-heavy
    # case: they are timed from the initial state, so without graphs (one launch per step for
    # every run alike) instead of after an untimed pre-run.
    evals = {"lognormal_256_seed10": (W.workload_256(10, 1010), 5, 100, True),
             "stromgren_256": (W.stromgren_256(), 40, 100, True),
             "stromgren_256_first_40_steps": (W.stromgren_256(), 0, 40, False)}
    res = {}
    for wname, ((st, idx, rate, run), warm, k, graphs) in evals.items():
        out = {}
        for name, resid in (("exact", None), ("surrogate", 1e-4), ("rejected", 0.0)):
            a = A.from_workload(st, idx, rate, run)
            s = torch.cuda.Stream()
            a.set_stream(s)
            a.set_exec(A.MODE_FUSED, args.graph_batch if graphs else 0)
            a.step(warm)
            a.synchronize()
            if resid is not None:
                a.set_surrogate(m, gate_substeps=8.0, residual_max=resid)
            if graphs:
                a.step(k)
                a.synchronize()
            d0 = a.diag()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            a.step(k)
            e1.record(s)
            e1.synchronize()
            f = a.get_fields()
            b = a.photon_budget()
            d = a.diag()
            out[name] = dict(ms=e0.elapsed_time(e1) / k, x=f["x"], launches=a.launches_per_step(),
                             sur=(d["surrogate_cells"] - d0["surrogate_cells"]) / k,
                             sub=(d["substeps_total"] - d0["substeps_total"]) / (k * st["N"].size),
                             extra=(d["substeps_total"] - d0["substeps_total"] -
                                    k * st["N"].size) / k, submax=d["substeps_max"],
                             clos=(b["stored0"] + b["emitted"] - b["stored"] - b["absorbed"] -
                                   b["escaped"] - b["clipped"]) / b["emitted"])
            a.close()
        ion = lambda x: float(np.sum(st["nH"] * x))   # noqa: E731
        ex, su, rj = out["exact"], out["surrogate"], out["rejected"]
        res[wname] = {
            "steps": k, "after_warmup_steps": warm + k if graphs else warm,
            "cuda_graphs": graphs,
            "ms_per_step_exact": ex["ms"], "ms_per_step_surrogate": su["ms"],
            "ms_per_step_listed_exact": rj["ms"], "speedup": ex["ms"] / su["ms"],
            "launches_per_step": su["launches"],
            "surrogate_cells_per_step": su["sur"],
            "substeps_per_cell_update_exact": ex["sub"],
            "extra_substeps_per_step_exact": ex["extra"],
            "substeps_max_exact_since_start": ex["submax"],
            "ionised_atoms_rel_err": ion(su["x"]) / ion(ex["x"]) - 1,
            "max_abs_dx": float(np.abs(su["x"] - ex["x"]).max()),
            "budget_closure": su["clos"]}
    res["front_cells_128"] = front_cells_leg(m)
    m.close()
    return {"path": "fused step, network in the same launch", "residual_max": 1e-4, "gate_substeps": 8.0,
            "train_records": int(rec.shape[0]), "pair_collection_seconds": t1 - t0,
            "train_seconds": t2 - t1, "train_steps": 3000, "batch": 16384, **res}


def front_cells_workload():
    """The periodic 128^3 box of front-condition cells of the front-cells leg: every cell drawn
    from the exact operator's records with at least four sub-steps on lognormal boxes of the
    training recipe, seeds 300-303 (disjoint from training and evaluation); F = 0, no sources.
    Returns (state, src_idx, src_rate, run, records)."""
    from paper_1004_2503_b300 import surrogate as S
    wl = list(S.training_boxes(range(300, 304), n=64, sigma_ln=1.5, nsrc=8))
    rec = S.collect_pairs(wl, steps=120, stride=1, capacity=20_000_000, keep_light=0.0)
    st, idx, rate, run = S.front_cells_box(rec, 128, wl[0][3], min_substeps=4)
    return st, idx, rate, run, rec


def front_cells_step():
    """One exact plain step on the front-cells box, inside the NVTX start/end range
    'front_cells_exact_step' (for an ncu capture filtered to its chemistry pass); prints one
    JSON line with its CUDA-event time and the sub-steps per cell."""
    import torch
    from paper_1004_2503_b300 import aton as A
    st, idx, rate, run, _ = front_cells_workload()
    torch.cuda.empty_cache()   # (the pair records are dropped: little device memory in the capture)
    a = A.from_workload(st, idx, rate, run)
    s = torch.cuda.Stream()
    a.set_stream(s)
    a.set_exec(A.MODE_UNFUSED, 0)
    a.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    rid = torch.cuda.nvtx.range_start("front_cells_exact_step")
    e0.record(s)
    a.step(1)
    e1.record(s)
    e1.synchronize()
    torch.cuda.nvtx.range_end(rid)
    d = a.diag()
    a.close()
    print(json.dumps({"workload": "front_cells_128", "cells": st["N"].size,
                      "ms_plain_step": e0.elapsed_time(e1),
                      "substeps_per_cell": d["substeps_total"] / st["N"].size}), flush=True)


def front_cells_leg(m):
    """Where the exact operator sub-cycles heavily: a periodic 128^3 box whose every cell is
    drawn from the pair records of the exact operator that took >= 4 sub-steps, on lognormal
    boxes of the training recipe with seeds 300-303 (disjoint from training and evaluation);
    F = 0, no sources. One step from that state (best of three, no graphs), exact and with the
    surrogate at residual thresholds 1e-4 and 1e-3, in the plain three-kernel mode for both (its
    chemistry pass lists every candidate device-wide; the fused kernel lists at most 64 per
    CTA)."""
    import torch
    from paper_1004_2503_b300 import aton as A
    st, idx, rate, run, rec = front_cells_workload()
    ncell = st["N"].size
    out = {"cells": ncell, "records_ge4_substeps": int((rec[:, 7] >= 4).sum()),
           "records_gt1_substep": int(rec.shape[0])}
    ex = None
    for name, resid in (("exact", None), ("surrogate_1e-4", 1e-4), ("surrogate_1e-3", 1e-3)):
        best = None
        for _ in range(3):
            a = A.from_workload(st, idx, rate, run)
            s = torch.cuda.Stream()
            a.set_stream(s)
            a.set_exec(A.MODE_UNFUSED, 0)
            if resid is not None:
                a.set_surrogate(m, gate_substeps=8.0, residual_max=resid)
            a.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            a.step(1)
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            if best is None or ms < best[0]:
                f, b, d = a.get_fields(), a.photon_budget(), a.diag()
                best = (ms, float(np.sum(st["nH"].astype(np.float64) * f["x"])), b["absorbed"], d)
            a.close()
        ms, ion, ab, d = best
        r = {"ms": ms, "substeps_per_cell": d["substeps_total"] / ncell,
             "network_fraction": d["surrogate_cells"] / ncell}
        if ex is None:
            ex = best
        else:
            r.update(speedup=ex[0] / ms, ionised_atoms_rel_err=ion / ex[1] - 1,
                     absorbed_rel_err=ab / ex[2] - 1)
        out[name] = r
    return out


def reference_arm(args, world, rank):
    if rank != 0:
        return
    (st, idx, rate, run), desc = workload(args.grid)
    total = max(1, args.steps + args.warmup)
    # about 90 s of single-core oracle work in total (about 1 us per cell-update)
    cst, cidx, crate, crun, side, org = cpu_sample(st, idx, rate, run, 9e7 / total)
    import oracle as O
    p = O.params(c=crun["c"], dx=crun["dx"], dt=crun["dt"], sigma_n=crun["sigma_n"],
                 sigma_e=crun["sigma_e"], e_gamma_eV=crun["e_gamma_eV"], bc=O.BC_PERIODIC)
    cur = cst
    for _ in range(args.warmup):
        cur, _, _ = O.run(p, cur, 1, cidx, crate)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cur, _, _ = O.run(p, cur, 1, cidx, crate)
    dt = time.perf_counter() - t0
    v = cst["N"].size * args.steps / dt
    sample = f"{side}^3 periodic crop at {org} of the {args.grid}^3 workload, one step per step"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "grid": args.grid, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ours(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    from paper_1004_2503_b300 import aton as A
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    (st, idx, rate, run), desc = workload(args.grid)
    ncell = st["N"].size
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def maxtime(t):
        return replica_time(t, dist, "cuda")

    flux = {"glf": A.FLUX_GLF, "hll": A.FLUX_HLL}[args.flux]
    a = A.from_workload(st, idx, rate, run, flux=flux)
    a.set_stream(stream)
    if args.tile:
        ty, tz = (int(v) for v in args.tile.split(","))
        a.set_tile(ty, tz)
        if args.rows:
            a.set_tile_rows(args.rows)
        tune_ms = None
        a.set_exec({"tma": A.MODE_FUSED, "ldg": A.MODE_FUSED_LDG}.get(args.kernel, A.MODE_FUSED),
                   args.graph_batch)
    else:
        ty, tz, tune_ms = a.autotune(5)
    fused_mode = a.get_exec()["mode"]
    args.tile_rows = a.get_tile_rows()
    kernel = "k_fused_tma" if fused_mode == A.MODE_FUSED else "k_fused"
    a.set_exec(fused_mode, args.graph_batch)
    sur_info = None
    if args.with_surrogate:
        # the network of the surrogate leg (trained on lognormal boxes of the 128^3 recipe,
        # seeds disjoint from this workload), then the timed steps with it in the fused kernel
        from paper_1004_2503_b300 import surrogate as S
        t0s = time.perf_counter()
        sur_net, nrec, _ = S.train_on_lognormal_boxes()
        a.set_surrogate(sur_net, gate_substeps=8.0, residual_max=1e-4)
        sur_info = {"gate_substeps": 8.0, "residual_max": 1e-4, "train_records": nrec,
                    "train_seconds_incl_pairs": time.perf_counter() - t0s}
    a.step(args.warmup)
    a.synchronize()
    clocks = Clocks(local)
    barrier()
    clocks.start()
    history = []
    if args.history > 0:
        # timed in chunks of `history` steps; the statistics between chunks are not timed
        t_dev = 0.0
        done = 0
        while done < args.steps:
            k = min(args.history, args.steps - done)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            a.step(k)
            e1.record(stream)
            e1.synchronize()
            t_dev += e0.elapsed_time(e1) / 1e3
            done += k
            s = a.ionisation_stats()
            bb = a.photon_budget()
            history.append({"step": args.warmup + done, "x_volume": s["x_volume"],
                            "x_mass": s["x_mass"], "J21_volume": s["J21_volume"],
                            "T_volume": s["T_volume"],
                            "budget_closure": (bb["stored0"] + bb["emitted"] - bb["stored"] -
                                               bb["absorbed"] - bb["escaped"] - bb["clipped"]) /
                            max(bb["emitted"], 1e-300)})
        barrier()
        clk = clocks.stop()
        t = maxtime(t_dev)
        args.history_records = history
    else:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        a.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        barrier()
        clk = clocks.stop()
        t = maxtime(e0.elapsed_time(e1) / 1e3)
    rc = a.synchronize()
    diag = a.diag()
    bud = a.photon_budget()
    launches = a.launches_per_step() * args.steps
    if sur_info is not None:
        sur_info["surrogate_cells_per_step"] = diag["surrogate_cells"] / max(diag["steps"], 1)
        a.set_surrogate(None)
        sur_net.close()
        args.with_surrogate_info = sur_info
    value = replica_value(world, ncell, args.steps, t)
    ms = 1e3 * t / args.steps

    # plain unfused three-kernel step at the same accuracy, from the same state: the transport
    # pass (the TMA-staged kernel's transport-only instance, one closure per cell), the source
    # pass and the chemistry pass, each reading and writing its fields in HBM
    unfused = None
    ku = max(3, min(args.steps, 200))
    if args.no_unfused:
        ku = 0
    if ku:
        a.set_exec(A.MODE_UNFUSED, args.graph_batch)
        a.step(3)
        a.synchronize()
        u0 = torch.cuda.Event(enable_timing=True)
        u1 = torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        a.step(ku)
        u1.record(stream)
        u1.synchronize()
        tu = u0.elapsed_time(u1) / 1e3
        pk, _ = peaks()
        unfused = {"value": ncell * ku / tu, "ms_per_step": 1e3 * tu / ku,
                   "launches_per_step": a.launches_per_step(), "steps": ku,
                   "achieved_gbs_at_52B": BYTES_PER_CELL * ncell * ku / tu / 1e9,
                   # its own roofline: transport (read N, F; write N, F: 32 B) and chemistry
                   # (read N, F, y, T, nH; write N, F, y, T: 52 B) as separate passes
                   "bytes_per_cell_update": PLAIN_BYTES_PER_CELL,
                   "passes": "transport (k_fused_tma transport-only instance), sources, "
                             "chemistry (k_plain_chem)",
                   "frac_of_hbm_at_84B": PLAIN_BYTES_PER_CELL * ncell * ku / tu / 1e9 / pk}
    a.close()
    if args.no_e2e:
        return finish(args, world, rank, dist, st, idx, rate, run, desc, ncell, value, ms, t,
                      ty, tz, tune_ms, unfused, None, launches, clk, rc, diag, bud, kernel)

    # end to end through the C ABI with host buffers (pinned): state in, every step a source
    # list in and the photon budget out, state out at the end
    pin = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).pin_memory().numpy()
           for k, v in st.items()}
    ypin = torch.from_numpy(np.ascontiguousarray(1.0 - st["x"], np.float32)).pin_memory().numpy()
    outs = {k: torch.empty(st["N"].shape, dtype=torch.float32).pin_memory().numpy()
            for k in ("N", "Fx", "Fy", "Fz", "y", "T")}
    b = A.Aton(run["nx"], run["ny"], run["nz"], run["dx"], run["c"], run["dt"])
    b.set_params(bc=A.BC_PERIODIC, sigma_n=run["sigma_n"], sigma_e=run["sigma_e"],
                 e_gamma_eV=run["e_gamma_eV"], flux=flux)
    b.set_tile(ty, tz)
    b.set_tile_rows(args.tile_rows)
    b.set_exec(fused_mode, args.graph_batch)
    b.set_fields(pin["N"], pin["Fx"], pin["Fy"], pin["Fz"], pin["T"], pin["nH"], y=ypin)
    b.add_sources(idx, rate)
    b.step(1)
    b.budget_request()
    b.budget_collect()
    barrier()
    ke = max(args.steps, E2E_MIN_STEPS)
    t0 = time.perf_counter()
    b.set_fields(pin["N"], pin["Fx"], pin["Fy"], pin["Fz"], pin["T"], pin["nH"], y=ypin)
    for k in range(ke):
        b.add_sources(idx, rate)
        b.step(1)
        if k:
            b.budget_collect()      # the previous step's budget: ready while this step runs
        b.budget_request()
    b.budget_collect()
    b.get_fields(out=outs)
    barrier()
    te = maxtime(time.perf_counter() - t0)
    b.close()
    h2d = (7 * 4 * ncell) / ke + (8 + 8) * len(idx)
    d2h = 6 * 8 + (6 * 4 * ncell) / ke
    e2e = {"value": replica_value(world, ncell, ke, te), "unit": UNIT, "steps": ke,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "what": f"a {ke}-step run from host buffers: set_fields(host, pinned) once + per step "
                   "add_sources(host) + aton_step(1) + the step's photon budget to the host "
                   "(aton_budget_request after the step, collected while the next step runs) + "
                   "get_fields(host) once"}

    return finish(args, world, rank, dist, st, idx, rate, run, desc, ncell, value, ms, t,
                  ty, tz, tune_ms, unfused, e2e, launches, clk, rc, diag, bud, kernel)


def finish(args, world, rank, dist, st, idx, rate, run, desc, ncell, value, ms, t, ty, tz,
           tune_ms, unfused, e2e, launches, clk, rc, diag, bud, kernel):
    peak, peak_kind = peaks()
    achieved = BYTES_PER_CELL * ncell / (t / args.steps) / 1e9
    kh = kernel_hash()
    traffic = NCU_TRAFFIC.get(kh)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "grid": args.grid, "cells": ncell, "sources": len(idx),
                   "mode": kernel, "flux": args.flux, "graph_batch": args.graph_batch,
                   "tile_ty_tz": [ty, tz], "tile_rows_per_thread": getattr(args, "tile_rows", None),
                   "autotune_ms_per_step": tune_ms, "parallelism": f"replicas x{world}",
                   "l2": f"no flush: {44 * ncell / 1e9:.1f} GB of state per step >> 126 MB L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind,
                     "traffic": None if traffic is None else traffic * ncell,
                     "kernel": kernel, "bytes_per_cell_update": BYTES_PER_CELL,
                     "kernel_hash": kh},
        "unfused": unfused,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "status": rc,
        "history": getattr(args, "history_records", None) or None,
        "diag": diag,
        "with_surrogate": getattr(args, "with_surrogate_info", None),
        "budget_closure": (bud["stored0"] + bud["emitted"] - bud["stored"] - bud["absorbed"] -
                           bud["escaped"] - bud["clipped"]) / max(bud["emitted"], 1e-300),
    }
    if rank == 0 and not args.no_surrogate:
        line["surrogate"] = surrogate_leg(args)
    if rank == 0 and not args.no_cpu:
        cst, cidx, crate, crun, side, org = cpu_sample(st, idx, rate, run, 2.5e6)
        v1, d1 = time_oracle(cst, cidx, crate, crun, 4)
        vo, do = time_oracle(cst, cidx, crate, crun, 4, omp=True)
        line["cpu_baseline"] = {
            "value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"4 steps of a {side}^3 periodic crop at {org} of the same workload "
                      f"({d1:.1f} s)",
            "omp": {"value": vo, "cores": os.cpu_count(), "seconds": do}}
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=512)
    ap.add_argument("--graph-batch", type=int, default=100)
    ap.add_argument("--history", type=int, default=0,
                    help="time in chunks of this many steps and record the ionised fraction, "
                         "J21, T and the budget after each chunk (statistics not timed)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-unfused", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--with-surrogate", action="store_true",
                    help="run the timed steps with the chemistry surrogate in the fused kernel")
    ap.add_argument("--tile", default="", help="TY,TZ of the fused kernel (skips the autotuner)")
    ap.add_argument("--rows", type=int, default=0,
                    help="rows of the fused tile per thread (1 or 2; with --tile)")
    ap.add_argument("--flux", default="glf", choices=["glf", "hll"],
                    help="intercell flux: global Lax-Friedrichs (the paper's) or HLL")
    ap.add_argument("--kernel", default="tma", choices=["tma", "ldg"],
                    help="fused kernel used with --tile (the autotuner chooses otherwise)")
    ap.add_argument("--front-cells-step", action="store_true",
                    help="only one exact plain step on the front-cells box, inside an NVTX range "
                         "(for a filtered ncu capture of its chemistry pass)")
    args = ap.parse_args()
    if args.front_cells_step:
        front_cells_step()
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        reference_arm(args, world, rank)
    else:
        ours(args, world, rank, local)


if __name__ == "__main__":
    main()
