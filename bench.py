"""Throughput of the manufactured-solution PIC + DSMC step on GB300.

Default workload: the precision-form study (128^3 cells, 64 particles per
cell = 134,217,728 particles, K = 32, dt = 0.005, hard-sphere collisions at
0.01 expected collisions per particle per call). The headline value is the
precision form (FP32 particle state, int32 cell + FP32 offset, FP64-accurate
charge sums, CG inner products and error norms); the plain FP64 path runs
the same workload beside it, and both sets of MMS error norms are
reported. A step is one full velocity-Verlet step of every particle: two
K-averaged DSMC calls, kick, drift, sort, deposit, Poisson CG and E. The
library records, per timed step, the CG iterations and the candidate,
collision and g > g_max counts (its per-step history), which the line
carries. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload precision|precisionN|refine4|refineL|smallest|batched|batchedN|adjoint]
                  [--form mixed|fp64] [--no-fp64-beside] [--no-cpu-baseline]

The end-to-end figure (key "e2e") runs pic_set_state from pinned host
arrays, one step and pic_get_state into pinned host arrays; the library
reads and writes those arrays in place from its kernels (NVLink-C2C).
--impl reference times the FP64 CPU oracle (the only reference this method
has) on a bounded sample of the same workload on all host cores.
Multi-GPU: independent replicas (one per rank, own Philox seed), no
collective on the data path; value = particles x steps of all ranks / max
rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (PIC+DSMC, K-avg) vs plain FP64 at stated error; % HBM roofline"
UNIT = "particle-steps/s"


def workload(name: str) -> dict:
    from paper_2602_15130_gb300 import workloads as W

    if name == "precision":
        return W.precision_form()
    if name.startswith("precision"):
        # "precisionN": the same workload on N^3 cells (64 particles per cell)
        n = int(name[9:])
        return W.precision_form(n=n, n_particles=64 * n ** 3)
    if name.startswith("batched"):
        # "batched": the 256-replicate study; "batchedN": its first N replicates
        return {"batch": W.batched(int(name[7:]) if name[7:] else 256)}
    if name == "refine4":
        return W.refinement_level(4)
    if name.startswith("refine"):
        return W.refinement_level(int(name[6:]))
    if name == "smallest":
        return W.smallest()
    if name == "adjoint":
        return W.differentiation()
    raise SystemExit(f"unknown workload {name}")


def describe(name: str, p: dict) -> str:
    form = "precision form (FP32 state, FP64-accurate sums)" if p.get("precision") else "plain FP64"
    return (f"{name}: {p['n']}^3 cells, {p['n_particles']} particles, K={p['K']}, dt={p['dt']}, "
            f"hard-sphere sigma0={p['sigma0']:.4f}, {form}")


# ----------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock samples unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json: STREAM-style copy)"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


# Algorithmic HBM bytes per unit of each kernel class of one step: what the
# method must move, per particle for the particle kernels (one launch
# processes every particle), per node for the RHS and per node-iteration for
# the CG. "method": the per-particle-step figures the method implies for
# the FP32 state of 56 B (cell, three offsets, three velocities, three xi,
# three v^M, pid; this implementation regenerates xi from the pid instead
# of storing it) or the FP64 state of 104 B: the push
# reads and writes the state once per step (two launches: half each), the
# sort scatter reads and writes it once, the deposit reads the positions
# once, and each CG iteration moves about 28 B (FP32) or 56 B (FP64) per
# node. "impl": the arrays this implementation's kernels read and write once
# (for example the precision-form drift launch: cell, three offsets, three
# velocities after the collision half kick, three v^M, pid and three Lorentz
# terms in; three offsets, three velocities, key and slot out: 88 B; the
# closing kick, by cells: three offsets and three velocities in, three
# velocities and three Lorentz terms out: 48 B).
BYTES_PER_UNIT = {
    "fp64": {
        "method": {"kick_drift": 104.0, "sort_gather_deposit": 208.0 + 24.0, "cg_efield": 56.0},
        "impl": {"kick_drift": (228 + 120) / 2.0, "sort_gather_deposit": 208 + 64 / 32.0, "dsmc": 48.0,
                 "sort": 12.0, "cg_efield": 88.0, "rhs": 8 * 8 + 16},
    },
    "mixed": {
        "method": {"kick_drift": 56.0, "sort_gather_deposit": 112.0 + 16.0, "cg_efield": 28.0},
        "impl": {"kick_drift": (88 + 48) / 2.0, "sort_gather_deposit": 88 + 64 / 32.0, "dsmc": 24.0,
                 "sort": 12.0, "cg_efield": 44.0, "rhs": 8 * 8 + 8 + 4},
    },
}

# Integer and FP operations per candidate pair of the collision algorithm
# (the middle of the 200-300 range of the method's statement of work: one
# Philox4x32-10 block and a quarter at about 100 integer operations each,
# the index draws, the relative speed, the accept test, and the scattering
# of the accepted ones)
OPS_PER_CANDIDATE = 250

# DRAM bytes of one launch of the dominant kernels, per unit, from an ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the
# kernel source it was taken on: bench.py compares the source file's hash
# and reports null traffic once the kernel has changed.
NCU_TRAFFIC = {
    ("mixed", "dsmc"): {
        "bytes_per_unit": 22.69,
        # the collision kernel and its device routines, its launch, and the
        # device code of the headers they include (the shared header up to
        # its sort-gather section, which the collision kernel does not use):
        # (path, first line, line after) or whole files
        "sources": [
            ("paper_2602_15130_gb300/csrc/k_mixed.cu", "struct Counts32 {",
             "// ------------------------------------------------------------ kick/drift --"),
            ("paper_2602_15130_gb300/csrc/k_mixed.cu", "cudaError_t launch_dsmc32(", "\n}\n"),
            ("paper_2602_15130_gb300/csrc/mixed_common.cuh",
             "// Device helpers shared by the precision-form kernels (single domain and",
             "// ----------------------------------------------------- sort gather + CIC --"),
            ("paper_2602_15130_gb300/csrc/pic_internal.cuh", "// Internal definitions",
             "// Context (host side)"),
        ],
        "sha16": "f6d9375ef1dd8ba7",
        "how": "ncu --set full of k_dsmc32 at 64^3 (--workload precision64, both calls of a step): "
               "dram__bytes_read.sum + dram__bytes_write.sum = 22.69 B per particle, times the "
               "launch's particles (the state exceeds L2 at both sizes)",
    },
}


def source_hash(sources) -> str:
    """Hash of the source text a kernel is built from: whole files, or the
    span of a file from a first line to the next occurrence of an end
    marker; empty when a marker is missing."""
    h = hashlib.sha256()
    for path, first, end in sources:
        with open(os.path.join(ROOT, path), "rb") as f:
            text = f.read()
        if first is not None:
            i = text.find(first.encode())
            j = text.find(end.encode(), i + 1) if i >= 0 else -1
            if i < 0 or j < 0:
                return ""
            text = text[i:j]
        h.update(text)
    return h.hexdigest()[:16]


def traffic_per_launch(form: str, kernel: str, units: float):
    e = NCU_TRAFFIC.get((form, kernel))
    if not e or source_hash(e["sources"]) != e["sha16"]:
        return None, None
    return e["bytes_per_unit"] * units, e["how"]


# ------------------------------------------------------------- replicas -----
def replica_params(p: dict, rank: int) -> dict:
    """Each rank runs an independent replica: same workload, own Philox seed."""
    q = dict(p)
    q["seed"] = int(p.get("seed", 0)) + rank
    return q


def max_over_ranks(x: float, device: str = "cpu") -> float:
    """Max of a per-rank scalar over the process group (timing only)."""
    import torch
    import torch.distributed as td

    if not td.is_available() or not td.is_initialized() or td.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(n_particles: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job particle-steps/s: all ranks' particle-steps over the slowest rank's time."""
    return world * n_particles * steps / (max_ms / 1000.0)


# ----------------------------------------------------------------- GPU arm ---
def per_step(hist) -> dict:
    """The library's per-step history of the timed steps, as lists."""
    return {"cg_iters": [int(r[0]) for r in hist], "n_cand": [int(r[1]) for r in hist],
            "n_coll": [int(r[2]) for r in hist], "n_gmax_exceed": [int(r[3]) for r in hist]}


# The precision form solves meshes of 2^k >= 16 nodes an edge by CG
# preconditioned with a multigrid V-cycle: an iteration then moves about
# 125 B a fine node (the product A p, the vector updates, the V-cycle's
# four smoothing sweeps, residual, restriction and prolongation on the
# finest level, and about a seventh more on the coarser ones), and the
# plain CG's per-iteration figure of the method does not apply.
MG_CG_BYTES_PER_NODE_ITERATION = 125.0


def multigrid_cg(p: dict, form: str) -> bool:
    n = int(p["n"])
    return form == "mixed" and n >= 16 and n & (n - 1) == 0


def class_rates(p: dict, form: str, kt: dict, st: dict, hbm: float) -> dict:
    """Per kernel class: ms per launch and the achieved fraction of the
    measured HBM bandwidth by the method's bytes and by the implementation's."""
    out = {}
    mg = multigrid_cg(p, form)
    for k, v in kt.items():
        if not v["launches"]:
            continue
        ms = v["ms"] / v["launches"]
        units = p["n"] ** 3 * max(1, st["cg_iters_mean"]) if k == "cg_efield" else (
            p["n"] ** 3 if k == "rhs" else p["n_particles"])
        row = {"ms_per_launch": round(ms, 4), "launches": v["launches"], "units_per_launch": units}
        for which in ("method", "impl"):
            b = BYTES_PER_UNIT[form][which].get(k)
            if mg and k == "cg_efield":
                b = MG_CG_BYTES_PER_NODE_ITERATION if which == "impl" else None
            if b is not None and ms > 0:
                gbs = b * units / (ms * 1e-3) / 1e9
                row[f"bytes_per_unit_{which}"] = b
                row[f"gbs_{which}"] = round(gbs, 1)
                row[f"frac_of_measured_hbm_{which}"] = round(gbs / hbm, 4)
        out[k] = row
    return out


def run_gpu(args, rank: int, world: int, form: str, with_e2e: bool = True) -> dict | None:
    import numpy as np
    import torch

    from paper_2602_15130_gb300 import Pic, measure_alu_peaks, measure_link, workloads as W

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    p = workload(args.workload)
    if form == "mixed":
        p = W.mixed(p)
    else:
        p = dict(p, precision=0)
    p = replica_params(p, rank)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = Pic(p, stream=stream)
        # sampling (A1 with the first sort and field) and the error norms
        # (A10) are timed apart from the steps: one warm call each on the
        # host clock (each call returns with its stream synchronised)
        sim.sample_mms(0.0)
        t_s = time.perf_counter()
        sim.sample_mms(0.0)
        sample_ms = (time.perf_counter() - t_s) * 1000.0
        sim.step(args.warmup)
        dist = world > 1
        if dist:
            import torch.distributed as td
            td.barrier()
        torch.cuda.synchronize()
        sim.reset_stats()  # counters, and the per-step history starts here
        sim.set_profiling(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev) as clk:
            time.sleep(0.3)
            ev0.record(stream)
            sim.step(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        kt = sim.kernel_times()
        st = sim.stats()
        hist = sim.step_history()
        sim.set_profiling(False)
        ms = max_over_ranks(ms, "cuda")
        sim.mms_error()
        t_e = time.perf_counter()
        errs = sim.mms_error()
        err_ms = (time.perf_counter() - t_e) * 1000.0
        npart = p["n_particles"]
        apart = {"sample_mms": {"ms": sample_ms, "particles_per_s": npart / (sample_ms * 1e-3)},
                 "mms_error": {"ms": err_ms, "particles_per_s": npart / (err_ms * 1e-3)},
                 "how": "host clock around one warm call each, outside the timed steps"}
        st["cg_iters_mean"] = float(np.mean(hist[:, 0])) if len(hist) else float(st["cg_iters_max"])
        stats = {"n_coll": st["n_coll"], "n_cand": st["n_cand"], "n_gmax_exceed": st["n_gmax_exceed"],
                 "n_near_ties": st["n_near_ties"], "n_floor_ties": st["n_floor_ties"],
                 "cg_iters_mean": round(st["cg_iters_mean"], 2), "cg_iters_max": st["cg_iters_max"],
                 "cg_res_last": st["cg_res_last"]}
        if not with_e2e:
            sim.close()
            if rank != 0:
                return None
            return {"value": aggregate_value(npart, args.steps, world, ms), "ms_per_step": ms / args.steps,
                    "kernel_ms": {k: round(v["ms"], 3) for k, v in kt.items()},
                    "kernels": class_rates(p, form, kt, st, measured_peaks()["hbm_gbs"]),
                    "mms_error": {"eps2": errs["eps2"], "epsinf": errs["epsinf"]},
                    "stats": stats, "per_step": per_step(hist), "timed_apart": apart, "clocks": clk.summary()}
        # end to end through the C ABI with host buffers: pinned x, v in, step, x, v out
        xh = torch.empty((npart, 3), dtype=torch.float64, pin_memory=True)
        vh = torch.empty((npart, 3), dtype=torch.float64, pin_memory=True)
        sim.get_state((xh, vh))
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        if dist:
            td.barrier()
        t0 = time.perf_counter()
        call_s = [0.0, 0.0, 0.0]  # each call returns with its stream synchronised
        for _ in range(e2e_steps):
            ta = time.perf_counter()
            sim.set_state(xh, vh, 0.0, int(st["step"]))
            tb = time.perf_counter()
            sim.step(1)
            tc = time.perf_counter()
            sim.get_state((xh, vh))
            te = time.perf_counter()
            call_s[0] += tb - ta
            call_s[1] += tc - tb
            call_s[2] += te - tc
        e2e_s = max_over_ranks(time.perf_counter() - t0, "cuda")
        # the host link's own rate each way, by DMA copies of the same pinned
        # buffer (pic_measure_link): the ceiling of the state's load and store
        lk = measure_link(xh, stream)
        link = {"h2d_gbs": lk["h2d"] / 1e9, "d2h_gbs": lk["d2h"] / 1e9, "bytes": lk["bytes"],
                "source": "pic_measure_link: cudaMemcpyAsync of an end-to-end pinned buffer in this run"}
        sim.close()
        alu = measure_alu_peaks(stream) if rank == 0 else None
    if rank != 0:
        return None
    value = aggregate_value(npart, args.steps, world, ms)
    peaks = measured_peaks()
    kernels = class_rates(p, form, kt, st, peaks["hbm_gbs"])
    # dominant kernel class by device time inside the timed region
    dom = max(kt, key=lambda k: kt[k]["ms"])
    row = kernels[dom]
    if dom == "dsmc":
        # integer/FP ALU bound: the method's work is its candidate pairs at
        # OPS_PER_CANDIDATE integer and FP operations each (one Philox4x32-10
        # block and a quarter, the index draws, g, the accept test and, for
        # the accepted ones, the scattering), against this GPU's INT32 issue
        # rate measured in this run (the multiply-add pipe that Philox loads)
        nl = max(1, kt["dsmc"]["launches"])
        cand = st["n_cand"] / nl
        per_launch_s = kt["dsmc"]["ms"] / nl / 1000.0
        achieved = cand * OPS_PER_CANDIDATE / per_launch_s / 1e12
        peak = alu["imad"] / 1e12
        # Philox blocks per launch: an outcome with N candidates takes
        # N + floor(N / 4) + 1 (the chi stream's first block carries the
        # N_pairs uniform), so the totals bound them between outcomes +
        # candidates and outcomes + 1.25 candidates
        outcomes = p["n"] ** 3 * p["K"]
        blocks = (outcomes + cand, outcomes + 1.25 * cand)
        traffic, how = traffic_per_launch(form, "dsmc", npart)
        roof = {"bound": "alu", "kernel": "dsmc", "achieved": achieved, "peak": peak, "unit": "Tops/s (INT32)",
                "frac": achieved / peak, "traffic": traffic, "traffic_source": how,
                "ops_per_candidate": OPS_PER_CANDIDATE, "candidates_per_launch": cand,
                "peak_source": "measured in this run: INT32 multiply-add issue rate of a full-grid kernel "
                               "(pic_measure_alu_peaks); 64 lanes x SMs x clock gives the same",
                "philox_block_frac_range": [b / per_launch_s / alu["philox_blocks"] for b in blocks],
                "ms_per_launch": row["ms_per_launch"]}
    else:
        b = BYTES_PER_UNIT[form]["method"].get(dom) or BYTES_PER_UNIT[form]["impl"].get(dom, 0.0)
        units = row["units_per_launch"]
        achieved = b * units / (row["ms_per_launch"] * 1e-3) / 1e9
        traffic, how = traffic_per_launch(form, dom, units)
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "traffic_source": how,
                "peak_source": peaks["source"], "bytes_per_unit": b, "units_per_launch": units,
                "ms_per_launch": row["ms_per_launch"]}
    launches = int(st["kernel_launches"])
    # the link's share of the end-to-end step: 48 B a particle each way
    # (x and v in FP64) at the rates measured on the same buffers
    e2e_ms = e2e_s * 1000.0 / e2e_steps
    h2d_ms = npart * 48 / (link["h2d_gbs"] * 1e9) * 1e3
    d2h_ms = npart * 48 / (link["d2h_gbs"] * 1e9) * 1e3
    calls = {k: v * 1000.0 / e2e_steps for k, v in zip(("set_state", "step", "get_state"), call_s)}
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if form == "mixed" else "f64",
        "data": "synthetic manufactured-solution workload",
        "config": {"workload": describe(args.workload, p), "n": p["n"], "n_particles": npart, "K": p["K"],
                   "dt": p["dt"], "sigma0": p["sigma0"], "form": form, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (particle state %.1f GB)" % (npart * (44 if form == "mixed" else 100) / 1e9)},
        "e2e": {"value": aggregate_value(npart, e2e_steps, world, e2e_s * 1000.0), "unit": UNIT,
                "h2d_bytes_per_step": npart * 48, "d2h_bytes_per_step": npart * 48,
                "path": "pic_set_state(host) + pic_step(1) + pic_get_state(host), pinned buffers",
                "ms_per_step": e2e_ms, "ms_per_call": calls,
                "link": dict(link, h2d_ms_floor=h2d_ms, d2h_ms_floor=d2h_ms,
                             set_state_link_frac=h2d_ms / calls["set_state"],
                             get_state_link_frac=d2h_ms / calls["get_state"],
                             floor_ms_per_step=h2d_ms + d2h_ms + ms / args.steps)},
        "gpu_launches": launches,
        "roofline": roof,
        "kernels": kernels,
        "kernel_ms": {k: round(v["ms"], 3) for k, v in kt.items()},
        "alu_peaks_per_s": alu,
        "stats": stats,
        "per_step": per_step(hist),
        "timed_apart": apart,
        "mms_error": {"eps2": errs["eps2"], "epsinf": errs["epsinf"]},
        "clocks": clk.summary(),
    }


# --------------------------------------------------------------- batches ---
def run_batched(args, rank: int, world: int) -> dict | None:
    """256 uneven replicates advanced together (pic_create_batch)."""
    import torch

    from paper_2602_15130_gb300 import Batch, measure_alu_peaks

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cfgs = [replica_params(p, rank * 100000) for p in workload(args.workload)["batch"]]
    npart = sum(p["n_particles"] for p in cfgs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = Batch(cfgs, stream=stream)
        b.sample_mms(0.0)
        b.step(max(args.warmup, 4))  # 3 autotuning steps, then graph capture
        torch.cuda.synchronize()
        b.reset_stats()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev) as clk:
            time.sleep(0.3)
            ev0.record(stream)
            b.step(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = max_over_ranks(ev0.elapsed_time(ev1), "cuda")
        st = b.stats()
        # per-phase times from a profiled pass (one launch per phase instead
        # of the persistent step)
        b.set_profiling(True)
        b.step(1)
        kt = b.kernel_times()
        b.set_profiling(False)
        cand_prof = b.stats()["n_cand"] - st["n_cand"]
        errs = b.mms_error()
        iters = b.cg_iters()
        b.close()
        alu = measure_alu_peaks(stream) if rank == 0 else None
    if rank != 0:
        return None
    ns = sorted({p["n"] for p in cfgs})
    # the dominant phase, collisions, against the INT32 issue rate measured in
    # this run: the profiled step's candidate pairs at OPS_PER_CANDIDATE
    # operations each over its collision launches' time (the per-phase pass
    # runs the collision phase as launches of its own)
    dsmc_s = kt["dsmc"]["ms"] / 1000.0
    achieved = cand_prof * OPS_PER_CANDIDATE / dsmc_s / 1e12 if dsmc_s > 0 else 0.0
    roof = {"bound": "alu", "kernel": "dsmc (kb_dsmc, the profiled step's collision launches)",
            "achieved": achieved, "peak": alu["imad"] / 1e12, "unit": "Tops/s (INT32)",
            "frac": achieved / (alu["imad"] / 1e12), "traffic": None,
            "traffic_source": "not captured for the batched collision kernel",
            "ops_per_candidate": OPS_PER_CANDIDATE, "candidates": cand_prof,
            "peak_source": "measured in this run (pic_measure_alu_peaks)",
            "ms": kt["dsmc"]["ms"], "launches": kt["dsmc"]["launches"]}
    return {
        "metric": METRIC, "value": aggregate_value(npart, args.steps, world, ms), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 4), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic manufactured-solution workload",
        "config": {"workload": "batched: %d replicates, n in %s, %d particles in total, K in [%d, %d], dt = 0.005, "
                               "precision form" % (len(cfgs), ns, npart, min(p["K"] for p in cfgs),
                                                   max(p["K"] for p in cfgs)),
                   "n_particles": npart, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2"},
        "e2e": None, "e2e_note": "batches have no host-buffer input path (states are sampled on the device)",
        "gpu_launches": int(st["kernel_launches"]), "graph_replays": int(st["graph_replays"]),
        "launches_per_step": int(st["kernel_launches"]) / max(1, args.steps),
        "tuned_block": int(st["tuned_block"]), "tuned_tile": int(st["tuned_tile"]),
        "kernel_ms_one_profiled_step": {k: round(v["ms"], 3) for k, v in kt.items()},
        "roofline": roof,
        "stats": {"n_coll": st["n_coll"], "n_cand": st["n_cand"], "n_near_ties": st["n_near_ties"],
                  "cg_iters_max": st["cg_iters_max"], "cg_iters_median": sorted(iters)[len(iters) // 2]},
        "mms_error_eps2_x_median": float(sorted(e[0] for e in errs)[len(errs) // 2]),
        "clocks": clk.summary(),
    }


def run_adjoint(args) -> dict:
    """One pathwise gradient of J (field energy + velocity error at t_N)
    with respect to E_app and v0 on the differentiation workload (collisions
    on, pairs frozen), timed with CUDA events after a warm-up gradient. With
    collisions, J is discontinuous in E_app at this size (a 1e-6 change
    moves cell memberships and with them whole cells' pair draws), so the
    central-difference check (h = 1e-6) of dJ/dE_app runs on the same
    workload without collisions, where J is smooth."""
    import numpy as np
    import torch

    from paper_2602_15130_gb300 import Pic

    torch.cuda.set_device(0)
    p = workload("adjoint")
    steps, every, E = p["steps"], p["checkpoint_every"], tuple(p["E_app"])
    sim = Pic(p)
    sim.adjoint_gradient(steps, every, E)  # warm-up: allocates the working set
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record()
        r = sim.adjoint_gradient(steps, every, E)
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    ev0.record()
    sim.adjoint_gradient(steps, every, E, grad=False)
    ev1.record()
    torch.cuda.synchronize()
    ms_fwd = ev0.elapsed_time(ev1)
    st = sim.stats()
    sim.close()
    del sim
    # central differences without collisions
    p0 = dict(p, K=0)
    s0 = Pic(p0)
    r0 = s0.adjoint_gradient(steps, every, E)
    fd = []
    for d in range(3):
        ep, em = list(E), list(E)
        ep[d] += 1e-6
        em[d] -= 1e-6
        jp = s0.adjoint_gradient(steps, every, ep, grad=False)["J"]
        jm = s0.adjoint_gradient(steps, every, em, grad=False)["J"]
        fd.append((jp - jm) / 2e-6)
    g0 = r0["dJ_dEapp"]
    return {
        "metric": "pathwise gradient of J(E_app, v0): particle-steps/s (forward with checkpoints + adjoint)",
        "value": p["n_particles"] * steps / (ms / 1e3), "unit": "particle-steps/s", "n_gpus": 1,
        "steps": steps, "warmup": 1, "ms_per_gradient": ms, "ms_forward_only": ms_fwd,
        "gradient_over_forward": ms / ms_fwd, "higher_is_better": True, "dtype": "f64",
        "data": "synthetic manufactured-solution workload",
        "config": {"workload": describe("adjoint", p), "n": p["n"], "n_particles": p["n_particles"], "K": p["K"],
                   "dt": p["dt"], "steps": steps, "checkpoint_every": every, "E_app": list(E)},
        "J": r["J"], "J_field": r["J_field"], "J_vel": r["J_vel"], "dJ_dEapp": [float(x) for x in r["dJ_dEapp"]],
        "dJ_dv0_rms": float(np.sqrt(np.mean(r["dJ_dv0"] ** 2))),
        "stats": {"n_coll": st["n_coll"], "n_gmax_exceed": st["n_gmax_exceed"], "cg_iters_max": st["cg_iters_max"]},
        "fd_check_collisionless": {"J": r0["J"], "dJ_dEapp": [float(x) for x in g0], "fd": fd,
                                   "rel_err": [abs(g0[d] - fd[d]) / max(abs(fd[d]), 1e-300) for d in range(3)]},
        "clocks": clk.summary(),
    }


# ------------------------------------------------------------ CPU oracle ----
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample_params(args, n_small: int) -> tuple[dict, str]:
    from paper_2602_15130_gb300 import workloads as W

    p = workload(args.workload)
    n_small = min(p["n"], n_small)
    q = W.scaled(p, n_small)
    return q, (f"oracle on a {n_small}^3 sub-problem with the workload's particles per cell, K, dt and sigma0 "
               f"({q['n_particles']} particles)")


def run_oracle_steps(q: dict, steps: int, warmup: int, threads: int) -> tuple[float, float, int]:
    from oracle import oracle as O

    used = O.set_threads(threads)
    try:
        o = O.Oracle(q)
        o.sample(0.0)
        if warmup:
            o.step(warmup)
        t0 = time.perf_counter()
        o.step(steps)
        dt = time.perf_counter() - t0
        o.close()
    finally:
        O.set_threads(1)
    return q["n_particles"] * steps / dt, dt, used


def cpu_baseline(args) -> dict:
    """The oracle as it stands on the host cores: threaded over independent
    cells and particles on every core (the same bits as one thread), and
    single-threaded on a smaller sample."""
    cores = host_cores()
    q, sample = oracle_sample_params(args, args.cpu_mesh)
    rate, dt, used = run_oracle_steps(q, args.cpu_steps, 0, cores)
    q1, sample1 = oracle_sample_params(args, args.cpu_mesh_1thread)
    rate1, dt1, _ = run_oracle_steps(q1, 1, 0, 1)
    return {"value": rate, "unit": UNIT, "cores": used, "host_cores": cores, "kind": "oracle",
            "sample": sample + f", {used} threads, {args.cpu_steps} step(s), {dt:.1f} s",
            "value_1thread": rate1, "sample_1thread": sample1 + f", 1 thread, 1 step, {dt1:.1f} s"}


def run_reference(args, rank: int) -> dict | None:
    if rank != 0:
        return None
    cores = host_cores()
    q, sample = oracle_sample_params(args, args.cpu_mesh)
    rate, dt, used = run_oracle_steps(q, args.steps, args.warmup, cores)
    sample += f", {used} threads"
    return {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1000 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic manufactured-solution workload",
        "config": {"workload": describe(args.workload, workload(args.workload)), "sample": sample},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": used, "host_cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="precision")
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-beside", action="store_true")
    ap.add_argument("--cpu-mesh", type=int, default=24)
    ap.add_argument("--cpu-mesh-1thread", type=int, default=12)
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    if world > 1 and args.impl != "reference":
        import torch.distributed as td

        td.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, rank)
        if out:
            print(json.dumps(out), flush=True)
        return
    import __graft_entry__ as g

    if rank == 0:
        g.build()
    if world > 1:
        import torch.distributed as td

        td.barrier()
    if args.workload == "adjoint":
        if rank == 0:
            print(json.dumps(run_adjoint(args)), flush=True)
        return
    if args.workload.startswith("batched"):
        out = run_batched(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        if world > 1:
            import torch.distributed as td

            td.destroy_process_group()
        return
    out = run_gpu(args, rank, world, args.form)
    beside = None
    if args.form == "mixed" and not args.no_fp64_beside:
        beside = run_gpu(args, rank, world, "fp64", with_e2e=False)
    if out is not None:
        if beside is not None:
            out["fp64_beside"] = beside
            out["speedup_vs_fp64"] = out["value"] / beside["value"]
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as td

        td.destroy_process_group()


if __name__ == "__main__":
    main()
