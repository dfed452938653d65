"""Benchmark: symmetric HSS compress + factor + solve on one B300 (replicas for N > 1).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload star16k|batch64]

Workload (default): star r(theta) = 1 + 0.3 cos(5 theta), 16384 Nystrom nodes (32768 complex128
unknowns), k_ext = 20, k_int = 30, eps0 = 1, eps1 = (k_int/k_ext)^2, leaf 128, ID tolerance 1e-10,
rings of at least 64 proxy points at 1.5x the box radius, plane wave at angle 0.
A step is one full compress + factor + right-hand side + solve of that scatterer through the
C ABI, with the curve already resident on the device.  The symmetric single-ID solver is the
headline; the non-symmetric two-ID baseline is timed on the same GPU and inputs.

--workload batch64: 64 independent random star scatterers r = 1 + sum_{m=2..8} a_m cos(m theta + phi_m),
a_m ~ U(0, 0.05), node counts log-uniform in [2048, 32768] (664375 nodes in total), k_ext ~ U(5, 40),
k_int / k_ext ~ U(1.2, 2), solved together in one handle (one launch per kernel and tree height);
a step is the whole batch.

Metric: seconds per scatterer (compress + factor + solve); for N GPUs every rank solves its own
copy of the workload (replicas, weak scaling) and value = max-over-ranks seconds per step / N.
L2: flushed between timed steps by writing a 512 MiB buffer outside the timed events.

--impl reference times the FP64 CPU oracle on this host (bounded sample, see cpu_baseline).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HSS compress+factor+solve sec, sym vs non-sym, rel err ≤1e-8; % roofline"
FP64_PEAK_TFLOPS = 1.25   # nominal dense FP64 of a B300 (148 SMs at up to 2032 MHz)


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _is_batch(name):
    from synth.curves import BATCH_WORKLOADS
    return name in BATCH_WORKLOADS


def _workload(name):
    from synth.curves import batch_workload, workload
    return batch_workload(name) if _is_batch(name) else workload(name)


def _config(w, mode):
    if "problems" in w:
        P = w["problems"]
        ns = [p["curve"].n for p in P]
        k0 = [p["k0"] for p in P]
        return {"workload": f"{w['name']}: {len(P)} random star scatterers in one batch, N={sum(ns)} nodes in "
                            f"total ({min(ns)}..{max(ns)} per scatterer), k_ext in [{min(k0):.1f}, {max(k0):.1f}], "
                            f"k_int/k_ext in [1.2, 2], eps1=(k_int/k_ext)^2, leaf {w['leaf']}, ID tol {w['tol']:g}, "
                            f">= {w['nproxy']}-point proxy rings at 1.5x box radius",
                "mode": mode, "l2": "inputs larger than L2 (tens of GB of tiles per step); 512 MiB flush too",
                "parallelism": "replicas (one batch per GPU)"}
    c = w["curve"]
    return {"workload": f"{w['name']}: {c.name} curve, N={c.n} nodes ({2 * c.n} complex128 unknowns), "
                        f"k_ext={w['k0']:g}, k_int={w['k1']:g}, eps1=(k_int/k_ext)^2, leaf {w['leaf']}, "
                        f"ID tol {w['tol']:g}, >= {w['nproxy']}-point proxy rings at 1.5x box radius",
            "mode": mode, "l2": "flushed between timed steps (512 MiB write outside the timed events)",
            "parallelism": "replicas (one scatterer per GPU)"}


# ----------------------------------------------------------------------------------- ours

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2609_33216_b300 import symhss as S
    from paper_2609_33216_b300.solver import BatchSolver, Solver

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    w = _workload(args.workload)
    batch = "problems" in w
    curves = [p["curve"] for p in w["problems"]] if batch else [w["curve"]]
    n_total = sum(cv.n for cv in curves)
    kw = dict(leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"])
    if args.precision == "mixed":
        kw["precision"] = S.SYMHSS_MIXED

    net, prop_info = None, None
    if args.proposer:  # train the rank proposer first (outside every timed region)
        from paper_2609_33216_b300.proposer import train_default
        t_train = time.perf_counter()
        net = train_default(seed=0, steps=3000)
        prop_info = {"train_s": time.perf_counter() - t_train, "samples": int(net.data_size), "margin": 1.3,
                     "training_data": "plain IDs of disk512, star16k, star64k (k 40/60 and 80/120) and 6 random "
                                      "stars (k 5..60) at tol 1e-10 and 1e-8"}

    def make(mode):
        if batch:
            P = w["problems"]
            sv = BatchSolver(curves, [p["k0"] for p in P], [p["k1"] for p in P], [p["eps0"] for p in P],
                             [p["eps1"] for p in P], mode=mode, **kw)
        else:
            kws = dict(kw)
            if "precision" in kws:
                kws["precision"] = "mixed"
            sv = Solver(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], mode=mode, curve_on_device=True, **kws)
        if net is not None:
            net.attach(sv, margin=1.3)
        return sv

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(s):
        if args.pipeline:  # compression of height t + 1 overlaps factorisation of height t
            s.build()
        else:
            s.compress()
            s.factor()
        return s.solve(s.rhs(0.0))

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    results = {}
    solvers = {}
    tunings = {}
    for mode in ("base", "sym"):  # the symmetric handle stays alive for the end-to-end leg
        s = make(mode)
        solvers[mode] = s
        if args.autotune:  # launch shapes chosen by the library's autotuner, outside the timed region
            t_at = time.perf_counter()
            tn = S.symhss_autotune(s.h, reps=2, stream=stream.cuda_stream)
            tunings[mode] = dict(tn.as_dict(), seconds=time.perf_counter() - t_at)
        for _ in range(args.warmup):
            x = step(s)
        barrier()
        sampler = ClockSampler(local) if (mode == "sym" and rank == 0) else None
        if sampler:
            sampler.start()
        times = []
        launches0 = S.lib.symhss_launch_count()
        kms = [0.0] * 8
        kwork = [0.0] * 8
        klaunch = [0] * 8
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x = step(s)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            st = s.stats()
            for k in range(8):
                kms[k] += st.kernel_ms[k]
                kwork[k] += st.kernel_work[k]
                klaunch[k] += st.kernel_launches[k]
        barrier()
        launches = S.lib.symhss_launch_count() - launches0
        clocks = sampler.stop() if sampler else None
        tot = torch.tensor([sum(times)], device="cuda", dtype=torch.float64)
        if world > 1:
            dist.all_reduce(tot, op=dist.ReduceOp.MAX)
        st = s.stats()
        results[mode] = dict(ms_total=float(tot.item()), times=times, x=x.cpu().numpy(), stats=st, clocks=clocks,
                             launches=launches, kms=kms, kwork=kwork, klaunch=klaunch)
        del x
        if mode == "base":
            s.close()
            torch.cuda.empty_cache()

    # comparator: the symmetric PMCHWT system (first-order accurate) on the same solver
    comparators = {}
    if not batch and args.comparators:
        pm = Solver(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], mode="sym", curve_on_device=True,
                    formulation="pmchwt", **kw)
        if "sym" in tunings:  # the symmetric solver's launch tuning
            S.symhss_set_tuning(pm.h, **{k: v for k, v in tunings["sym"].items() if k != "seconds"})
        for _ in range(args.warmup):
            step(pm)
        barrier()
        tms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(pm)
            e1.record(stream)
            e1.synchronize()
            tms.append(e0.elapsed_time(e1))
        stp = pm.stats()
        comparators["pmchwt_sym"] = {"ms_per_step": sum(tms) / len(tms), "max_rank": list(stp.max_rank),
                                     "root_size": stp.root_size,
                                     "accuracy": "first order in h (O(h^3) for the Muller-like system)"}
        pm.close()
        bm = Solver(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], mode="base", curve_on_device=True,
                    formulation="bm", **kw)
        if "base" in tunings:
            S.symhss_set_tuning(bm.h, **{k: v for k, v in tunings["base"].items() if k != "seconds"})
        for _ in range(args.warmup):
            step(bm)
        barrier()
        tms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(bm)
            e1.record(stream)
            e1.synchronize()
            tms.append(e0.elapsed_time(e1))
        stb = bm.stats()
        comparators["burton_miller_nonsym"] = {"ms_per_step": sum(tms) / len(tms), "max_rank": list(stb.max_rank),
                                               "root_size": stb.root_size,
                                               "accuracy": "first order in h (hypersingular N_k0)"}
        bm.close()

    mixed_diff = None
    if args.precision == "mixed" and not batch:
        ref = Solver(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], mode="sym", curve_on_device=True,
                     leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"])
        xr = step(ref).cpu().numpy()
        ref.close()
        for md in ("sym", "base"):
            xm = results[md]["x"]
            results[md]["vs_fp64"] = float(np.linalg.norm(xm - xr) / np.linalg.norm(xr))
        mixed_diff = {"sym_vs_fp64_sym": results["sym"]["vs_fp64"], "base_vs_fp64_sym": results["base"]["vs_fp64"],
                      "refinement_steps": 2}

    xs = results["sym"]["x"]
    xb = results["base"]["x"]
    if batch:  # largest per-scatterer relative difference
        e2e_tmp = solvers["sym"]
        rel_diff = max(float(np.linalg.norm(xs[r:r + 2 * n] - xb[r:r + 2 * n]) / np.linalg.norm(xb[r:r + 2 * n]))
                       for r, n in zip(e2e_tmp.row0, e2e_tmp.ns))
    else:
        rel_diff = float(np.linalg.norm(xs - xb) / np.linalg.norm(xb))

    # end to end through the C ABI: host curves in, host solution out, every step
    e2e_s = solvers["sym"]
    host = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in cv.arrays()] for cv in curves]
    xh = torch.empty(2 * n_total, dtype=torch.complex128).pin_memory()
    curve_structs = [S.curve_struct(cv.n, [t.data_ptr() for t in hs], S.SYMHSS_HOST) for cv, hs in zip(curves, host)]

    def e2e_step():
        S.symhss_set_curves(e2e_s.h, curve_structs, stream.cuda_stream)
        x = step(e2e_s)
        xh.copy_(x, non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(max(1, args.warmup)):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_sec = (time.perf_counter() - t0) / args.steps
    e2e_t = torch.tensor([e2e_sec], device="cuda", dtype=torch.float64)
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_sec = float(e2e_t.item())

    if rank == 0:
        r = results["sym"]
        sec_sym = r["ms_total"] / args.steps / 1000.0
        sec_base = results["base"]["ms_total"] / args.steps / 1000.0
        names = S.K_NAMES
        nk = len(names)
        per_kernel = {names[k]: {"ms_per_step": r["kms"][k] / args.steps, "launches_per_step": r["klaunch"][k] / args.steps,
                                 "work_per_step": r["kwork"][k] / args.steps} for k in range(nk)}
        # dominant kernel class by device time
        dom = max(range(nk), key=lambda k: r["kms"][k])
        roof = None
        if dom == S.K_SKETCH and r["kms"][dom] > 0:
            peaks = _measured_peaks()
            achieved = r["kwork"][dom] / (r["kms"][dom] * 1e-3) / 1e12
            pk = peaks.get("bf16_tflops")
            roof = {"kernel": names[dom], "bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                    "frac": achieved / pk if pk else None, "traffic": None, "peak_source": "measured bf16"}
        elif r["kms"][dom] > 0 and r["kwork"][dom] > 0 and dom != 0:
            achieved = r["kwork"][dom] / (r["kms"][dom] * 1e-3) / 1e12
            roof = {"kernel": names[dom], "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                    "peak_source": "nominal FP64 of the B300 (derived: not in the measured-peaks file)",
                    "avg_launch_ms": r["kms"][dom] / max(1, r["klaunch"][dom])}
        elif r["kms"][dom] > 0:
            roof = {"kernel": names[dom], "bound": "alu", "achieved": r["kwork"][dom] / (r["kms"][dom] * 1e-3),
                    "peak": None, "unit": "pairs/s", "frac": None, "traffic": None}
        st = r["stats"]
        out = {
            "metric": METRIC, "value": sec_sym / world, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec_sym * 1000.0, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "complex128 (f64)" if args.precision == "fp64" else "complex128 compression, complex64 factorisation, f64 refinement",
            "data": "synthetic",
            "config": _config(w, "sym"),
            "nonsym": {"value": sec_base / world, "unit": "s", "ms_per_step": sec_base * 1000.0},
            "speedup_sym_vs_nonsym": sec_base / sec_sym,
            "rel_diff_sym_vs_nonsym": rel_diff,
            "phases_ms": ({"build": st.ms_build, "solve": st.ms_solve} if args.pipeline else
                          {"compress": st.ms_compress, "factor": st.ms_factor, "solve": st.ms_solve}),
            "per_kernel": per_kernel,
            "proposer": prop_info,
            "comparators": comparators or None,
            "mixed_precision": mixed_diff,
            "tuning": tunings or None,
            "id_checks": {"failed_then_continued": int(st.check_failed), "max_accepted_ratio": st.check_max_ratio,
                          "proposals": int(st.proposals), "proposal_rank_err": st.proposal_rank_err},
            "sketch": {"redone_ids": int(st.sketch_redo),
                       "tensor_tflops": (r["kwork"][S.K_SKETCH] / (r["kms"][S.K_SKETCH] * 1e-3) / 1e12
                                         if r["kms"][S.K_SKETCH] > 0 else None)},
            "ranks": {"max_flux": st.max_rank[0], "max_trace": st.max_rank[1], "root_size": st.root_size,
                      "leaf_mean": [st.level_mean_rank[st.depth][0], st.level_mean_rank[st.depth][1]]},
            "roofline": roof,
            "e2e": {"value": e2e_sec / world, "unit": "s", "h2d_bytes_per_step": 6 * 8 * n_total,
                    "d2h_bytes_per_step": 16 * 2 * n_total},
            "gpu_launches": int(r["launches"]),
            "clocks": r["clocks"],
        }
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w, args.cpu_sample_boxes)
        print(json.dumps(out), flush=True)
    solvers["sym"].close()
    if world > 1:
        dist.destroy_process_group()


def run_profile(args):
    """One warm-up and one symmetric step of the workload, nothing else (for ncu captures)."""
    import torch

    from paper_2609_33216_b300.solver import Solver

    torch.cuda.set_device(0)
    w = _workload(args.workload)
    s = Solver(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], mode="sym", curve_on_device=True,
               leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"])
    for _ in range(2):
        s.compress()
        s.factor()
        x = s.solve(s.rhs(0.0))
    torch.cuda.synchronize()
    st = s.stats()
    print(json.dumps({"profile": w["name"], "ms_compress": st.ms_compress, "ms_factor": st.ms_factor,
                      "ms_solve": st.ms_solve, "x0": [float(x[0].real), float(x[0].imag)]}), flush=True)
    s.close()


# ----------------------------------------------------------------------------- CPU oracle

def _oracle_leaf_sample(curve, k0, k1, eps0, eps1, w, sample_boxes: int):
    """Oracle leaf-level compress + factor of `sample_boxes` leaf boxes of one scatterer:
    (seconds, boxes sampled, leaf boxes of the scatterer)."""
    import numpy as np
    import scipy.linalg as sla

    from oracle.hss import HSS, Options, cpqr_id
    from oracle.kernels import Params

    prm = Params(k0, k1, eps0, eps1)
    solver = HSS(curve, prm, Options(leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"]))
    lev = solver.levels[-1]
    for b in lev:
        ids = np.arange(b.begin, b.end)
        b.act = [ids, ids]
        b.actrow = [ids, ids]
    idx = np.linspace(0, len(lev) - 1, min(sample_boxes, len(lev))).astype(int)
    t0 = time.perf_counter()
    for i in idx:
        b = lev[i]
        mr = solver.m_r(b, lev)
        n0 = len(b.act[0])
        b.rank, b.perm, b.T = [], [], []
        for half in (mr[:, :n0], mr[:, n0:]):
            r, p, t = cpqr_id(half, w["tol"])
            b.rank.append(r)
            b.perm.append(p)
            b.T.append(t)
        b.rrank, b.rperm, b.rT = b.rank, b.perm, b.T
        d = solver._diag_block(b, solver.depth)
        lu = sla.lu_factor(d)
        rt = solver._basis(b, solver.depth, row=False)
        x = sla.lu_solve(lu, rt)
        np.linalg.inv(rt.T @ x)
    return time.perf_counter() - t0, len(idx), len(lev)


def cpu_baseline(w, sample_boxes: int):
    """Time the FP64 oracle on a bounded sample of the workload and scale it to the whole job.

    Sample: the leaf level of the oracle's compression and factorisation (M_R tiles, two column
    IDs, diagonal-block LU, X = D^-1 R^T and Atilde) for `sample_boxes` of the leaf boxes; the
    per-box time is multiplied by the number of leaf boxes (of every scatterer of a batch: the
    sampled boxes are then spread over up to 4 scatterers).  Upper levels are not included, so
    the value is a lower bound of the oracle's whole-job time.
    """
    import math as _m

    if "problems" in w:
        P = w["problems"]
        total_leaves = sum(2 ** max(0, _m.ceil(_m.log2(p["curve"].n / w["leaf"]))) if p["curve"].n > w["leaf"] else 1
                           for p in P)
        picks = sorted(set(int(round(v)) for v in
                           [i * (len(P) - 1) / max(1, min(4, len(P)) - 1) for i in range(min(4, len(P)))]))
        per = max(1, sample_boxes // len(picks))
        dt, cnt = 0.0, 0
        for i in picks:
            p = P[i]
            d, c, _ = _oracle_leaf_sample(p["curve"], p["k0"], p["k1"], p["eps0"], p["eps1"], w, per)
            dt += d
            cnt += c
        nlev, what = total_leaves, f"{cnt} leaf boxes of {len(picks)} of the {len(P)} scatterers"
    else:
        dt, cnt, nlev = _oracle_leaf_sample(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], w, sample_boxes)
        what = f"{cnt} of {nlev} leaf boxes"
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": dt / cnt * nlev, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": f"leaf level only: compress+factor of {what} ({dt:.1f} s), scaled to all {nlev} leaf boxes; "
                      f"numpy/scipy FP64, BLAS threads = host cores"}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    w = _workload(args.workload)
    for _ in range(args.warmup):
        cpu_baseline(w, args.ref_sample_boxes)
    vals = []
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(w, args.ref_sample_boxes)
        vals.append(last["value"])
    v = sum(vals) / len(vals)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v * 1000.0, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "complex128 (f64)", "data": "synthetic", "config": _config(w, "sym"),
           "cpu_baseline": dict(last, value=v),
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="star16k")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-boxes", type=int, default=16)
    ap.add_argument("--ref-sample-boxes", type=int, default=4)
    ap.add_argument("--profile", action="store_true", help="one warm-up + one symmetric step only")
    ap.add_argument("--proposer", action="store_true", help="train the learned rank proposer and attach it")
    ap.add_argument("--comparators", type=int, default=1, help="also time the symmetric PMCHWT comparator")
    ap.add_argument("--pipeline", type=int, default=1,
                    help="compress and factor through the pipelined build call (two streams)")
    ap.add_argument("--autotune", type=int, default=1, help="run the library's launch autotuner before timing")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="mixed: complex64 factorisation + iterative refinement (two steps) against the FP64 operator")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
