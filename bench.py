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
The timed steps use the pipelined build (compression of height t + 1 on a second stream while
height t is factorised), so per-kernel-class events overlap there; per_kernel and the roofline come
from up to 5 further serialised steps (compress, factor, solve on one stream) of the same handle.
At one GPU the default run also times the other configurations (extra_workloads): the 65536-node
star in mixed precision, the 64-scatterer batch and the 262144-node star with the learned proposer.

cpu_baseline: the FP64 oracle's whole job on the workload, run once on this host's cores.
--impl reference: the same oracle job as the reference arm, one whole job per step, as many steps
as fit in --ref-budget-s (the JSON line reports the steps actually run).
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

def fp64_peak_tflops(sm_mhz):
    """FP64 peak of this device: SMs x 4 FP64 flops per clock (two DFMA per SM per cycle, the
    rate ncu reports for this part) x the SM clock sampled while the timed steps ran."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_mhz or 2032.0
    return sms * 4.0 * mhz * 1e6 / 1e12, sms, mhz


# DRAM bytes of a kernel class on the star16k workload, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum over every launch of the class in the second step of `bench.py --profile`,
# cold cache per launch, so upper bounds); per class call ("launch" of the library's class timing)
# and per step.  A class whose kernels change after the capture must lose its entry (its traffic is
# then reported as null).
NCU_TRAFFIC = {
    "getrf": {"bytes_per_launch": 1728.7e6 / 15, "bytes_per_step": 1728.7e6,
              "capture": "profiles/star16k_launch_list.md (DRAM table)"},
    "getrs": {"bytes_per_launch": 3215.5e6 / 22, "bytes_per_step": 3215.5e6,
              "capture": "profiles/star16k_launch_list.md (DRAM table)"},
    "id": {"bytes_per_launch": 68.8e6 / 8, "bytes_per_step": 68.8e6,
           "capture": "profiles/star16k_launch_list.md (DRAM table)"},
}


class _Timer:
    def __init__(self, stream):
        import torch
        self.stream = stream
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)

    def __enter__(self):
        self.e0.record(self.stream)
        return self

    def __exit__(self, *exc):
        self.e1.record(self.stream)
        self.e1.synchronize()
        self.ms = self.e0.elapsed_time(self.e1)


def _class_accumulate(acc, st):
    for k in range(8):
        acc["ms"][k] += st.kernel_ms[k]
        acc["work"][k] += st.kernel_work[k]
        acc["launch"][k] += st.kernel_launches[k]


def _new_acc():
    return {"ms": [0.0] * 8, "work": [0.0] * 8, "launch": [0] * 8}


def bench_workload(w, args, steps, warmup, precision="fp64", net=None, autotune=True, sample_clocks=False,
                   serial_pass=0, world=1):
    """Time the symmetric and the two-ID solver on workload `w`: `warmup` untimed and `steps` timed
    steps each (CUDA events on the caller's stream, L2 flushed between steps).  Returns per mode the
    total ms, the solution, stats, launches and per-class device time of the timed (pipelined) steps,
    and, if serial_pass > 0, per-class device time of that many serialised steps of the symmetric
    solver (compress then factor on one stream, so class events do not overlap)."""
    import torch
    import torch.distributed as dist

    from paper_2609_33216_b300 import symhss as S
    from paper_2609_33216_b300.solver import BatchSolver, Solver

    batch = "problems" in w
    curves = [p["curve"] for p in w["problems"]] if batch else [w["curve"]]
    kw = dict(leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"])

    def make(mode):
        if batch:
            P = w["problems"]
            sv = BatchSolver(curves, [p["k0"] for p in P], [p["k1"] for p in P], [p["eps0"] for p in P],
                             [p["eps1"] for p in P], mode=mode, precision=S.SYMHSS_MIXED if precision == "mixed"
                             else S.SYMHSS_FP64, **kw)
        else:
            sv = Solver(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], mode=mode, curve_on_device=True,
                        precision=precision, **kw)
        if net is not None:
            net.attach(sv, margin=1.3)
        return sv

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(s, pipelined=True):
        if pipelined:  # compression of height t + 1 overlaps factorisation of height t
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

    out = {"solvers": {}, "tuning": {}}
    for mode in ("base", "sym"):
        s = make(mode)
        if autotune:  # launch shapes chosen by the library's autotuner, outside the timed region
            t_at = time.perf_counter()
            tn = S.symhss_autotune(s.h, reps=2, stream=stream.cuda_stream)
            out["tuning"][mode] = dict(tn.as_dict(), seconds=time.perf_counter() - t_at)
        # the clock sampler (an nvidia-smi process polling every 200 ms) starts before the warm-up
        # steps: its start-up competes for the host cores that enqueue the pipelined build, and
        # inside the timed region it stalled the first timed step by about 20 ms
        sampler = ClockSampler(torch.cuda.current_device()) if (mode == "sym" and sample_clocks) else None
        if sampler:
            sampler.start()
        for _ in range(warmup):
            x = step(s)
        barrier()
        times = []
        launches0 = S.lib.symhss_launch_count()
        acc = _new_acc()
        for _ in range(steps):
            flush.fill_(1.0)
            with _Timer(stream) as tm:
                x = step(s)
            times.append(tm.ms)
            _class_accumulate(acc, s.stats())
        barrier()
        launches = S.lib.symhss_launch_count() - launches0
        clocks = sampler.stop() if sampler else None
        tot = torch.tensor([sum(times)], device="cuda", dtype=torch.float64)
        if world > 1:
            dist.all_reduce(tot, op=dist.ReduceOp.MAX)
        r = dict(ms_total=float(tot.item()), times=times, x=x.cpu().numpy(), stats=s.stats(), clocks=clocks,
                 launches=launches, acc=acc)
        del x
        if mode == "sym" and serial_pass > 0:
            ser = _new_acc()
            ser_ms = []
            for _ in range(serial_pass):
                flush.fill_(1.0)
                with _Timer(stream) as tm:
                    step(s, pipelined=False)
                ser_ms.append(tm.ms)
                _class_accumulate(ser, s.stats())
            r["serial"] = dict(acc=ser, steps=serial_pass, ms=ser_ms)
        out[mode] = r
        if mode == "base":
            s.close()
            torch.cuda.empty_cache()
        else:
            out["solvers"]["sym"] = s
    del flush
    xs, xb = out["sym"]["x"], out["base"]["x"]
    import numpy as np
    if batch:  # largest per-scatterer relative difference
        sv = out["solvers"]["sym"]
        out["rel_diff"] = max(float(np.linalg.norm(xs[r:r + 2 * n] - xb[r:r + 2 * n]) / np.linalg.norm(xb[r:r + 2 * n]))
                              for r, n in zip(sv.row0, sv.ns))
    else:
        out["rel_diff"] = float(np.linalg.norm(xs - xb) / np.linalg.norm(xb))
    out["step"] = step
    return out


def _per_kernel(acc, steps, names):
    return {names[k]: {"ms_per_step": acc["ms"][k] / steps, "launches_per_step": acc["launch"][k] / steps,
                       "work_per_step": acc["work"][k] / steps} for k in range(len(names))}


def _roofline(acc, steps, names, sm_mhz, K_SKETCH):
    """Roofline of the dominant kernel class (largest serialised device time) with algorithmic work."""
    nk = len(names)
    cand = [k for k in range(nk) if acc["ms"][k] > 0 and acc["work"][k] > 0 and names[k] != "tiles"]
    if not cand:
        return None
    dom = max(cand, key=lambda k: acc["ms"][k])
    ms_launch = acc["ms"][dom] / max(1, acc["launch"][dom])
    work_launch = acc["work"][dom] / max(1, acc["launch"][dom])
    achieved = acc["work"][dom] / (acc["ms"][dom] * 1e-3) / 1e12
    tr = NCU_TRAFFIC.get(names[dom])
    if dom == K_SKETCH:
        pk = _measured_peaks().get("bf16_tflops")
        roof = {"kernel": names[dom], "bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                "frac": achieved / pk if pk else None, "peak_source": "measured bf16 (MEASURED_PEAKS.json)"}
    else:
        pk, sms, mhz = fp64_peak_tflops(sm_mhz)
        roof = {"kernel": names[dom], "bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                "frac": achieved / pk,
                "peak_source": f"derived FP64: {sms} SMs x 4 flop/clk x {mhz:.0f} MHz (median sampled SM clock)"}
    roof["traffic"] = tr["bytes_per_launch"] if tr else None
    if tr:
        roof["traffic_source"] = tr["capture"]
    roof["timing"] = ("serialised steps (compress then factor on one stream): CUDA events around every launch "
                      "of the class on the stream it runs on")
    roof["avg_launch_ms"] = ms_launch
    roof["work_per_launch"] = work_launch
    return roof


def _hbm(acc, steps, names):
    """Achieved HBM bandwidth of the column ID (c) and the block LU and solves (d): DRAM bytes per step
    from the ncu capture in NCU_TRAFFIC over the class's serialised device time per step."""
    peak = _measured_peaks().get("hbm_gbs")
    out = {}
    for cls in ("id", "getrf", "getrs"):
        k = names.index(cls)
        tr = NCU_TRAFFIC.get(cls)
        if not tr or acc["ms"][k] <= 0:
            continue
        gbs = tr["bytes_per_step"] / (acc["ms"][k] / steps * 1e-3) / 1e9
        out[cls] = {"GB_per_s": gbs, "frac_of_measured_hbm": gbs / peak if peak else None,
                    "dram_bytes_per_step": tr["bytes_per_step"]}
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2609_33216_b300 import symhss as S

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    w = _workload(args.workload)
    batch = "problems" in w
    curves = [p["curve"] for p in w["problems"]] if batch else [w["curve"]]
    n_total = sum(cv.n for cv in curves)
    stream = torch.cuda.current_stream()

    net, prop_info = None, None
    if args.proposer:  # train the rank proposer first (outside every timed region)
        net, prop_info = _train_proposer()

    res = bench_workload(w, args, args.steps, args.warmup, precision=args.precision, net=net,
                         autotune=bool(args.autotune), sample_clocks=(rank == 0),
                         serial_pass=min(args.steps, 5), world=world)
    step = res["step"]
    r = res["sym"]
    names = S.K_NAMES

    # comparators: the symmetric PMCHWT and the Burton-Miller systems on the same solver
    comparators = {}
    if not batch and args.comparators:
        comparators = _comparators(w, args, res["tuning"], step, world)

    mixed_diff = None
    if args.precision == "mixed" and not batch:
        mixed_diff = _mixed_vs_fp64(w, res, step)

    # end to end through the C ABI: host curves in, host solution out, every step
    e2e_s = res["solvers"]["sym"]
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
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e2e_sec = (time.perf_counter() - t0) / args.steps
    e2e_t = torch.tensor([e2e_sec], device="cuda", dtype=torch.float64)
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_sec = float(e2e_t.item())
    e2e_s.close()
    del res["solvers"]
    torch.cuda.empty_cache()

    extras = None
    if world == 1 and args.extras and args.workload == "star16k":
        extras = _extra_workloads(args)

    if rank == 0:
        sec_sym = r["ms_total"] / args.steps / 1000.0
        sec_base = res["base"]["ms_total"] / args.steps / 1000.0
        st = r["stats"]
        clocks = r["clocks"] or {}
        ser = r["serial"]
        out = {
            "metric": METRIC, "value": sec_sym / world, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec_sym * 1000.0, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "complex128 (f64)" if args.precision == "fp64" else "complex128 compression, complex64 factorisation, f64 refinement",
            "data": "synthetic",
            "config": _config(w, "sym"),
            "nonsym": {"value": sec_base / world, "unit": "s", "ms_per_step": sec_base * 1000.0},
            "speedup_sym_vs_nonsym": sec_base / sec_sym,
            "rel_diff_sym_vs_nonsym": res["rel_diff"],
            "phases_ms": {"build": st.ms_build, "solve": st.ms_solve},
            "step_ms": {"median": statistics.median(r["times"]), "min": min(r["times"]), "max": max(r["times"])},
            "per_kernel": _per_kernel(ser["acc"], ser["steps"], names),
            "per_kernel_timing": ("serialised steps (compress, then factor, then solve, one stream), CUDA events "
                                  f"around every launch; {ser['steps']} steps of "
                                  f"{statistics.median(ser['ms']):.1f} ms (median) against "
                                  f"{sec_sym * 1000.0:.1f} ms for the pipelined timed step"),
            "proposer": prop_info,
            "comparators": comparators or None,
            "mixed_precision": mixed_diff,
            "tuning": res["tuning"] or None,
            "id_checks": {"failed_then_continued": int(st.check_failed), "max_accepted_ratio": st.check_max_ratio,
                          "proposals": int(st.proposals), "proposal_rank_err": st.proposal_rank_err},
            "sketch": {"redone_ids": int(st.sketch_redo)},
            "ranks": {"max_flux": st.max_rank[0], "max_trace": st.max_rank[1], "root_size": st.root_size,
                      "leaf_mean": [st.level_mean_rank[st.depth][0], st.level_mean_rank[st.depth][1]]},
            "roofline": _roofline(ser["acc"], ser["steps"], names, clocks.get("sm_mhz"), S.K_SKETCH)
            if args.workload == "star16k" else None,
            "hbm": _hbm(ser["acc"], ser["steps"], names) if args.workload == "star16k" else None,
            "e2e": {"value": e2e_sec / world, "unit": "s", "h2d_bytes_per_step": 6 * 8 * n_total,
                    "d2h_bytes_per_step": 16 * 2 * n_total},
            "gpu_launches": int(r["launches"]),
            "clocks": r["clocks"],
        }
        if extras:
            out["extra_workloads"] = extras
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline(w, args.cpu_budget_s)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _train_proposer():
    from paper_2609_33216_b300.proposer import train_default
    t_train = time.perf_counter()
    net = train_default(seed=0, steps=3000)
    info = {"train_s": time.perf_counter() - t_train, "samples": int(net.data_size), "margin": 1.3,
            "training_data": "plain IDs of disk512, star16k, star64k (k 40/60 and 80/120) and 6 random "
                             "stars (k 5..60) at tol 1e-10 and 1e-8"}
    return net, info


def _comparators(w, args, tunings, step, world):
    import torch

    from paper_2609_33216_b300 import symhss as S
    from paper_2609_33216_b300.solver import Solver

    kw = dict(leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"])
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    out = {}
    for key, form, mode, acc in (("pmchwt_sym", "pmchwt", "sym", "first order in h (O(h^3) for the Muller-like system)"),
                                 ("burton_miller_nonsym", "bm", "base", "first order in h (hypersingular N_k0)")):
        sv = Solver(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], mode=mode, curve_on_device=True,
                    formulation=form, **kw)
        if mode in tunings:
            S.symhss_set_tuning(sv.h, **{k: v for k, v in tunings[mode].items() if k != "seconds"})
        for _ in range(args.warmup):
            step(sv)
        torch.cuda.synchronize()
        tms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            with _Timer(stream) as tm:
                step(sv)
            tms.append(tm.ms)
        st = sv.stats()
        out[key] = {"ms_per_step": sum(tms) / len(tms), "max_rank": list(st.max_rank), "root_size": st.root_size,
                    "accuracy": acc}
        sv.close()
    return out


def _mixed_vs_fp64(w, res, step):
    """Relative differences of the mixed-precision solutions (after the default two refinement
    steps, and with none) from the FP64 symmetric solution of the same workload."""
    import numpy as np

    from paper_2609_33216_b300.solver import Solver
    ref = Solver(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], mode="sym", curve_on_device=True,
                 leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"])
    xr = step(ref).cpu().numpy()
    ref.close()
    out = {}
    for md in ("sym", "base"):
        out[f"{md}_vs_fp64_sym"] = float(np.linalg.norm(res[md]["x"] - xr) / np.linalg.norm(xr))
    sv = res["solvers"]["sym"]
    sv.set_refinement(0)
    x0 = sv.solve(sv.rhs(0.0)).cpu().numpy()
    sv.set_refinement(2)
    out["sym_vs_fp64_sym_before_refinement"] = float(np.linalg.norm(x0 - xr) / np.linalg.norm(xr))
    out["refinement_steps"] = 2
    return out


def _fixed_rank_sweep(sizes=(4096, 8192, 16384, 32768, 65536, 131072, 262144), steps=3, warmup=2):
    """The fixed-rank schedule k_l = ceil(1.15^(L - l) 30) (Sec. 4.3) on the star r = 1 + 0.3 cos 5t
    with k 20/30, leaf 128, for N = 4096 .. 262144: device ms of build + solve per step (CUDA
    events, median of `steps`), and ms per 1000 nodes (flat for the linear complexity of
    Theorem `order`, which holds for a < 2^(1/3))."""
    import torch

    from paper_2609_33216_b300.solver import Solver
    from synth import star

    stream = torch.cuda.current_stream()
    rows = []
    for n in sizes:
        sv = Solver(star(n), 20.0, 30.0, mode="sym", curve_on_device=True, leaf=128, nproxy=64, tol=1e-10,
                    fixed_rank_kL=30, rank_scale_a=1.15)
        for _ in range(warmup):
            sv.build()
            sv.solve(sv.rhs(0.0))
        ms = []
        for _ in range(steps):
            with _Timer(stream) as tm:
                sv.build()
                sv.solve(sv.rhs(0.0))
            ms.append(tm.ms)
        st = sv.stats()
        rows.append({"n": n, "ms": statistics.median(ms), "ms_per_1000_nodes": statistics.median(ms) / (n / 1000.0),
                     "root_size": st.root_size, "depth": st.depth})
        sv.close()
    return {"schedule": "k_l = ceil(1.15^(L-l) 30), symmetric, FP64, star r = 1 + 0.3 cos 5t, k 20/30, leaf 128",
            "rows": rows}


def _extra_workloads(args):
    """The other benchmark configurations, each timed with `args.extra_steps` steps after 3 warm-up
    steps (default launch tuning; no autotuner): the 65536-node star in mixed precision, the batch of
    64 random scatterers, and the 262144-node star with the learned rank proposer."""
    import torch

    from paper_2609_33216_b300 import symhss as S

    out = {"fixed_rank_sweep": _fixed_rank_sweep()}
    specs = [("star64k", "mixed", False), ("batch64", "fp64", False), ("star262k", "fp64", True)]
    for name, prec, proposer in specs:
        w = _workload(name)
        net, pinfo = (None, None)
        if proposer:
            net, pinfo = _train_proposer()
        res = bench_workload(w, args, args.extra_steps, 3, precision=prec, net=net, autotune=False,
                             sample_clocks=True, serial_pass=0)
        st = res["sym"]["stats"]
        sec_sym = res["sym"]["ms_total"] / args.extra_steps / 1000.0
        sec_base = res["base"]["ms_total"] / args.extra_steps / 1000.0
        d = {"config": _config(w, "sym"), "precision": prec, "value": sec_sym, "unit": "s",
             "steps": args.extra_steps, "warmup": 3, "nonsym": sec_base, "speedup_sym_vs_nonsym": sec_base / sec_sym,
             "rel_diff_sym_vs_nonsym": res["rel_diff"], "phases_ms": {"build": st.ms_build, "solve": st.ms_solve},
             "per_kernel_pipelined": _per_kernel(res["sym"]["acc"], args.extra_steps, S.K_NAMES),
             "ranks": {"max_flux": st.max_rank[0], "max_trace": st.max_rank[1], "root_size": st.root_size},
             "clocks": res["sym"]["clocks"]}
        if prec == "mixed":
            d["mixed_precision"] = _mixed_vs_fp64(w, res, res["step"])
        if proposer:
            d["proposer"] = pinfo
            d["id_checks"] = {"failed_then_continued": int(st.check_failed), "redone_ids": int(st.sketch_redo),
                              "proposals": int(st.proposals), "proposal_rank_err": st.proposal_rank_err}
        out[name] = d
        res["solvers"]["sym"].close()
        del res
        torch.cuda.empty_cache()
    return out


def run_profile(args):
    """One warm-up and one symmetric step of the workload, nothing else (for ncu captures)."""
    import torch

    from paper_2609_33216_b300.solver import Solver

    torch.cuda.set_device(0)
    w = _workload(args.workload)
    s = Solver(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], mode="sym", curve_on_device=True,
               leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"])
    from paper_2609_33216_b300 import symhss as S
    if args.lu_tc is not None:
        S.symhss_set_tuning(s.h, lu_tc=args.lu_tc)
    if args.lu_outer is not None:
        S.symhss_set_tuning(s.h, lu_outer=args.lu_outer)
    if args.panel_cluster is not None:
        S.symhss_set_tuning(s.h, lu_panel_cluster=args.panel_cluster)
    if args.lookahead is not None:
        S.symhss_set_tuning(s.h, lu_lookahead=args.lookahead)
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

def _oracle_job(curve, k0, k1, eps0, eps1, w):
    """The FP64 oracle's whole job for one scatterer: compress (proxy tiles and column IDs of every
    level), factor, right-hand side and solve.  Returns the seconds of each phase."""
    from oracle.hss import HSS, Options
    from oracle.kernels import Params, rhs

    prm = Params(k0, k1, eps0, eps1)
    t0 = time.perf_counter()
    solver = HSS(curve, prm, Options(leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"]))
    solver.compress()
    t1 = time.perf_counter()
    solver.factor()
    t2 = time.perf_counter()
    solver.solve(rhs(curve, prm))
    t3 = time.perf_counter()
    return {"compress": t1 - t0, "factor": t2 - t1, "solve": t3 - t2, "total": t3 - t0}


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def cpu_baseline(w, budget_s: float):
    """The FP64 oracle (numpy/scipy, BLAS threads = host cores) timed on this host.

    One scatterer: the whole compress + factor + solve of the workload, run once (no sampling,
    no extrapolation).  A batch: whole oracle jobs of its scatterers in a fixed order until
    `budget_s` is spent (at least one); the per-node time of those jobs is scaled to the batch's
    node count, which the value says."""
    if "problems" in w:
        P = w["problems"]
        order = sorted(range(len(P)), key=lambda i: P[i]["curve"].n)
        done, nodes, t = 0, 0, 0.0
        for i in order:
            p = P[i]
            ph = _oracle_job(p["curve"], p["k0"], p["k1"], p["eps0"], p["eps1"], w)
            t += ph["total"]
            nodes += p["curve"].n
            done += 1
            if t >= budget_s:
                break
        total_nodes = sum(p["curve"].n for p in P)
        return {"value": t / nodes * total_nodes, "unit": "s", "cores": _cores(), "kind": "oracle",
                "sample": f"whole oracle jobs of the {done} smallest of {len(P)} scatterers ({nodes} nodes, "
                          f"{t:.1f} s), scaled by node count to all {total_nodes} nodes (an extrapolation)"}
    ph = _oracle_job(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], w)
    return {"value": ph["total"], "unit": "s", "cores": _cores(), "kind": "oracle",
            "phases_s": {k: ph[k] for k in ("compress", "factor", "solve")},
            "sample": "the whole job, run once: oracle compress (proxy tiles and column IDs of every level), "
                      "factor and solve of the workload; numpy/scipy FP64, BLAS threads = host cores"}


def run_reference(args):
    """The oracle as the reference arm: whole jobs of the workload, one per step, for at most
    `args.steps` steps and until `args.ref_budget_s` of timed work is spent (at least one step).
    The oracle holds no device or compiled state, so no warm-up step is run; the JSON line reports
    the steps and warm-up actually run."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    w = _workload(args.workload)
    vals = []
    last = None
    t_start = time.perf_counter()
    while len(vals) < max(1, args.steps):
        last = cpu_baseline(w, args.cpu_budget_s)
        vals.append(last["value"])
        spent = time.perf_counter() - t_start
        if spent + spent / len(vals) > args.ref_budget_s:
            break
    v = sum(vals) / len(vals)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": len(vals),
           "warmup": 0, "ms_per_step": v * 1000.0, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "complex128 (f64)", "data": "synthetic", "config": _config(w, "sym"),
           "cpu_baseline": dict(last, value=v),
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if len(vals) < args.steps:
        out["steps_requested"] = args.steps
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="star16k")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=60.0,
                    help="batch workloads: oracle seconds to spend on whole scatterer jobs")
    ap.add_argument("--ref-budget-s", type=float, default=150.0,
                    help="reference arm: stop adding whole-job steps once this many seconds are spent")
    ap.add_argument("--extras", type=int, default=1,
                    help="with the default workload at one GPU, also time the 65536-node mixed-precision star, "
                         "the 64-scatterer batch and the 262144-node star with the proposer")
    ap.add_argument("--extra-steps", type=int, default=3)
    ap.add_argument("--profile", action="store_true", help="one warm-up + one symmetric step only")
    ap.add_argument("--lu-tc", type=int, default=None, choices=[0, 1, 2],
                    help="with --profile: factorisation path (1: tensor-core updates, 0: FP64 pipe, 2: by launch size)")
    ap.add_argument("--lu-outer", type=int, default=None, choices=[16, 32, 64],
                    help="with --profile: column block of the tensor-core LU updates")
    ap.add_argument("--panel-cluster", type=int, default=None, choices=[1, 2, 4, 8, 16],
                    help="with --profile: largest thread-block cluster of an LU panel")
    ap.add_argument("--lookahead", type=int, default=None, choices=[0, 1],
                    help="with --profile: depth-1 look-ahead of the FP64-pipe LU (panel on a side stream)")
    ap.add_argument("--proposer", action="store_true", help="train the learned rank proposer and attach it")
    ap.add_argument("--comparators", type=int, default=1, help="also time the symmetric PMCHWT comparator")
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
