"""Benchmark: Newton-converged gel steps per second of the GB300 IPC gel step.

Workload (default): the GelSight-Mini-scale gel -- 20x25x4 mm on a 41x51x9 vertex grid (18819
vertices, 96000 tets, bottom face fixed), Neo-Hookean E = 0.3 MPa, nu = 0.45, rho = 1100, a
seeded rigid indenter (sphere r in [2, 6] mm / cylinder r 2 mm x 10 mm / triangular prism side
4 mm, 300-2000 triangles) pressed 1.0 mm over 60 steps then slid 2 mm over 60 steps at
dt = 1/60 s, d_hat = 0.1 mm, kappa automatic, Newton tolerance 1e-5 (relative), FP64.

One "step" is one implicit time step of one gel (all phases of the hot path: placement, broad
phase, assembly, PCG, ACCD, line search, until Newton convergence).  Warm-up steps are the first
W steps of the trajectory, the timed steps the next K.  Every timed step is bracketed by CUDA
events on the library's stream; an L2 flush (256 MB write) separates timed steps outside the
events.  Under torchrun each rank simulates its own gel (seed = rank): weak scaling, no
collective on the data path.

--impl reference times the CPU oracle (FP64, every host core) on the same workload and the same
window of steps (the warm-up steps run untimed first).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="mini", choices=["mini", "small", "batch_mini", "batch_mixed", "serve", "softball"])
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: total request rate [1/s]")
    ap.add_argument("--duration", type=float, default=10.0, help="serve: seconds of arrivals")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serve: HBM admission budget")
    ap.add_argument("--rate-sweep", default="", help="serve: further offered rates, comma separated")
    ap.add_argument("--plain-sample", type=int, default=32,
                    help="serve: gels of the plain FP64 one-at-a-time comparison (0: skip)")
    ap.add_argument("--n-gels", type=int, default=0, help="gels per batch (batch workloads)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--features", action="store_true",
                    help="mini: also time friction, the attachment-driven step and the surface readout")
    ap.add_argument("--softball", default="",
                    help="mini: also time the soft-ball scenes (gel + deformable ball + rigid plate) at these ball "
                         "grid sizes, comma separated (10, 20, 23: the three ball resolutions of Table 3)")
    ap.add_argument("--reference-budget", type=float, default=200.0, help="seconds of timed oracle work")
    ap.add_argument("--batched-gels", type=int, default=64,
                    help="default run: gels of the batched mixed-precision companion measurement (0: skip)")
    ap.add_argument("--pcg-plan", type=int, default=0, choices=[0, 1, 2],
                    help="PCG kernel family (tx_params.pcg_plan): 0 automatic, 1 per-gel-group streaming, 2 pooled")
    ap.add_argument("--pcg-cta-slices", type=int, default=0,
                    help="PCG work split: 32-row slices per CTA at least (0: library default, -1: autotune; "
                         "the autotuner measured no gain on the default workloads)")
    ap.add_argument("--pcg-rel-tol", type=float, default=None,
                    help="PCG forcing term near Newton convergence (default: the library's)")
    ap.add_argument("--pcg-rel-tol-far", type=float, default=None,
                    help="PCG forcing term far from Newton convergence (default: the library's)")
    return ap.parse_args()


def make_workload(kind, seed, n_gels=0):
    """A list of workloads (one per gel of the handle)."""
    from paper_2411_04776_gb300 import workloads as W
    if kind == "small":
        return [W.small_gel_sphere(seed)]
    if kind == "batch_mini":  # config 3 geometry: n copies of the GelSight-Mini gel, own indenters
        return [W.mini_gel(seed + g) for g in range(n_gels or 64)]
    if kind in ("batch_mixed", "serve"):  # config 2 / 4: resolutions drawn from the three grids
        return W.mixed_batch(n_gels or (1024 if kind == "serve" else 256), seed0=seed)
    if kind == "softball":  # soft-to-soft contact: the gel, a 20^3 soft ball, a rigid plate
        return [W.gel_ball(20, seed=seed)]
    return [W.mini_gel(seed)]


NAMES = {"mini": "GelSight-Mini gel 41x51x9 (config 1)", "small": "small gel 10x13x4 (config 0)",
         "batch_mini": "batch of GelSight-Mini gels 41x51x9 (config 3 geometry)",
         "batch_mixed": "batch of gels with mixed resolutions (config 2)",
         "serve": "serving: RL envs with mixed-resolution gels, Poisson step requests (config 4)",
         "softball": "GelSight-Mini gel 41x51x9 + soft ball 20^3 (8000 verts) + rigid plate (soft-to-soft contact)"}


def workload_config(wls, kind, precision):
    n_v = sum(len(w.gel.verts) for w in wls)
    n_t = sum(len(w.gel.tets) for w in wls)
    return {"workload": NAMES[kind], "gels": len(wls), "trajectory": wls[0].name if len(wls) == 1 else "per-gel seeded",
            "verts": n_v, "tets": n_t, "indenter_tris": int(sum(len(w.indenter.tris) for w in wls)),
            "dt": wls[0].dt, "dhat": wls[0].dhat, "newton_tol": wls[0].newton_tol, "precision": precision,
            "l2": "flushed between timed steps (256 MB write)"}


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_QUERY}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [ln.strip().split(",") for ln in self.f.read().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def fp64_peak_tflops(sm_mhz):
    """GB300 FP64 (non-tensor) rate from the datasheet: the nominal 1.25 TFLOP/s at 152 SMs x
    2.07 GHz is 4 FLOP (2 DFMA) per SM per clock; scaled to the given SM clock.  Used only if the
    on-device measurement below fails."""
    return 4.0 * 152 * (sm_mhz or 2070.0) * 1e6 / 1e12


def measure_fma_peaks(dev, target_ms=150.0):
    """FP64 and FP32 FMA-pipe peaks measured on this device now (tx_peak_fma: every SM, four
    independent FMA chains per thread, CUDA-event timed), with the SM clock sampled while they
    run.  Each is the best of three launches sized to about target_ms."""
    from paper_2411_04776_gb300 import binding as B
    out = {}
    with ClockSampler(dev) as clk:
        for bits in (64, 32):
            f, ms = B.tx_peak_fma(bits, 2000)  # warm-up and size probe
            iters = max(2000, int(2000 * target_ms / max(ms, 1e-3)))
            best = 0.0
            for _ in range(3):
                f, ms = B.tx_peak_fma(bits, iters)
                best = max(best, f / (ms * 1e-3) / 1e12)
            out[f"fp{bits}_tflops"] = best
    out["clocks"] = clk.summary()
    out["how"] = "tx_peak_fma: 4 independent FMA chains per thread over every SM, best of 3 CUDA-event-timed launches"
    return out


def run_gpu(args, rank, world, e2e=True):
    import torch
    from paper_2411_04776_gb300 import _build
    from paper_2411_04776_gb300 import binding as B

    if not _build.up_to_date():
        _build.build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    wls = make_workload(args.workload, rank_seed(args.seed, rank), args.n_gels)
    prec = B.TX_PREC_MIXED if args.precision == "mixed" else B.TX_PREC_FP64
    K, Wm = args.steps, args.warmup
    T = min(len(w.poses) for w in wls)
    assert Wm + K <= T, f"the trajectories have {T} steps"
    kw = {k: getattr(args, k) for k in ("pcg_rel_tol", "pcg_rel_tol_far") if getattr(args, k) is not None}
    if getattr(args, "pcg_plan", 0):
        kw["pcg_plan"] = args.pcg_plan
    descs = [B.GelDesc.from_workload(w, precision=prec, pcg_cta_slices=args.pcg_cta_slices, **kw) for w in wls]
    single = len(wls) == 1
    if single:
        gel = B.Gel(descs[0], stream=stream)
        handle, prof_fn = gel.h, gel.profile
    else:
        handle = B.tx_batch_create(descs, stream=stream)
        prof_fn = lambda on: B.tx_batch_profile(handle, on)  # noqa: E731
    dts = np.array([w.dt for w in wls])

    def step(s):
        if single:
            return gel.step(wls[0].poses[s], wls[0].dt)
        st, sts = B.tx_batch_step(handle, np.stack([w.poses[s] for w in wls]), dts)
        return st

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for s in range(Wm):
        st = step(s)
        assert st == 0, B.STATUS_NAMES[st]
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    stats = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    prof_fn(True)
    with ClockSampler(dev) as clk:
        for i in range(K):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            st = step(Wm + i)
            ev[i][1].record(stream)
            assert st == 0, B.STATUS_NAMES[st]
            if single:
                stats.append(gel.stats())
        torch.cuda.synchronize()
    prof = prof_fn(False)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    total_s = float(step_ms.sum()) / 1e3
    clocks = clk.summary()
    # ---- end to end through the public API with host buffers: poses in, positions out
    n = sum(len(w.gel.verts) for w in wls)
    if not e2e:  # companion measurements: the final states are compared across configurations
        finals = []
        for g, w in enumerate(wls):
            x, _, fc, _ = (gel.state() if single else B.tx_batch_state(handle, g, len(w.gel.verts)))
            finals.append((x, fc))
        if single:
            gel.close()
        else:
            B.tx_batch_destroy(handle)
        return dict(total_s=total_s, step_ms=step_ms, stats=stats, prof=prof, clocks=clocks, e2e_s=None,
                    n=n, wls=wls, h2d=0, d2h=0, finals=finals)
    if single:
        gel.reset()
        for s in range(Wm):
            gel.step(wls[0].poses[s], wls[0].dt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(K):
            pose = np.ascontiguousarray(wls[0].poses[Wm + i])
            st = B.tx_gel_step(gel.h, pose, wls[0].dt)
            x, v, fc, _ = B.tx_gel_state(gel.h, n)
            assert st == 0
        e2e_s = time.perf_counter() - t0
        gel.close()
    else:
        for g in range(len(wls)):
            B.tx_batch_reset(handle, g)
        for s in range(Wm):
            step(s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(K):
            st = step(Wm + i)
            assert st == 0
            for g, w in enumerate(wls):
                B.tx_batch_state(handle, g, len(w.gel.verts))
        e2e_s = time.perf_counter() - t0
        B.tx_batch_destroy(handle)
    return dict(total_s=total_s, step_ms=step_ms, stats=stats, prof=prof, clocks=clocks, e2e_s=e2e_s,
                n=n, wls=wls, h2d=len(wls) * (7 * 8 + 8), d2h=2 * n * 3 * 8 + len(wls) * (3 * 8 + 96))


def iteration_histogram(stats):
    """Per-step Newton and PCG iteration counts of the timed steps: percentiles and binned counts."""
    if not stats:
        return None
    out = {}
    for key, name, edges in (("newton_iters", "newton", [0, 5, 10, 20, 50, 100, 200]),
                             ("pcg_iters", "pcg", [0, 100, 500, 1000, 2000, 5000, 10000])):
        v = np.array([s[key] for s in stats], dtype=float)
        bins = []
        for a, b in zip(edges, edges[1:] + [None]):
            inside = (v >= a) & (v < b) if b is not None else (v >= a)
            bins.append({"from": a, "to": b, "steps": int(inside.sum())})
        out[name] = {"p50": float(np.percentile(v, 50)), "p90": float(np.percentile(v, 90)),
                     "max": float(v.max()), "bins": bins}
    return out


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


def roofline(prof, clocks, precision, kernel, fma=None):
    """Roofline of the dominant kernel (the persistent PCG, one launch per Newton round).  FP64:
    bound by the FP64 pipe (GB300 runs FP64 at 1/64 of FP32; no tensor cores on this path), peak
    derived from the unit count and the SM clock.  Mixed precision: the inner solve streams FP32
    blocks, bound by HBM, peak = the measured copy bandwidth."""
    ph = prof["phases"]["pcg"]
    launches = max(ph["launches"], 1)
    avg_ms = ph["ms"] / launches
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            t = json.load(open(tpath)).get(kernel)
            if t and t.get("source_hash") == source_hash(t["files"]):
                traffic = t["bytes_per_launch"]
        except (ValueError, KeyError):
            traffic = None
    if precision == "fp64":
        if fma and fma.get("fp64_tflops"):
            peak = fma["fp64_tflops"]
            note = "measured in this run (tx_peak_fma, FP64 FMA pipe, sampled SM clock %s MHz)" % (
                fma.get("clocks", {}).get("sm_mhz"))
        else:
            peak = fp64_peak_tflops(clocks.get("sm_max_mhz") or 2070.0)
            note = "derived (measurement failed): FP64 (non-tensor) 4 FLOP/clk/SM x 152 SMs x max SM clock"
        achieved = (ph["flops"] / launches) / (avg_ms * 1e-3) / 1e12 if ph["flops"] else None
        return {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "avg_launch_ms": avg_ms, "launches": ph["launches"],
                "peak_note": note + "; achieved = algorithmic FLOP (18 per 3x3 block, 60 per row per iteration; the "
                                    "resident solver adds its Galerkin start: one SpMV and 30 per row per solve)"}
    pk = measured_peaks()
    peak = float(pk.get("hbm_gbs") or 6800.0)
    achieved = (ph["bytes"] / launches) / (avg_ms * 1e-3) / 1e9 if ph["bytes"] else None
    return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "avg_launch_ms": avg_ms, "launches": ph["launches"],
            "peak_note": ("measured copy bandwidth (MEASURED_PEAKS.json)" if pk.get("hbm_gbs") else "fallback 6.8 TB/s")
                         + "; achieved = algorithmic bytes of streaming iterations (40 B per block, 212 B per row; the "
                            "single-gel solver adds its Galerkin start per solve)"}


def pcg_kernel_name(precision, n_gels):
    """The PCG kernel the library's automatic plan runs for n_gels gels: resident for one gel,
    the pooled streaming form from 32 gels on, the per-gel-group streaming form between."""
    if n_gels == 1:
        return "k_pcg64_res" if precision == "fp64" else "k_pcg_mixed_res"
    if n_gels >= 32:
        return "k_pcg64_pool" if precision == "fp64" else "k_pcg_mixed_pool"
    return "k_pcg64" if precision == "fp64" else "k_pcg_mixed"


def ran_pcg_kernel(prof, precision, n_gels):
    """pcg_kernel_name, unless the profile shows that a single gel's solves took the streaming
    kernels (its slices did not fit the resident kernels' shared memory)."""
    if n_gels == 1 and prof.get("pcg_resident_launches", 1) == 0 and prof.get("pcg_streaming_launches", 0) > 0:
        return "k_pcg64" if precision == "fp64" else "k_pcg_mixed"
    return pcg_kernel_name(precision, n_gels)


def source_hash(files):
    """Hash of the CUDA sources a kernel is built from (the ncu counters in profiles/traffic.json
    are used only while these are unchanged)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2411_04776_gb300", "csrc")
    for f in sorted(files):
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def host_description():
    """CPU model and core count of this host (the oracle's timings are quoted with them)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model, "nproc": os.cpu_count(), "arch": os.uname().machine}


def oracle_window(wl, first, count, budget, threads):
    """The oracle as it stands on the trajectory of workload wl: steps 0..first-1 untimed (all host
    cores: the same state whatever the thread count, the oracle's sums do not depend on it), then
    up to `count` steps from `first` on timed with `threads` threads until `budget` seconds of
    oracle work are spent (at least one step).  Returns (timed steps, seconds, threads used)."""
    from oracle import oracle as O
    O.set_threads(0)
    og = O.OracleGel.from_workload(wl)
    for s in range(first):
        assert og.step(wl.poses[s], wl.dt)["status"] == 0
    used = O.set_threads(threads)
    t0 = time.perf_counter()
    done = 0
    while done < count and first + done < len(wl.poses):
        assert og.step(wl.poses[first + done], wl.dt)["status"] == 0
        done += 1
        if time.perf_counter() - t0 > budget:
            break
    el = time.perf_counter() - t0
    O.set_threads(0)
    return done, el, used


def cpu_baseline(args, budget=30.0):
    """The oracle as it stands (FP64 C++, every host core; bitwise the result of one thread) on
    the first timed steps of the GPU arm's window: the same trajectory (first gel of a batch),
    steps args.warmup, args.warmup + 1, ... until about `budget` seconds."""
    wl = make_workload(args.workload, args.seed, 1)[0]
    done, el, used = oracle_window(wl, args.warmup, args.steps, budget, 0)
    host = host_description()
    return {"value": done / el, "unit": "steps/s", "cores": used, "kind": "oracle",
            "sample": f"oracle (FP64 C++, OpenMP, {used} threads) steps {args.warmup}..{args.warmup + done - 1} of "
                      f"the GPU arm's trajectory (the start of its timed window), {el:.1f} s; steps 0..{args.warmup - 1} "
                      f"run untimed first", "host": host}


def run_serve(args):
    """Continuous-batching server over resident gels (config 4): Poisson step requests from the
    environments, admission by HBM footprint, one Newton iteration per round for all admitted.
    The offered rate args.rate is the headline; --rate-sweep adds lower rates (same server; before
    each rate the environments are reset and take the warm-up steps again, so every rate serves
    the same trajectory window) to find the highest rate the server sustains (served rate >= 95 %
    of the offered one).  Beside it, the plain FP64 path stepping a sample of the same
    gels one at a time."""
    import torch
    from paper_2411_04776_gb300 import binding as B
    from paper_2411_04776_gb300 import serving as S
    torch.cuda.set_device(0)
    wls = make_workload("serve", args.seed, args.n_gels)
    prec = B.TX_PREC_MIXED if args.precision == "mixed" else B.TX_PREC_FP64
    t0 = time.perf_counter()
    srv = S.GelServer(wls, args.budget_gb * 1e9, precision=prec, stream=torch.cuda.current_stream(),
                      pcg_cta_slices=args.pcg_cta_slices or 0)
    t_create = time.perf_counter() - t0
    # warm-up: every environment takes its first steps
    srv.run_schedule([list(range(srv.n))] * max(1, args.warmup))
    rates = [args.rate] + [float(r) for r in args.rate_sweep.split(",") if r.strip()]
    runs = []
    for k, rate in enumerate(rates):
        if k > 0:  # every rate starts from the same state: the environments back at the warm-up's end
            for e in range(srv.n):
                B.tx_batch_reset(srv.handle, e)
            srv.cursor[:] = 0
            srv.run_schedule([list(range(srv.n))] * max(1, args.warmup))
        srv.completed.clear()
        srv.max_inflight, srv.max_inflight_bytes = 0, 0.0
        arrivals = S.poisson_arrivals(srv.n, rate, args.duration, args.seed + 1 + k)
        with ClockSampler(0) as clk:
            t1 = time.perf_counter()
            done = list(srv.serve(arrivals, drain=True))
            wall = time.perf_counter() - t1
        ok = [r for r in done if r.status == 0]
        served = len(ok) / wall
        runs.append({"rate": rate, "requests": len(arrivals), "value": served, "unit": "steps/s",
                     "wall_s": wall, "sustained": served >= 0.95 * len(arrivals) / args.duration,
                     "latency_ms": S.latency_summary(done), "failed": len(done) - len(ok),
                     "failed_requests": [[r.env, r.step % len(wls[r.env].poses), B.STATUS_NAMES.get(r.status, r.status)]
                                         for r in done if r.status != 0][:16],
                     "max_inflight": srv.max_inflight, "max_inflight_gb": srv.max_inflight_bytes / 1e9,
                     "clocks": clk.summary()})
    srv.close()
    plain = plain_fp64_sequential(wls[:args.plain_sample], 4, max(1, args.warmup))[0] if args.plain_sample else None
    head = runs[0]
    sustained = [r["rate"] for r in runs if r["sustained"]]
    line = {"metric": "gel Newton-converged steps/sec", "value": head["value"], "unit": "steps/s", "n_gpus": 1,
            "steps": int(round(head["value"] * head["wall_s"])), "warmup": args.warmup,
            "ms_per_step": 1e3 / max(head["value"], 1e-9), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
            "config": dict(workload_config(wls, "serve", args.precision), rate=args.rate, duration=args.duration,
                           budget_gb=args.budget_gb),
            "latency_ms": head["latency_ms"], "requests": head["requests"], "failed": head["failed"],
            "failed_requests": head["failed_requests"], "max_inflight": head["max_inflight"],
            "max_inflight_gb": head["max_inflight_gb"], "resident_gb": float(srv.footprint.sum() / 1e9),
            "create_s": t_create, "rate_sweep": runs[1:],
            "max_sustained_rate": max(sustained) if sustained else None,
            "plain_fp64_one_at_a_time": plain,
            "vs_plain_fp64": (head["value"] / plain["value"]) if plain else None,
            "clocks": head["clocks"]}
    print(json.dumps(line))


def max_over_ranks(values, device):
    """The job's time is the slowest rank's: element-wise maximum over the process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def job_throughput(world, gels_per_rank, steps, max_seconds):
    """Whole-job gel steps per second: every rank steps its own gels (weak scaling, no exchange)."""
    return world * gels_per_rank * steps / max_seconds


def rank_seed(seed, rank):
    """Each rank draws its own gels (distinct seeded workloads)."""
    return seed + 1000 * rank


def main():
    args = parse_args()
    if args.workload == "serve" and args.impl == "gpu":
        return run_serve(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        from oracle import oracle as O
        O.build()
        wls = make_workload(args.workload, args.seed, args.n_gels)
        done, el, used = oracle_window(wls[0], args.warmup, args.steps, args.reference_budget, 0)
        value = done / el
        host = host_description()
        cb = {"value": value, "unit": "steps/s", "cores": used, "kind": "oracle",
              "sample": f"oracle (FP64 C++, OpenMP, {used} threads) steps {args.warmup}..{args.warmup + done - 1} "
                        f"of the GPU arm's trajectory, {el:.1f} s (steps 0..{args.warmup - 1} untimed first); "
                        f"budget {args.reference_budget:.0f} s", "host": host}
        line = {"metric": "gel Newton-converged steps/sec", "value": value, "unit": "steps/s",
                "impl": "reference", "n_gpus": args.gpus, "steps": done, "steps_requested": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * el / max(done, 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(wls[:1] if args.workload == "mini" else wls, args.workload, "fp64"),
                "cpu_baseline": cb,
                "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    r = run_gpu(args, rank, world)
    fma = None
    if rank == 0:
        try:
            fma = measure_fma_peaks(int(os.environ.get("LOCAL_RANK", 0)))
        except Exception as e:  # noqa: BLE001
            fma = {"error": f"{type(e).__name__}: {e}"}
    total_s, e2e_s = r["total_s"], r["e2e_s"]
    if world > 1:
        total_s, e2e_s = max_over_ranks([total_s, e2e_s], "cuda")
    if rank != 0:
        return
    K = args.steps
    ng = len(r["wls"])
    value = job_throughput(world, ng, K, total_s)
    step_ms = r["step_ms"]
    prof = r["prof"]
    line = {
        "metric": "gel Newton-converged steps/sec", "value": value, "unit": "steps/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic",
        "config": workload_config(r["wls"], args.workload, args.precision),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "max": float(step_ms.max())},
        "newton_iters_per_step": prof["newton_iters"] / (ng * K),
        "pcg_iters_per_step": prof["pcg_iters"] / (ng * K),
        "roofline": roofline(r["prof"], r["clocks"], args.precision, ran_pcg_kernel(r["prof"], args.precision, ng), fma),
        "phases_ms": {k: round(v["ms"], 3) for k, v in r["prof"]["phases"].items()},
        "gpu_launches": r["prof"]["kernel_launches"],
        "pcg_launches": {"resident": r["prof"]["pcg_resident_launches"],
                         "streaming": r["prof"]["pcg_streaming_launches"],
                         "pooled": r["prof"]["pcg_pool_launches"]},
        "fma_peaks": fma,
        "iteration_histogram": iteration_histogram(r["stats"]),
        "clocks": r["clocks"],
        "e2e": {"value": world * ng * K / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"]},
    }
    args.fma_peaks = fma
    if world == 1 and args.workload == "mini" and args.batched_gels > 0:
        try:  # a companion measurement: its failure is reported, the main line still prints
            line["batched_mixed"] = batched_mixed(args)
        except Exception as e:  # noqa: BLE001
            line["batched_mixed"] = {"error": f"{type(e).__name__}: {e}"}
    if world == 1 and args.workload == "mini" and args.features:
        try:
            line["features"] = features_companion(args)
        except Exception as e:  # noqa: BLE001
            line["features"] = {"error": f"{type(e).__name__}: {e}"}
    if world == 1 and args.workload == "mini" and args.softball:
        try:
            line["softball"] = softball_companion(args)
        except Exception as e:  # noqa: BLE001
            line["softball"] = {"error": f"{type(e).__name__}: {e}"}
    if world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(args)
        except Exception as e:  # noqa: BLE001
            line["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}", "kind": "oracle"}
    print(json.dumps(line))


def features_companion(args):
    """Companion measurement of the further couplings on the GelSight-Mini gel (41x51x9, the
    benchmark's trajectory, FP64): the same step window (warm-up steps untimed, then CUDA-event
    timed steps with L2 flushed before each) for the plain step, with IPC lagged friction
    (mu 0.5, eps_v 1e-3 m/s), and attachment-driven (the case carries the bottom face 2 um per
    step along x while the indenter presses); and the gel-surface readout through the C ABI (a
    9 x 7 marker grid and a 320 x 240 height map of the top surface, host arrays returned) after
    every timed plain step, timed on the host clock around each call."""
    import torch
    from paper_2411_04776_gb300 import binding as B
    from paper_2411_04776_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    wl = W.mini_gel(args.seed)
    K, Wm = args.steps, args.warmup
    X = wl.gel.verts
    lo, hi = X.min(axis=0), X.max(axis=0)
    gx, gy = np.meshgrid(np.linspace(lo[0], hi[0], 9)[1:-1], np.linspace(lo[1], hi[1], 11)[1:-1], indexing="ij")
    markers = np.column_stack([gx.ravel(), gy.ravel()])  # 7 x 9 = 63 rest points inside the top face
    nx, ny = 320, 240
    grid = dict(nx=nx, ny=ny, x0=float(lo[0]), y0=float(lo[1]), dx=float(hi[0] - lo[0]) / nx,
                dy=float(hi[1] - lo[1]) / ny)

    def case(s):
        return W.pose((2e-6 * (s + 1), 0.0, 0.0))

    def run(kind):
        kw = dict(friction=0.5, friction_eps_v=1e-3) if kind == "friction" else {}
        gel = B.Gel.from_workload(wl, stream=stream, **kw)

        def step(s):
            if kind == "attached":
                return gel.step_attached(wl.poses[s], case(s), wl.dt)
            return gel.step(wl.poses[s], wl.dt)
        for s in range(Wm):
            assert step(s) == 0, (kind, s)
        ms, newton, pcg, rd_m, rd_h = [], 0, 0, [], []
        for i in range(K):
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = step(Wm + i)
            e1.record(stream)
            torch.cuda.synchronize()
            assert st == 0, (kind, Wm + i, st)
            ms.append(e0.elapsed_time(e1))
            stt = gel.stats()
            newton += stt["newton_iters"]
            pcg += stt["pcg_iters"]
            if kind == "plain":
                t0 = time.perf_counter()
                _, found = gel.markers(markers)
                t1 = time.perf_counter()
                hm = gel.height_map(**grid)
                t2 = time.perf_counter()
                assert found.all() and np.isfinite(hm).mean() > 0.9
                rd_m.append(t1 - t0)
                rd_h.append(t2 - t1)
        fc = np.array(gel.stats()["contact_force"])
        gel.close()
        ms = np.array(ms)
        out = {"value": K / (ms.sum() / 1e3), "unit": "steps/s", "p50_ms": float(np.percentile(ms, 50)),
               "newton_iters_per_step": newton / K, "pcg_iters_per_step": pcg / K,
               "final_contact_force_N": fc.tolist()}
        if kind == "plain":
            out["readout"] = {"markers": len(markers), "markers_us_per_call": 1e6 * float(np.median(rd_m)),
                              "height_map_px": nx * ny, "height_map_us_per_call": 1e6 * float(np.median(rd_h)),
                              "timing": "host clock around the C-ABI call (device work, copy to host)"}
        return out
    res = {"workload": NAMES["mini"], "steps": K, "warmup": Wm, "precision": "fp64"}
    for kind in ("plain", "friction", "attached"):
        res[kind] = run(kind)
    return res


# GIPC's time per frame of the soft-ball scene at three ball resolutions (Table 3: vertices, tets, ms),
# measured by the paper on its own machine: context for the same-sized scenes here, not a target
TABLE3_GIPC = {10: (1029, 3717, 24.95), 20: (7900, 40370, 110.47), 23: (12509, 66563, 221.61)}


def softball_companion(args):
    """Companion measurement of soft-to-soft contact: the GelSight-Mini gel (41x51x9) with a soft
    ball of radius 4 mm on it (an n^3 ball grid, the gel's material) squeezed by a rigid 12 mm plate
    (`workloads.gel_ball`), FP64: warm-up steps untimed, then CUDA-event timed steps with L2 flushed
    before each; per ball size the mean time per step (frame), its Newton and PCG iterations, and
    the soft-soft pair assemblies whose cross-body blocks found no spare matrix position."""
    import torch
    from paper_2411_04776_gb300 import binding as B
    from paper_2411_04776_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    K, Wm = args.steps, args.warmup
    res = {"steps": K, "warmup": Wm, "precision": "fp64", "sizes": []}
    for n in (int(v) for v in args.softball.split(",") if v.strip()):
        wl = W.gel_ball(n, seed=args.seed)
        gel = B.Gel.from_workload(wl, stream=stream, newton_max_iter=1000)
        for s in range(Wm):
            assert gel.step(wl.poses[s], wl.dt) == 0, (n, s)
        ms, newton, pcg, cut, act = [], 0, 0, 0, 0
        for i in range(K):
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = gel.step(wl.poses[Wm + i], wl.dt)
            e1.record(stream)
            torch.cuda.synchronize()
            assert st == 0, (n, Wm + i, st)
            ms.append(e0.elapsed_time(e1))
            stt = gel.stats()
            newton += stt["newton_iters"]
            pcg += stt["pcg_iters"]
            cut += stt["soft_pairs_cut"]
            act = max(act, stt["active_pairs"])
        gel.close()
        ms = np.array(ms)
        nb = n ** 3
        row = {"workload": wl.name, "ball_verts": nb, "ball_tets": 6 * (n - 1) ** 3, "mesh_verts": len(wl.gel.verts),
               "ms_per_step": float(ms.mean()), "p50_ms": float(np.percentile(ms, 50)),
               "newton_iters_per_step": newton / K, "pcg_iters_per_step": pcg / K, "most_active_pairs": act,
               "soft_pairs_cut": cut}
        if n in TABLE3_GIPC:
            v, t, g = TABLE3_GIPC[n]
            row["table3_gipc"] = {"ball_verts": v, "ball_tets": t, "ms_per_frame": g}
        res["sizes"].append(row)
    return res


def plain_fp64_sequential(wls, steps, warmup):
    """The plain FP64 path on the same gels and the same step window, one gel at a time: each gel
    takes its warm-up steps untimed, then its timed steps (CUDA events, L2 flushed before each)."""
    import torch
    from paper_2411_04776_gb300 import binding as B
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ms, finals = [], []
    for w in wls:
        gel = B.Gel(B.GelDesc.from_workload(w, precision=B.TX_PREC_FP64), stream=stream)
        for s in range(warmup):
            assert gel.step(w.poses[s], w.dt) == 0
        for i in range(steps):
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            assert gel.step(w.poses[warmup + i], w.dt) == 0
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        x, _, fc, _ = gel.state()
        finals.append((x, fc))
        gel.close()
    ms = np.array(ms)
    return {"gels": len(wls), "value": len(ms) / (ms.sum() / 1e3), "unit": "steps/s",
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))}}, finals


def state_difference(a, b):
    """Max / RMS vertex displacement difference and max relative contact-force difference between
    two sets of final gel states (same gels, same steps)."""
    dmax, sq, cnt, fmax = 0.0, 0.0, 0, 0.0
    for (xa, fa), (xb, fb) in zip(a, b):
        d = np.abs(xa - xb)
        dmax = max(dmax, float(d.max()))
        sq += float((d ** 2).sum())
        cnt += d.size
        fmax = max(fmax, float(np.abs(fa - fb).max() / max(np.abs(fb).max(), 1e-30)))
    return {"max_disp_m": dmax, "rms_disp_m": (sq / max(cnt, 1)) ** 0.5, "max_force_rel": fmax}


def batched_mixed(args):
    """Companion measurement of the same metric on the batched configurations: args.batched_gels
    GelSight-Mini gels (41x51x9, each with its own seeded indenter and press/slide trajectory)
    stepped together (one handle) in mixed precision (FP32 elastic blocks and FP32 inner PCG with
    FP64 residual refinement) and in FP64, and the plain FP64 path stepping the same gels one at
    a time over the same steps.  vs_plain_fp64 splits into the batching gain (batched FP64 / one
    at a time) and the precision gain (batched mixed / batched FP64).  Accuracy: the final states
    of the mixed batch against the one-at-a-time FP64 run (both at the workload's Newton
    tolerance, so the difference includes where each run stopped within it)."""
    import argparse
    a = argparse.Namespace(**vars(args))
    a.workload, a.n_gels, a.precision = "batch_mini", args.batched_gels, "mixed"
    a.steps, a.warmup = 4, 3
    r = run_gpu(a, 0, 1, e2e=False)
    ng = len(r["wls"])
    value = ng * a.steps / r["total_s"]
    prof = r["prof"]
    a64 = argparse.Namespace(**vars(a))
    a64.precision = "fp64"
    r64 = run_gpu(a64, 0, 1, e2e=False)
    value64 = ng * a.steps / r64["total_s"]
    plain, plain_finals = plain_fp64_sequential(r["wls"], a.steps, a.warmup)
    return {"workload": workload_config(r["wls"], a.workload, "mixed")["workload"], "gels": ng,
            "precision": "mixed", "value": value, "unit": "steps/s", "steps": a.steps, "warmup": a.warmup,
            "ms_per_batch_step": r["total_s"] * 1e3 / a.steps,
            "latency_ms": {"p50": float(np.percentile(r["step_ms"], 50)),
                           "p99": float(np.percentile(r["step_ms"], 99))},
            "newton_iters_per_step": prof["newton_iters"] / (ng * a.steps),
            "pcg_iters_per_step": prof["pcg_iters"] / (ng * a.steps),
            "batched_fp64": {"value": value64, "unit": "steps/s", "ms_per_batch_step": r64["total_s"] * 1e3 / a.steps,
                             "newton_iters_per_step": r64["prof"]["newton_iters"] / (ng * a.steps),
                             "pcg_iters_per_step": r64["prof"]["pcg_iters"] / (ng * a.steps),
                             "roofline": roofline(r64["prof"], r64["clocks"], "fp64", pcg_kernel_name("fp64", ng),
                                                  args.fma_peaks),
                             "pcg_launches": {"resident": r64["prof"]["pcg_resident_launches"],
                                              "streaming": r64["prof"]["pcg_streaming_launches"],
                                              "pooled": r64["prof"]["pcg_pool_launches"]}},
            "plain_fp64_same_steps": plain,
            "vs_plain_fp64": value / plain["value"],
            "batching_gain_fp64": value64 / plain["value"],
            "precision_gain_batched": value / value64,
            "accuracy_vs_plain_fp64": state_difference(r["finals"], plain_finals),
            "accuracy_batched_fp64_vs_plain_fp64": state_difference(r64["finals"], plain_finals),
            "roofline": roofline(prof, r["clocks"], "mixed", pcg_kernel_name("mixed", ng)),
            "pcg_launches": {"resident": prof["pcg_resident_launches"], "streaming": prof["pcg_streaming_launches"],
                             "pooled": prof["pcg_pool_launches"]},
            "phases_ms": {k: round(v["ms"], 3) for k, v in prof["phases"].items()},
            "gpu_launches": prof["kernel_launches"], "clocks": r["clocks"]}


if __name__ == "__main__":
    main()
