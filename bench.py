"""KBE time-stepping benchmark on GB300.

A bench *step* is one whole Kadanoff-Baym trajectory of the driven 2-D
workload c2 (N_b = 4 bands, 8x8 mesh, N_t = 512 steps, dt = 0.02, P(EC)^2 E):
reset to the Fermi state, then 512 time steps on the device-resident history
(4.3 GB, larger than L2). The metric is KBE time-steps per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The headline value is the plain FP64 path; the reduced-storage forms (DF64:
FP32 hi/lo pairs with a double-float sweep, C64: complex64 history) are timed
on the same workload and reported under "forms" with their speedup and their
error against the FP64 trajectory. With N > 1 (torchrun, one process per GPU)
every rank advances its own independent c2 system (weak scaling, no
data-path collective).
--impl reference times the FP64 CPU oracle on the host cores: each bench step
is one row evaluation (Sigma row + collision row, as the oracle's stepper
performs it) plus one row update at a sampled row n of the c2 trajectory, on a
random history of c2's shape; the full 512-step trajectory time is integrated
from those samples (3 evaluations and 3 updates per step), so the value is an
extrapolated whole-trajectory rate, not the rate of its cheap first rows.
The line also carries the reverse mode on the same system ("gradient":
forward + kbe_backward for dL/dA_i, dL/dU) and the full c3 trajectory in all
three forms; --gradient-fd checks the gradient by central differences instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import kbe_inputs as ki  # noqa: E402

METRIC = "KBE time-steps/s"
WORKLOAD = ("c2: N_b=4, 8x8 mesh (n_k=64), N_t=512, dt=0.02, U=1.0, beta=20, "
            "Peierls pulse A0=0.3, HF + second Born, P(EC)^2E")
# Roofline denominators of the sweep (the dominant kernel). The ALU peaks are
# measured live by kbe_measure_fma_peaks (FP64 and FP32 FMA throughput); the
# HBM peak is the measured copy bandwidth in MEASURED_PEAKS.json. The
# FP64 form is bound by the FP64 pipe; the double-float form by FP32 issue (6
# FP32 instructions per double-float flop: a complex multiply-add is 4
# products x 12 instructions = 8 flop); the complex64 form streams half the
# bytes and is reported against HBM, with its FP32 fraction beside it.
HBM_FALLBACK_GBS = 6800.0
# DRAM traffic of the sweep per launch as a multiple of its algorithmic bytes,
# from ncu (dram__bytes_read.sum + dram__bytes_write.sum) at row 501 of the
# full c2 run, one launch per form; traffic grows with the triangle like the
# algorithmic bytes, so the average launch is scaled by the same factor.
# None: the form's kernel changed after its counters were taken.
TRAFFIC_RATIO = {"fp64": None, "df64": 2.77, "c64": None, "f16x2": None}
DTYPES = {"fp64": "f64", "df64": "df64 (f32 hi/lo pairs; everything but the sweep f64)",
          "c64": "c64/f32 history + sweep (everything else f64)",
          "f16x2": "split-f16 pair history, tcgen05 f16 MMAs with f32 accumulation (Sigma c64; everything else f64)"}
FORMS = ("fp64", "df64", "c64", "f16x2")
# rows of the c2 trajectory at which the oracle is timed (its cost grows as n^2)
ORACLE_ROWS = [63, 127, 191, 255, 319, 383, 447, 511]
ORACLE_ROWS_1T = [31, 95, 159]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--nt", type=int, default=None, help="truncate N_t (testing only)")
    p.add_argument("--precision", default="fp64", choices=["fp64", "df64", "c64", "f16x2"],
                   help="history storage / sweep arithmetic of the headline value (fp64 meets "
                        "the 1e-10 bar; df64 / c64 are the reduced-storage forms)")
    p.add_argument("--forms", default="all", choices=["all", "none", "gradient", "batched"],
                   help="also time the other storage forms (speedup and error vs the headline), "
                        "the batched and paper-shaped forms and the gradient; 'gradient' or "
                        "'batched': only that one")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true",
                   help="skip kbe_autotune (the sweep's l-split chosen by timing before the timed region)")
    p.add_argument("--sweep-row", type=int, default=None,
                   help="time the collision sweep alone at this row on random history of c2's and c3's "
                        "shape, every launch choice of the C64 form, then exit")
    p.add_argument("--sweep-shapes", default="c2,c3", help="workloads for --sweep-row")
    p.add_argument("--sweep-forms", default=None,
                   help="comma list of forms for --sweep-row (default: every form of the workload)")
    p.add_argument("--sweep-ti", type=int, default=None,
                   help="--sweep-row: only the tile / tensor-core choices with this TI")
    p.add_argument("--gradient-fd", action="store_true",
                   help="check the c5 gradient (512 steps) by central differences on 16 A_i and U, then exit")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(times_s, units_per_rank):
    """Whole-job throughput: units all ranks processed / slowest rank's time."""
    t = max(times_s)
    return sum(units_per_rank) / t, t


def reduce_max(values, dist=None, device="cuda"):
    """Element-wise max over ranks (timing only; no data-path collective)."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(values, device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in a thread."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._th = None

    def start(self):
        def run():
            while not self._stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits"],
                                         capture_output=True, text=True, timeout=5).stdout.strip()
                    if out:
                        self.rows.append([x.strip() for x in out.split(",")])
                except Exception:
                    pass
                self._stop.wait(0.2)
        self._th = threading.Thread(target=run, daemon=True)
        self._th.start()

    def stop(self):
        self._stop.set()
        if self._th:
            self._th.join(timeout=10)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def time_trajectories(g, nt, steps, warmup, stream, sampler=None, dist=None):
    """W untimed + K timed trajectories (reset + nt steps) with the sweep profiled."""
    import torch
    for _ in range(warmup):
        g.reset()
        g.step(nt)
    g.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    g.profile(True)
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.reset()
        g.step(nt)
    e1.record(stream)
    e1.synchronize()
    g.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    prof = g.profile_read()
    g.profile(False)
    return e0.elapsed_time(e1) / 1e3, prof, clocks


def hbm_peak():
    """(GB/s, source) of the measured copy bandwidth, else the fallback"""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs: STREAM-style copy)"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback (no measured HBM peak on this box)"


def tensor_peak():
    """(GFLOP/s, source): dense FP16 tensor rate = the measured sustained bf16
    cuBLAS rate (the same tensor-core rate), else the fallback"""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return (float(json.load(f)["bf16_tflops_sustained"]) * 1e3,
                    "measured (MEASURED_PEAKS.json bf16_tflops_sustained; FP16 dense runs at the bf16 rate)")
    except Exception:
        return 1.7e6, "fallback (1.7 PFLOP/s sustained bf16)"


def alu_peaks(kbe):
    """measured FMA throughput (GFLOP/s) of this GPU: {"fp64": .., "fp32": ..}"""
    f64, f32 = kbe.measure_fma_peaks()
    return {"fp64": f64, "fp32": f32}


def roofline(prof, precision, t_dev, peaks):
    """The sweep's roofline over the summed sweep event time. HBM-bound forms
    (C64, split-FP16): achieved = the triangle read once plus the Sigma and I
    rows, in bytes. ALU-bound forms (FP64, DF64): achieved = the flops the
    kernel's algorithm performs (the I^<, I^> - I^< form: 2/3 of the method's
    24 n^2 N_b^3 n_k count; the FP64 kernel's three-multiplication products:
    FP64-pipe operations as flops), so frac is a pipe utilisation; the
    method's count is reported beside it (achieved_method_count)."""
    sweep_s = prof["sweep_ms"] / 1e3
    nl = max(1, prof["sweep_launches"])
    alg_bytes = prof["sweep_bytes"] / nl
    flops = prof["sweep_flops"] / sweep_s / 1e9 if sweep_s > 0 else 0.0
    executed = prof["sweep_flops_executed"] / sweep_s / 1e9 if sweep_s > 0 else 0.0
    gbs = prof["sweep_bytes"] / sweep_s / 1e9 if sweep_s > 0 else 0.0
    hbm, hsrc = hbm_peak()
    ratio = TRAFFIC_RATIO[precision]
    common = {"kernel": "collision sweep (a2)", "traffic": ratio * alg_bytes if ratio else None,
              "traffic_unit": "bytes per launch", "algorithmic_bytes_per_launch": alg_bytes,
              "launches": prof["sweep_launches"],
              "sweep_share_of_step": sweep_s / t_dev if t_dev > 0 else None,
              "hbm_gbs_achieved": gbs, "hbm_frac": gbs / hbm, "hbm_peak_gbs": hbm, "hbm_peak_source": hsrc}
    if precision == "c64":
        fp32 = peaks["fp32"]
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "peak_source": hsrc, **common,
                "alu": {"achieved_executed": executed, "peak": fp32, "unit": "GFLOP/s FP32",
                        "frac_executed": executed / fp32,
                        "peak_source": "measured FP32 FMA throughput (kbe_measure_fma_peaks)"}}
    if precision == "f16x2":   # executed = the MMAs' flops (hi and lo parts of both operands)
        tpk, tsrc = tensor_peak()
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "peak_source": hsrc, **common,
                "tensor": {"achieved_executed": executed, "peak": tpk, "unit": "GFLOP/s FP16 dense",
                           "frac_executed": executed / tpk, "peak_source": tsrc}}
    if precision == "df64":
        peak = peaks["fp32"] / 6.0
        unit, src = ("GFLOP/s FP64-equivalent (double-float)",
                     "measured FP32 FMA throughput / 6 FP32 instructions per double-float flop")
    else:
        peak = peaks["fp64"]
        unit, src = "GFLOP/s FP64", "measured FP64 FMA throughput (kbe_measure_fma_peaks)"
    return {"bound": "alu", "achieved": executed, "peak": peak, "unit": unit, "frac": executed / peak,
            "peak_source": src, "achieved_method_count": flops, "frac_method_count": flops / peak, **common}


def run_ours(args, rank, world, local):
    import torch
    import paper_2505_19467_gb300 as kbe

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    s = ki.config("c2", nt=args.nt)
    nt = s.nt
    stream = torch.cuda.Stream()
    g = kbe.KBE.from_system(s, stream=stream, precision=kbe.PRECISIONS[args.precision])
    tuned = {}
    if not args.no_autotune:   # before the timed region; choices are kept per shape for the process
        tuned[args.precision] = [int(x) for x in g.autotune() if x]
    peaks = alu_peaks(kbe)     # measured FMA throughput, the ALU roofline denominators

    sampler = ClockSampler(local) if rank == 0 else None
    t_dev, prof, clocks = time_trajectories(g, nt, args.steps, args.warmup, stream, sampler, dist)
    _, ref_obs = g.observables_all()

    # ---- end to end through the C ABI with host buffers -------------------
    R = np.ascontiguousarray(s.hop_R, np.int32)
    T = np.ascontiguousarray(s.hop_T, np.complex128)
    Uarr = np.array([s.U], np.float64)
    v = np.ascontiguousarray(s.v, np.float64)
    A = np.ascontiguousarray(s.A, np.float64)
    nkb_host = np.empty((nt + 1, s.nk, s.nb), np.float64)
    sc_host = np.empty((nt + 1, 6), np.float64)
    h2d = R.nbytes + T.nbytes + Uarr.nbytes + v.nbytes + A.nbytes + 16
    d2h = nkb_host.nbytes + sc_host.nbytes
    n_e2e = min(args.steps, 5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        g.set_hamiltonian(R, T)
        g.set_interaction(Uarr, v)
        g.set_drive(A, s.direction)
        g.reset()
        g.step(nt)
        g.observables_all(nkb_host, sc_host)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    ref_nkb = nkb_host.copy()
    g.close()
    if dist:
        dist.barrier()

    times = reduce_max([t_dev, t_e2e], dist)
    units = nt * args.steps
    value, tmax = aggregate([times[0]], [units * world])
    e2e_value = nt * n_e2e * world / times[1]

    # ---- the reduced-storage forms on the same workload (speedup, error) ----
    forms = {}
    for form in ([] if args.forms != "all" else [f for f in FORMS if f != args.precision]):
        gf = kbe.KBE.from_system(s, stream=stream, precision=kbe.PRECISIONS[form])
        if not args.no_autotune:
            tuned[form] = [int(x) for x in gf.autotune() if x]
        kf = min(args.steps, 5)
        tf, pf, _ = time_trajectories(gf, nt, kf, max(3, min(args.warmup, 3)), stream, None, dist)
        nkb_f, sc_f = gf.observables_all()
        gf.close()
        escale = np.abs(ref_obs[:, 5]).max()
        forms[form] = {"value": nt * kf / tf, "trajectories_timed": kf,
                       "speedup_vs_" + args.precision: (nt * kf / tf) / (units / t_dev),
                       "max_abs_err_density": float(np.abs(nkb_f - ref_nkb).max()),
                       "max_rel_err_energy": float(np.abs(sc_f[:, 1:] - ref_obs[:, 1:]).max() / escale),
                       "max_rel_err_N": float(np.abs(sc_f[:, 0] - ref_obs[:, 0]).max() / abs(ref_obs[0, 0])),
                       "dtype": DTYPES[form], "roofline": roofline(pf, form, tf, peaks)}

    # ---- batched form: uneven systems together vs one after another ----------
    def leg(fn, *a):   # a failing side measurement is reported, the headline still printed
        try:
            return fn(*a)
        except Exception as exc:   # noqa: BLE001
            return {"error": f"{type(exc).__name__}: {exc}"}

    batched = paper = gradient = c3 = None
    if args.forms in ("all", "batched"):
        batched = leg(batched_form, kbe, stream, args)
    if args.forms == "all":
        paper = leg(paper_shape, kbe, stream)
        c3 = leg(c3_form, kbe, stream, peaks)
    if args.forms in ("all", "gradient"):
        gradient = leg(gradient_form, kbe, stream, args, peaks)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "time-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision], "data": "synthetic (seeded c2 system, kbe_inputs)",
            "config": {"workload": WORKLOAD, "precision": args.precision,
                       "bench_step": f"one trajectory: reset + {nt} time steps",
                       "time_steps_per_bench_step": nt, "n_corr": 2,
                       "l2": "history 4.3 GB > 129 MB L2 (inputs larger than L2)",
                       "parallelism": f"replicas x{world} (independent systems)",
                       "autotune": {"sweep_split_ctas_per_sm_by_row_bucket": tuned} if tuned else "off"},
            "roofline": roofline(prof, args.precision, t_dev, peaks),
            "e2e": {"value": e2e_value, "unit": "time-steps/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "trajectories": n_e2e},
            "measured_alu_peaks_gflops": peaks,
            "gpu_launches": int(prof["launches"]),
            "clocks": clocks,
            "forms": forms,
            "batched": batched,
            "paper_shape": paper,
            "gradient": gradient,
            "c3": c3,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(s)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def paper_shape(kbe, stream):
    """The paper's model-problem shape (two bands, 1-D ring of n_k = 1024,
    n = 500, Sec. 6 Tables I-II): one Sigma row and one collision row at
    t_500 on a synthetic (random) history of that shape; their cost does not
    depend on the values. Context for the paper's per-step times."""
    import torch
    nb, L, n = 2, (1024, 1), 500
    nk, blk = 1024, 4 * 1024
    ntri = (n + 1) * (n + 2) // 2
    g = torch.Generator(device="cuda").manual_seed(5)
    out = {"shape": "N_b=2, n_k=1024 (1-D), row n=500, one evaluation (P(EC)^2E does 3 per step)"}
    row = torch.randn((n + 1, 2, nb, nb, nk), dtype=torch.complex128, device="cuda", generator=g)
    sig = torch.empty_like(row)
    work = torch.empty(kbe.sigma_row_workspace(nb, L, n) // 16 + 1, dtype=torch.complex128, device="cuda")
    v = ki.pair_pattern(2)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    with torch.cuda.stream(stream):
        out["sigma_row_ms"] = timed(lambda: kbe.sigma_row(nb, L, v, n, 0.5, row, sig, work, stream=stream))
        for name, prec in (("fp64", 0), ("df64", 1), ("c64", 2)):
            H64 = torch.randn((ntri, 2, nb, nb, nk), dtype=torch.complex128, device="cuda", generator=g)
            esz = 8 if prec == 2 else 16
            H = torch.empty(H64.numel() * esz // 4, dtype=torch.float32, device="cuda")
            kbe.pack(prec, H64, H, ntri, blk, stream=stream)
            del H64
            I = torch.empty_like(row)
            w = torch.empty(kbe.collision_row_workspace(nb, L, n, prec) // 4 + 1, dtype=torch.float32,
                            device="cuda")
            out[f"collision_row_ms_{name}"] = timed(
                lambda: kbe.collision_row(nb, L, n, 0.02, H, sig, I, precision=prec, work=w, stream=stream))
            del H, I, w
            torch.cuda.empty_cache()
    return out


def gradient_form(kbe, stream, args, peaks):
    """c5: the gradient of L = sum_kb (n_kb(t_N) - n*_kb)^2 (n* ~ U(0,1), seed 4)
    with respect to the 512 Peierls samples A_i and U on c2's system: one
    forward trajectory, then kbe_backward, each timed with CUDA events on the
    handle's stream. The collision-row transposes are set against the FP64
    pipe (their flops: kbe_profile_stats.backward_sweep_flops)."""
    import torch
    s = ki.config("c2", nt=args.nt)
    nt = s.nt
    tgt = ki.targets(s.nk, s.nb, seed=4)
    g = kbe.KBE.from_system(s, stream=stream)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record(stream)
    g.step(nt)
    e[1].record(stream)
    nkb, _ = g.observables(nt)
    g.profile(True)
    dA, dU = g.backward(2.0 * (nkb - tgt))
    e[2].record(stream)
    e[2].synchronize()
    pb = g.profile_read()
    g.close()
    fwd, bwd = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    bm = pb["backward_ms"]
    achieved = pb["backward_sweep_flops"] / (bm[1] * 1e-3) / 1e9
    peak = peaks["fp64"]
    return {"workload": f"c5: c2's system, {nt} steps, loss sum (n_kb(t_N) - n*)^2, n* ~ U(0,1) seed 4; "
                        f"gradient w.r.t. {nt} A_i and U",
            "forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd,
            "phases_ms": {"recompute": bm[0], "collision_transposes": bm[1], "sigma_transposes": bm[2],
                          "update_and_h_transposes": bm[3]},
            "collision_transposes_roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                                              "unit": "GFLOP/s FP64", "frac": achieved / peak,
                                              "peak_source": "measured FP64 FMA throughput (kbe_measure_fma_peaks)"},
            "dL_dU": dU, "max_abs_dL_dA": float(np.abs(dA).max())}


def gradient_fd_check(args):
    """c5 gradient against central differences of the library's own forward
    (h = 1e-6) on U and 16 seeded A_i; prints one JSON line."""
    import dataclasses
    import torch
    import paper_2505_19467_gb300 as kbe
    torch.cuda.set_device(0)
    s = ki.config("c2", nt=args.nt)
    nt = s.nt
    tgt = ki.targets(s.nk, s.nb, seed=4)

    def loss(A=None, U=None):
        ss = dataclasses.replace(s, A=s.A if A is None else A, U=s.U if U is None else U)
        g = kbe.KBE.from_system(ss)
        g.step(nt)
        n_, _ = g.observables(nt)
        g.close()
        return float(((n_ - tgt) ** 2).sum())

    g = kbe.KBE.from_system(s)
    g.step(nt)
    nkb, _ = g.observables(nt)
    dA, dU = g.backward(2.0 * (nkb - tgt))
    g.close()
    h = 1e-6
    idx = [int(i) for i in np.sort(np.random.default_rng(4).choice(nt, 16, replace=False))]
    fd, ad = [], []
    for i in idx:
        e = np.zeros(nt)
        e[i] = h
        fd.append((loss(A=s.A + e) - loss(A=s.A - e)) / (2 * h))
        ad.append(float(dA[i]))
    fd.append((loss(U=s.U + h) - loss(U=s.U - h)) / (2 * h))
    ad.append(dU)
    fd, ad = np.array(fd), np.array(ad)
    print(json.dumps({"check": "c5 gradient vs central differences (h = 1e-6)", "steps": nt,
                      "A_indices": idx, "adjoint": ad.tolist(), "fd": fd.tolist(),
                      "normwise_rel_err": float(np.linalg.norm(ad - fd) / np.linalg.norm(fd)),
                      "max_rel_err": float(np.max(np.abs(ad - fd)) / np.max(np.abs(fd)))}), flush=True)


def c3_form(kbe, stream, peaks):
    """c3 (N_b = 8, 16x16, U = 1.5, A0 = 0.5), the mixed forms' showcase: the
    full 512-step trajectory once per form (FP64 history 69 GB, C64 34 GB),
    each timed with CUDA events on the library's stream with the sweep
    profiled, and each reduced form's error against the FP64 trajectory."""
    import torch
    s = ki.config("c3")
    nt = s.nt
    out = {"workload": f"c3: N_b=8, 16x16 mesh (n_k=256), N_t={nt}, dt=0.02, U=1.5, Peierls A0=0.5, "
                       "P(EC)^2E, one full trajectory per form"}
    ref = None
    for form in FORMS:
        g = kbe.KBE.from_system(s, stream=stream, precision=kbe.PRECISIONS[form])
        g.step(8)   # warm-up (kernels loaded, attributes set)
        g.reset()
        torch.cuda.synchronize()
        g.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(nt)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        prof = g.profile_read()
        g.profile(False)
        nkb, sc = g.observables_all()
        g.close()
        torch.cuda.empty_cache()
        o = {"ms": ms, "time_steps_per_s": nt / ms * 1e3, "roofline": roofline(prof, form, ms / 1e3, peaks)}
        if ref is None:
            ref = (nkb, sc)
        else:
            o["speedup_vs_fp64"] = out["fp64"]["ms"] / ms
            o["max_abs_err_density"] = float(np.abs(nkb - ref[0]).max())
            o["max_rel_err_energy"] = float(np.abs(sc[:, 5] - ref[1][:, 5]).max() / np.abs(ref[1][:, 5]).max())
            o["max_rel_err_N"] = float(np.abs(sc[:, 0] - ref[1][:, 0]).max() / abs(ref[1][0, 0]))
        out[form] = o
    return out


BATCH_WINDOW = 128   # timed steps per system (every drawn N_t is >= 256)
BATCH_MARGIN = 8 << 30


def batch_admission(nbs, need, budget):
    """The order the batched form hands its systems to kbe_batch_create (the
    smallest system of each N_b class first, then the others ascending by
    bytes) and what that call admits under `budget` bytes (its rule: in order,
    each system that still fits). Returns (order, admitted indices, bytes)."""
    n = len(nbs)
    first = [min((i for i in range(n) if nbs[i] == c), key=lambda i: (need[i], i)) for c in sorted(set(nbs))]
    order = first + sorted((i for i in range(n) if i not in first), key=lambda i: (need[i], i))
    admitted, used = [], 0
    for i in order:
        if used + need[i] <= budget:
            admitted.append(i)
            used += need[i]
    return order, admitted, used


def batched_form(kbe, stream, args):
    """The uneven 64-system draw (seed 3: N_b in {2, 4, 6, 8, 12, 16}, 4x4..12x12
    meshes, N_t in [256, 1024]; FP64). Admission: systems allocated at their
    drawn N_t, taken while they fit in device memory (free memory less a margin),
    in the order: the smallest system of each N_b class, then the others
    ascending by size. Each distinct (N_b, mesh) shape is autotuned first
    (kbe_autotune on a handle of that shape over the window's rows). Every
    admitted system then runs its first BATCH_WINDOW steps (a truncation of its
    drawn N_t, reported per system), three ways: the stream form (one stream per
    system), the persistent form (stage-major steps, the sweeps of all systems in
    one launch per N_b class), and one system after another. One untimed pass,
    one timed pass each (a pass is reset + the window, all systems)."""
    import torch
    systems = ki.batched(64)
    need = [kbe.memory_bytes(kbe.system_config(x)) for x in systems]
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, tot = torch.cuda.mem_get_info()
    budget = max(0, free - BATCH_MARGIN)
    order, expect, used = batch_admission([x.nb for x in systems], need, budget)
    tiles = {}
    for i in expect:           # one tuning per distinct shape (the table is per shape and row bucket)
        x = systems[i]
        key = f"N_b={x.nb} {x.L[0]}x{x.L[1]}"
        if key in tiles:
            continue
        g = kbe.KBE.from_system(x, nt_max=BATCH_WINDOW, stream=stream)
        g.reset()
        t = g.autotune()
        g.close()
        tiles[key] = [int(v) for v in t if v != 0]
    sel = [systems[i] for i in order]
    b = kbe.KBEBatch(sel, budget_bytes=budget, stream=stream)
    adm = [order[q] for q in range(len(order)) if b.admitted[q]]
    runs = [b.systems[q] for q in range(len(order)) if b.admitted[q]]
    units = sum(min(BATCH_WINDOW, systems[i].nt) for i in adm)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def batch_pass():
        b.reset()
        b.step(BATCH_WINDOW)
        b.synchronize()

    def sequential_pass():
        for g in runs:
            g.reset()
            g.step(BATCH_WINDOW)
            g.synchronize()

    t_stream = timed(batch_pass)
    b.set_persistent(True)
    l0 = b.sweep_launches()
    t_pers = timed(batch_pass)
    launches = (b.sweep_launches() - l0) // 2
    b.set_persistent(False)
    t_seq = timed(sequential_pass)
    b.close()
    return {"workload": f"uneven 64-system draw (seed 3), FP64: {len(adm)} systems admitted at their drawn N_t "
                        f"({used / 1e9:.1f} GB of {tot / 1e9:.1f} GB), each timed over its first "
                        f"{BATCH_WINDOW} steps",
            "value": units / t_pers, "unit": "time-steps/s (summed over systems)",
            "persistent_value": units / t_pers, "stream_value": units / t_stream,
            "sequential_value": units / t_seq,
            "persistent_speedup_vs_sequential": t_seq / t_pers,
            "persistent_speedup_vs_stream": t_stream / t_pers,
            "stream_speedup_vs_sequential": t_seq / t_stream,
            "persistent_sweep_launches_per_pass": int(launches),
            "admitted": [{"system": i, "N_b": systems[i].nb, "mesh": f"{systems[i].L[0]}x{systems[i].L[1]}",
                          "drawn_N_t": systems[i].nt, "steps_timed": min(BATCH_WINDOW, systems[i].nt)}
                         for i in adm],
            "not_admitted": sorted(set(range(len(systems))) - set(adm)),
            "autotuned_l_split_targets_per_row_bucket": tiles,
            "full_64_system_fp64_bytes": int(sum(need)), "device_bytes": int(tot),
            "truncation": f"every admitted system runs steps 1..{BATCH_WINDOW} of its drawn N_t "
                          "(allocation and admission at the drawn N_t)"}


class OracleSampler:
    """Times the FP64 oracle, as it stands, at sampled rows n of a trajectory of
    system s: one row evaluation (Sigma row n + collision row, the code path of
    its stepper) and one row update, on a random history of the trajectory's
    shape (costs do not depend on the values). The trajectory time is then
    integrated: sum over n = 1..N_t of 3 evaluations + 3 updates (P(EC)^2E),
    with the evaluation time fitted as a + b (n+1) + c (n+1)^2 (Sigma is O(n),
    the collision row O(n^2)) and the update as a + b (n+1)."""

    def __init__(self, s, nmax, threads=None):
        import oracle
        self.oracle, self.s = oracle, s
        if threads:
            oracle.oracle.set_threads(int(threads))
        self.threads = oracle.oracle.threads()
        nk, nb = s.nk, s.nb
        ntri = (nmax + 1) * (nmax + 2) // 2
        rng = np.random.default_rng(7)
        base = ki.random_blocks(rng, (256, nk, nb, nb))
        self.Hl = np.empty((ntri, nk, nb, nb), np.complex128)
        self.Hg = np.empty_like(self.Hl)
        for a in range(0, ntri, 256):
            m = min(256, ntri - a)
            self.Hl[a:a + m] = base[:m]
            self.Hg[a:a + m] = base[::-1][:m]
        h = ki.random_blocks(rng, (nk, nb, nb))
        h = 0.5 * (h + np.conj(np.swapaxes(h, 1, 2)))
        self.props = oracle.propagators(nb, nk, s.dt, h)
        self.row = ki.random_blocks(rng, (nmax + 1, nk, nb, nb))
        self.samples = []   # (n, evaluation s, update s)

    def sample(self, n):
        s, o = self.s, self.oracle
        t0 = time.perf_counter()
        o.evaluate_row_on(s.nb, s.L, s.v, s.U, n, s.dt, self.Hl, self.Hg)
        t1 = time.perf_counter()
        U, V, W, lam = self.props
        r = self.row
        o.update_row(s.nb, s.nk, n, s.dt, 0.5, U, V, W, lam, r[:n], r[:n], r[:n], r[:n], r[:n + 1], r[:n + 1])
        t2 = time.perf_counter()
        self.samples.append((n, t1 - t0, t2 - t1))
        return t2 - t0

    def trajectory_seconds(self, nt):
        x = np.array([n + 1.0 for n, _, _ in self.samples])
        e = np.array([t for _, t, _ in self.samples])
        u = np.array([t for _, _, t in self.samples])
        ce = np.polyfit(x, e, min(2, len(x) - 1))
        cu = np.polyfit(x, u, min(1, len(x) - 1))
        xs = np.arange(2, nt + 2, dtype=float)     # n + 1 for n = 1..nt
        return float(np.sum(3 * np.maximum(np.polyval(ce, xs), 0) + 3 * np.maximum(np.polyval(cu, xs), 0)))


def sweep_row_study(kbe, row, names, reps=5, only_forms=None, only_ti=None):
    """The collision sweep (Sigma row -> coefficient rows -> sweep -> I row) alone at
    row `row` on random history of each workload's shape: every launch choice of
    the C64 form (the single-read tile form at TI = 32, 64, 128 rows per work item;
    the per-column staged / blocked kernel at its default split), the tensor-core
    sweep of the split-FP16 form at TI = 32, 64 (and 128 at N_b = 4) rows per
    panel and, at c2, the FP64 and DF64 forms. Time per launch from CUDA events on the launching stream
    (after 2 untimed launches; the history is larger than L2), algorithmic
    bytes (the triangle read once in the form's storage, the Sigma row read and
    the I row written in FP64) per time, and the fraction of the HBM peak."""
    import torch
    hbm, hsrc = hbm_peak()
    stream = torch.cuda.Stream()
    out = {"row": row, "hbm_peak_gbs": hbm, "hbm_peak_source": hsrc}
    for name in names:
        s = ki.config(name)
        nb, L, nk = s.nb, s.L, s.nk
        n = min(row, s.nt - 1)
        blk = nb * nb * nk
        ntri = (n + 1) * (n + 2) // 2
        g = torch.Generator(device="cuda").manual_seed(11)
        sig = torch.randn((n + 1, 2, nb, nb, nk), dtype=torch.complex128, device="cuda", generator=g)
        I = torch.empty_like(sig)
        res = {"shape": f"N_b={nb}, n_k={nk}, row n={n}"}
        forms = ["f16x2", "c64", "fp64", "df64"] if name == "c2" else ["f16x2", "c64"]
        if only_forms:
            forms = [f for f in forms if f in only_forms]
        for form in forms:
            prec = kbe.PRECISIONS[form]
            esz = 8 if form in ("c64", "f16x2") else 16
            if form == "f16x2":   # finite random halves (hi and lo parts of every real), padded rows
                H = torch.randn(kbe.history_bytes(nb, L, n, prec) // 2, dtype=torch.float16, device="cuda",
                                generator=g)
            else:
                H = torch.randn(ntri * 2 * blk * esz // 4, dtype=torch.float32, device="cuda", generator=g)
            w = torch.empty(kbe.collision_row_workspace(nb, L, n, prec) // 4 + 1, dtype=torch.float32, device="cuda")
            alg = 2.0 * blk * (ntri * esz + 2.0 * (n + 1) * 16.0)
            choices = [("default", 0)]
            if form == "f16x2":   # bulk copies of row groups, or loader warps (odd choice)
                choices = [(f"tc_TI{t}", -t) for t in (32, 64, 128) if nb == 4 or t <= 64]
                choices += [(f"tc_TI{t}_loader_warps", -(t + 1)) for t in (32, 64, 128) if nb == 4 or t <= 64]
            if form == "c64":
                choices = [("per_column", 12 if nb >= 4 else 8)]
                if nb in (2, 4, 8):
                    choices += [(f"tile_TI{t}", -t) for t in (32, 64, 128)]
                    choices += [(f"tile_TI{t}_one_unit_per_cta", -(t + 1)) for t in (32, 64, 128)]
            if only_ti:
                choices = [(lb, c) for lb, c in choices if c in (-only_ti, -(only_ti + 1))] or choices[:1]
            for label, choice in choices:
                if choice:
                    kbe.set_sweep_choice(nb, L, prec, choice)
                try:
                    with torch.cuda.stream(stream):
                        for _ in range(2):
                            kbe.collision_row(nb, L, n, s.dt, H, sig, I, precision=prec, work=w, stream=stream)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        for _ in range(reps):
                            kbe.collision_row(nb, L, n, s.dt, H, sig, I, precision=prec, work=w, stream=stream)
                        e1.record(stream)
                        e1.synchronize()
                    ms = e0.elapsed_time(e1) / reps
                    gbs = alg / (ms * 1e-3) / 1e9
                    res[f"{form}_{label}"] = {"ms": ms, "alg_gbs": gbs, "hbm_frac": gbs / hbm}
                finally:
                    if choice:
                        kbe.set_sweep_choice(nb, L, prec, 0)
            res[f"{form}_alg_bytes"] = alg
            del H, w
            torch.cuda.empty_cache()
        out[name] = res
        del sig, I
        torch.cuda.empty_cache()
    return out


def cpu_baseline(s):
    """The FP64 oracle on the host cores (all of them, and one thread): its
    whole-trajectory c2 rate integrated from timed rows across the trajectory."""
    import oracle
    full = OracleSampler(s, max(ORACLE_ROWS))
    for n in ORACLE_ROWS:
        full.sample(n)
    t_all = full.trajectory_seconds(s.nt)
    cores = full.threads
    del full
    one = OracleSampler(s, max(ORACLE_ROWS_1T), threads=1)
    for n in ORACLE_ROWS_1T:
        one.sample(n)
    t_one = one.trajectory_seconds(s.nt)
    oracle.oracle.set_threads(cores)
    return {"value": s.nt / t_all, "unit": "time-steps/s", "cores": cores, "kind": "oracle",
            "method": "extrapolated",
            "sample": f"one row evaluation (Sigma + collision row) and one row update timed at rows "
                      f"{ORACLE_ROWS} of c2 on random history; the {s.nt}-step trajectory integrated "
                      "from a quadratic fit in n (3 evaluations + 3 updates per step)",
            "trajectory_seconds": t_all,
            "one_thread": {"value": s.nt / t_one, "cores": 1, "trajectory_seconds": t_one,
                           "sample": f"rows {ORACLE_ROWS_1T}, same fit"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    s = ki.config("c2", nt=args.nt)
    rows = [n for n in ORACLE_ROWS if n <= s.nt - 1] or [s.nt - 1]
    smp = OracleSampler(s, max(rows))
    for _ in range(args.warmup):
        smp.sample(min(31, rows[0]))
    smp.samples.clear()
    total = 0.0
    for k in range(args.steps):
        total += smp.sample(rows[k % len(rows)])
    t_traj = smp.trajectory_seconds(s.nt)
    value = s.nt / t_traj
    line = {
        "metric": METRIC, "value": value, "unit": "time-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded c2 system, kbe_inputs)", "impl": "reference",
        "config": {"workload": WORKLOAD,
                   "bench_step": "oracle: one row evaluation (Sigma + collision row) and one row update "
                                 f"at a sampled row n (cycling over {rows}) on random history of c2's shape",
                   "value": f"the {s.nt}-step trajectory rate integrated from the timed rows "
                            "(3 evaluations + 3 updates per step, quadratic fit in n): extrapolated",
                   "n_corr": 2},
        "cpu_baseline": {"value": value, "unit": "time-steps/s", "cores": smp.threads, "kind": "oracle",
                         "method": "extrapolated", "trajectory_seconds": t_traj,
                         "sample": f"{args.steps} timed rows of c2 cycling over {rows}"},
        "e2e": {"value": value, "unit": "time-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.gradient_fd:
        if rank == 0:
            gradient_fd_check(args)
        return
    if args.sweep_row is not None:
        if rank == 0:
            import torch
            import paper_2505_19467_gb300 as kbe
            torch.cuda.set_device(local)
            print(json.dumps({"sweep_row": sweep_row_study(
                kbe, args.sweep_row, args.sweep_shapes.split(","),
                only_forms=args.sweep_forms.split(",") if args.sweep_forms else None, only_ti=args.sweep_ti)}),
                  flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
