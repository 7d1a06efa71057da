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
--impl reference times the FP64 CPU oracle on the host cores on a bounded
prefix of the same workload. The line also carries the reverse mode on the
same system ("gradient": forward + kbe_backward for dL/dA_i, dL/dU);
--gradient-fd checks that gradient by central differences instead.
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
# Roofline denominators of the sweep (the dominant kernel), per arithmetic form,
# from unit counts and the 2.07 GHz maximum SM clock (GB300, 152 SMs):
#  fp64: FP64 pipe, 2 DFMA/clk/SM (nominal 1.25 TFLOP/s; a probe measured 1.195)
#  df64: FP32 issue, 128 lanes/clk/SM, 6 FP32 instructions per double-float
#        flop (a complex multiply-add is 4 products x 12 instructions = 8 flop)
#  c64 : FP32 FMA, 128 lanes x 2 flop/clk/SM (a probe measured 73.2 TFLOP/s)
PEAKS = {
    "fp64": (152 * 2 * 2 * 2.07, "GFLOP/s FP64",
             "FP64 pipe: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)"),
    "df64": (152 * 128 * 2.07 / 6, "GFLOP/s FP64-equivalent (double-float)",
             "FP32 issue: 152 SM x 128 lanes x 2.07 GHz / 6 FP32 instructions per double-float flop"),
    "c64": (152 * 128 * 2 * 2.07, "GFLOP/s FP32",
            "FP32 FMA: 152 SM x 128 lanes x 2 flop x 2.07 GHz"),
}
# DRAM traffic of the sweep per launch as a multiple of its algorithmic bytes,
# from ncu (dram__bytes_read.sum + dram__bytes_write.sum) at row 501 of the
# full c2 run, all three forms (profiles/sweep_c2_n501_dram.md); traffic grows
# with the triangle like the algorithmic bytes, so the average launch is
# scaled by the same factor.
TRAFFIC_RATIO = {"fp64": 2.00, "df64": 2.77, "c64": 1.87}
DTYPES = {"fp64": "f64", "df64": "df64 (f32 hi/lo pairs; everything but the sweep f64)",
          "c64": "c64/f32 history + sweep (everything else f64)"}
ORACLE_PREFIX = 40


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--nt", type=int, default=None, help="truncate N_t (testing only)")
    p.add_argument("--precision", default="fp64", choices=["fp64", "df64", "c64"],
                   help="history storage / sweep arithmetic of the headline value (fp64 meets "
                        "the 1e-10 bar; df64 / c64 are the reduced-storage forms)")
    p.add_argument("--forms", default="all", choices=["all", "none", "gradient", "batched"],
                   help="also time the other storage forms (speedup and error vs the headline), "
                        "the batched and paper-shaped forms and the gradient; 'gradient' or "
                        "'batched': only that one")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true",
                   help="skip kbe_autotune (the sweep's l-split chosen by timing before the timed region)")
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


def roofline(prof, precision, t_dev):
    """achieved: the method's algorithmic flops (24 n^2 N_b^3 n_k per sweep, the
    G^> form of Eq. 6) over the summed sweep event time; the kernel executes
    2/3 of them (the I^<, I^> - I^< form), reported as achieved_executed / frac_executed."""
    sweep_s = prof["sweep_ms"] / 1e3
    achieved = prof["sweep_flops"] / sweep_s / 1e9 if sweep_s > 0 else 0.0
    executed = prof["sweep_flops_executed"] / sweep_s / 1e9 if sweep_s > 0 else 0.0
    peak, punit, psrc = PEAKS[precision]
    nl = max(1, prof["sweep_launches"])
    alg_bytes = prof["sweep_bytes"] / nl
    return {"kernel": "collision sweep (a2)", "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": punit, "frac": achieved / peak,
            "traffic": TRAFFIC_RATIO[precision] * alg_bytes, "traffic_unit": "bytes per launch",
            "algorithmic_bytes_per_launch": alg_bytes, "peak_source": psrc,
            "achieved_executed": executed, "frac_executed": executed / peak,
            "launches": prof["sweep_launches"],
            "sweep_share_of_step": sweep_s / t_dev if t_dev > 0 else None,
            "hbm_gbs_achieved": prof["sweep_bytes"] / sweep_s / 1e9 if sweep_s > 0 else 0.0}


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
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
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
    e2e_value = units * world / times[1]

    # ---- the reduced-storage forms on the same workload (speedup, error) ----
    forms = {}
    for form in ([] if args.forms != "all" else [f for f in ("fp64", "df64", "c64") if f != args.precision]):
        gf = kbe.KBE.from_system(s, stream=stream, precision=kbe.PRECISIONS[form])
        if not args.no_autotune:
            tuned[form] = [int(x) for x in gf.autotune() if x]
        tf, pf, _ = time_trajectories(gf, nt, args.steps, args.warmup, stream, None, dist)
        nkb_f, sc_f = gf.observables_all()
        gf.close()
        escale = np.abs(ref_obs[:, 5]).max()
        forms[form] = {"value": units / tf, "speedup_vs_" + args.precision: (units / tf) / (units / t_dev),
                       "max_abs_err_density": float(np.abs(nkb_f - ref_nkb).max()),
                       "max_rel_err_energy": float(np.abs(sc_f[:, 1:] - ref_obs[:, 1:]).max() / escale),
                       "max_rel_err_N": float(np.abs(sc_f[:, 0] - ref_obs[:, 0]).max() / abs(ref_obs[0, 0])),
                       "dtype": DTYPES[form], "roofline": roofline(pf, form, tf)}

    # ---- batched form: uneven systems together vs one after another ----------
    batched = paper = gradient = c3 = None
    if args.forms in ("all", "batched"):
        batched = batched_form(kbe, stream, args)
    if args.forms == "all":
        paper = paper_shape(kbe, stream)
        c3 = c3_form(kbe, stream)
    if args.forms in ("all", "gradient"):
        gradient = gradient_form(kbe, stream, args)

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
            "roofline": roofline(prof, args.precision, t_dev),
            "e2e": {"value": e2e_value, "unit": "time-steps/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(prof["launches"]),
            "clocks": clocks,
            "forms": forms,
            "batched": batched,
            "paper_shape": paper,
            "gradient": gradient,
            "c3_prefix": c3,
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


def gradient_form(kbe, stream, args):
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
    peak = PEAKS["fp64"][0]
    return {"workload": f"c5: c2's system, {nt} steps, loss sum (n_kb(t_N) - n*)^2, n* ~ U(0,1) seed 4; "
                        f"gradient w.r.t. {nt} A_i and U",
            "forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd,
            "phases_ms": {"recompute": bm[0], "collision_transposes": bm[1], "sigma_transposes": bm[2],
                          "update_and_h_transposes": bm[3]},
            "collision_transposes_roofline": {"bound": "fp64", "achieved": achieved, "peak": peak,
                                              "unit": "GFLOP/s FP64", "frac": achieved / peak},
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


C3_PREFIX = 96


def c3_form(kbe, stream):
    """c3 (N_b = 8, 16x16, U = 1.5, A0 = 0.5), the mixed forms' showcase, on its
    first C3_PREFIX steps (the full FP64 run takes ~6 min): each form's
    trajectory time (CUDA events) and its error against the FP64 trajectory."""
    import torch
    s = ki.config("c3", nt=C3_PREFIX)
    out = {"workload": f"c3: N_b=8, 16x16 mesh (n_k=256), first {C3_PREFIX} of 512 steps, dt=0.02, "
                       "U=1.5, Peierls A0=0.5, P(EC)^2E"}
    ref = None
    for form in ("fp64", "df64", "c64"):
        g = kbe.KBE.from_system(s, stream=stream, precision=kbe.PRECISIONS[form])
        g.step(8)   # warm-up (kernels loaded, attributes set)
        g.reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(C3_PREFIX)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        nkb, sc = g.observables_all()
        g.close()
        o = {"ms": ms, "time_steps_per_s": C3_PREFIX / ms * 1e3}
        if ref is None:
            ref = (nkb, sc)
        else:
            o["speedup_vs_fp64"] = out["fp64"]["ms"] / ms
            o["max_abs_err_density"] = float(np.abs(nkb - ref[0]).max())
            o["max_rel_err_energy"] = float(np.abs(sc[:, 5] - ref[1][:, 5]).max() / np.abs(ref[1][:, 5]).max())
        out[form] = o
    return out


BATCH_N, BATCH_NT = 16, 64


def batched_form(kbe, stream, args):
    """The first 16 systems of the uneven 64-system draw (N_b 2..16, 4x4..12x12,
    each truncated to 64 steps), advanced together (kbe_batch_*, one stream
    per system) and one after another on one stream; FP64."""
    import torch
    systems = ki.batched(64)
    full = sum(kbe.memory_bytes(kbe.system_config(x)) for x in systems)
    sel = systems[:BATCH_N]
    nts = [min(BATCH_NT, x.nt) for x in sel]
    units = sum(nts)
    b = kbe.KBEBatch(sel, nt_max=nts, stream=stream)
    for _ in range(max(1, args.warmup)):
        b.reset()
        b.step(BATCH_NT)
    b.synchronize()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.reset()
        b.step(BATCH_NT)
    b.synchronize()
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t0) / args.steps
    b.set_graphs(True)            # each system replays its 64 steps as one captured graph
    for _ in range(max(1, args.warmup)):
        b.reset()
        b.step(BATCH_NT)
    b.synchronize()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.reset()
        b.step(BATCH_NT)
    b.synchronize()
    torch.cuda.synchronize()
    t_graph = (time.perf_counter() - t0) / args.steps
    b.close()
    singles = [kbe.KBE.from_system(x, nt_max=nt, stream=stream) for x, nt in zip(sel, nts)]
    for g, nt in zip(singles, nts):
        g.reset()
        g.step(nt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for g, nt in zip(singles, nts):
            g.reset()
            g.step(nt)
    for g in singles:
        g.synchronize()
    torch.cuda.synchronize()
    t_seq = (time.perf_counter() - t0) / args.steps
    for g in singles:
        g.close()
    free, tot = torch.cuda.mem_get_info()
    return {"workload": f"first {BATCH_N} of the 64 uneven systems (seed 3), each truncated to "
                        f"{BATCH_NT} steps; N_b {sorted(set(x.nb for x in sel))}",
            "value": units / t_batch, "unit": "time-steps/s (summed over systems)",
            "sequential_value": units / t_seq, "speedup_vs_sequential": t_seq / t_batch,
            "graphs_value": units / t_graph, "graphs_speedup_vs_sequential": t_seq / t_graph,
            "full_64_system_fp64_bytes": int(full), "device_bytes": int(tot),
            "note": "the full 64-system draw needs this many bytes in FP64 and does not fit; "
                    "kbe_batch_create admits systems in order within the device budget"}


def cpu_baseline(s, prefix=ORACLE_PREFIX):
    """The FP64 oracle, as it stands, on the host cores: first `prefix` steps of c2."""
    import oracle
    o = oracle.Oracle(s, nt_max=prefix)
    t0 = time.perf_counter()
    o.step(prefix)
    dt = time.perf_counter() - t0
    return {"value": prefix / dt, "unit": "time-steps/s", "cores": oracle.oracle.threads(),
            "kind": "oracle",
            "sample": f"first {prefix} of {s.nt} steps of c2 (steps cost O(n^2); later steps are slower)",
            "seconds": dt}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    s = ki.config("c2", nt=args.nt)
    prefix = min(ORACLE_PREFIX // 2, s.nt)
    for _ in range(args.warmup):
        o = oracle.Oracle(s, nt_max=prefix)
        o.step(min(4, prefix))
    times = []
    for _ in range(args.steps):
        o = oracle.Oracle(s, nt_max=prefix)
        t0 = time.perf_counter()
        o.step(prefix)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = prefix * args.steps / total
    line = {
        "metric": METRIC, "value": value, "unit": "time-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded c2 system, kbe_inputs)", "impl": "reference",
        "config": {"workload": WORKLOAD, "bench_step": f"oracle: first {prefix} of {s.nt} time steps",
                   "n_corr": 2},
        "cpu_baseline": {"value": value, "unit": "time-steps/s", "cores": oracle.oracle.threads(),
                         "kind": "oracle", "sample": f"first {prefix} steps of c2 per bench step"},
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
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
