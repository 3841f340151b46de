"""Benchmark of the mode-space Langevin step on one GB300.

Workload: 4096 independent 256-bp dsDNA chains, FP32 state, dt = 15.9 ps
(dtau ~ 100, Table 2), equilibrium-sampled starts, zero shear, per-chain
Philox streams.  A bench "step" is one Langevin step of the whole batch
(inverse transform, bond force, bead noise, forward transform, mode update).  The K
timed steps run as sfp_step calls of --steps-per-call steps (20; one fused
launch each) with the L2 flushed before every call; the one-step-per-call
figure is reported beside it.

Prints one JSON line (rank 0).  Metric: bead-timesteps/s (chains x beads x
steps / s); simulated ns/s per chain is reported beside it.
  --impl reference   time the FP64 CPU oracle on the host cores instead
  --precision bf16   (default) fused step, transforms as three BF16 tcgen05
                     passes (hi/lo split, FP32 accumulate; SFP_MIXED_BF16)
  --precision tf32   the same with three TF32 passes (SFP_FP32)
  --precision simt   the plain FP32 CUDA-core path (no tensor cores)
  --path staged      time the per-stage tcgen05 kernels instead of the fused step
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
C_CHAINS, M_BEADS, DT_PS = 4096, 256, 15.9
WORKLOAD = "dsDNA 4096 chains x 256 bp, FP32 state, dt 15.9 ps, equilibrium starts, no shear"
METRIC, UNIT = "bead-timesteps/s", "bead-steps/s"
L2_FLUSH_BYTES = 256 << 20
# the scaled time unit c = T* (1 - 2 nu)^2 a^2 xi / kT (Eq. g2) from the printed
# dsDNA values (T* = 0.034, nu = 0.35, a^2 xi / kT = 52.0 ps): the oracle legs
# take their step from it, not from the library
C_PS = 0.034 * (1.0 - 2.0 * 0.35) ** 2 * 52.0
PREC_NAME, DTYPE = {}, {}     # filled once the library is imported


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--steps-per-call", type=int, default=20,
                    help="Langevin steps per sfp_step call (one fused launch); L2 is flushed between calls")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "bf16x2", "tf32", "tc", "simt"])
    ap.add_argument("--path", default="fused", choices=["fused", "staged"])
    ap.add_argument("--workload", default="batch", choices=["batch", "serving", "precision", "uneven"])
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="arrival window of the serving workload (config 5 runs 600 s; 60 s keeps the bench short)")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-budget-mb", type=float, default=40e3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-512", action="store_true", help="skip the 16384 x 512-bp legs")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the serving, uneven-batch and single-chain FP64 sub-keys of the default line")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def cpu_model() -> str:
    """Host CPU model as lscpu reports it (vendor and model name), else the platform string."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        f = dict(line.split(":", 1) for line in out.splitlines() if ":" in line)
        parts = [f.get(k, "").strip() for k in ("Vendor ID", "Model name")]
        name = " ".join(p for p in parts if p)
        if name:
            return name
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


# ------------------------------------------------------------------ oracle (CPU)

def cpu_oracle_rate(n_chains: int, n_steps: int, seed: int = 1, nthreads: int = 0):
    """Time the FP64 oracle on a sample of the workload (all host threads, or nthreads)."""
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    m = O.Model(M_BEADS, dtau=DT_PS / C_PS)
    R = np.stack([m.equilibrium_start(seed, j) for j in range(n_chains)])
    jobs = np.arange(n_chains)
    m.run_modes(R, seed, jobs, 0, 1, nthreads=nthreads)    # warm (page-in, thread pool)
    t0 = time.perf_counter()
    m.run_modes(R, seed, jobs, 0, n_steps, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return n_chains * M_BEADS * n_steps / dt, dt, (nthreads or O.threads())


def run_reference(args, rank):
    if rank != 0:
        return
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    m = O.Model(M_BEADS, dtau=DT_PS / C_PS)
    sample = 32
    R = np.stack([m.equilibrium_start(1, j) for j in range(sample)])
    jobs = np.arange(sample)
    for s in range(args.warmup):
        R = m.run_modes(R, 1, jobs, s, 1)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        R = m.run_modes(R, 1, jobs, args.warmup + s, 1)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = sample * M_BEADS * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "chains_per_gpu": C_CHAINS, "beads": M_BEADS, "dt_ps": DT_PS,
                   "dtau": DT_PS / C_PS, "precision": "FP64 oracle (CPU)",
                   "sample": f"{sample} of {C_CHAINS} chains per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"{sample} chains x 256 beads x {args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    def __init__(self, index: int):
        self.proc = None
        self.path = None
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.proc = subprocess.Popen([exe, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                      "-i", str(index), "-lms", "100"],
                                     stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm

def run_native(args, rank, world, local):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import paper_1411_3487_gb300 as sfp
    from paper_1411_3487_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    _names(sfp)
    DTYPE.update({sfp.SFP_MIXED_BF16: "f32 (bf16x3 transforms)", sfp.SFP_FP32: "f32 (tf32x3 transforms)",
                  sfp.SFP_MIXED_BF16_2: "f32 (bf16x2 transforms, tables rounded to bf16)", sfp.SFP_FP32_SIMT: "f32"})
    precision = {"bf16": sfp.SFP_MIXED_BF16, "bf16x2": sfp.SFP_MIXED_BF16_2, "tf32": sfp.SFP_FP32, "tc": sfp.SFP_FP32,
                 "simt": sfp.SFP_FP32_SIMT}[args.precision]
    tensor = precision in (sfp.SFP_FP32, sfp.SFP_MIXED_BF16, sfp.SFP_MIXED_BF16_2)
    # weak scaling: every rank owns its own 4096 chains (disjoint job ids)
    from paper_1411_3487_gb300 import shard
    chains = [{"n_beads": M_BEADS, "dt_ps": DT_PS, "job_id": j}
              for j in shard.job_range(rank, world, world * C_CHAINS)]

    path = sfp.SFP_PATH_FUSED if args.path == "fused" else sfp.SFP_PATH_STAGED
    if precision == sfp.SFP_FP32_SIMT:
        path = sfp.SFP_PATH_STAGED

    def timed_steps(prec, pth, steps, warmup, with_clocks, per_call=1, stages=True, noise=None):
        """`steps` timed Langevin steps as sfp_step calls of `per_call` steps,
        the L2 flushed before every call; returns per-call times (ms).  With
        `stages`, per-stage CUDA events are recorded inside the calls (which runs
        the staged path's noise kernel in line instead of beside the inverse
        transform); without, the kernel times come from a second, untimed pass."""
        b = sfp.Batch(chains, seed=1, precision=prec, stream=stream)
        b.set_path(pth)
        if noise is not None:
            b.set_noise(noise)
        b.init_equilibrium(0)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        for _ in range(warmup):
            b.step(per_call)
            flush.zero_()
        torch.cuda.synchronize()
        calls = [per_call] * (steps // per_call) + ([steps % per_call] if steps % per_call else [])
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in calls]
        launches0 = b.info()["launches"]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local) if with_clocks else None
        b.stage_timing(stages)                # per-stage CUDA events on the batch's stream
        for (e0, e1), n in zip(ev, calls):
            flush.zero_()                     # L2 flushed between timed calls
            e0.record(stream)
            b.step(n)
            e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop() if clk else None
        if world > 1:
            dist.barrier()
        launches = b.info()["launches"] - launches0
        if not stages:
            b.stage_timing(True)
            for n in calls:
                flush.zero_()
                b.step(n)
        kern = b.stage_times()
        b.stage_timing(False)
        ms = [a.elapsed_time(c) for a, c in ev]
        return b, ms, launches, clocks, kern

    spc = max(1, args.steps_per_call)
    b, ms, launches, clocks, kern = timed_steps(precision, path, args.steps, args.warmup, True, spc)
    tot_ms = float(sum(ms))
    if world > 1:
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    beads = C_CHAINS * M_BEADS
    value = world * beads * args.steps / (tot_ms * 1e-3)
    d = sfp.derive()
    dtau = DT_PS / d["c_ps"]
    ms_step = tot_ms / args.steps

    pk, how = peaks()
    if rank == 0:
        pk = dict(pk)
        pk["tf32_tflops"] = tf32_peak(torch)
    roof = roofline(kern, pk, how, precision, path, sfp)

    # sustained: 4 back-to-back calls of 100 steps, no flush at all (a long run)
    sustained = None
    if path == sfp.SFP_PATH_FUSED and tensor:
        per_call, calls = 100, 4
        b.step(per_call)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(calls):
            b.step(per_call)
        e1.record(stream)
        torch.cuda.synchronize()
        s_ms = e0.elapsed_time(e1)
        sustained = {"value": beads * per_call * calls / (s_ms * 1e-3), "unit": UNIT,
                     "ms_per_step": s_ms / (per_call * calls), "steps_per_call": per_call,
                     "l2": "not flushed between the steps of one call"}

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = end_to_end(sfp, b, torch, min(args.steps, 50))
    e64 = end_to_end(sfp, b, torch, min(args.steps, 50), f32=False)
    e2e["fp64_state"] = {k: e64[k] for k in ("value", "h2d_bytes_per_step", "d2h_bytes_per_step", "api")}

    plain = staged = other = single = modes = None
    if not args.no_plain and precision != sfp.SFP_FP32_SIMT:
        b.close()
        n_o = min(args.steps, 100)

        def leg(prec, pth, per_call, what, noise=None):
            staged_path = pth == sfp.SFP_PATH_STAGED
            _, ms_l, _, _, k_l = timed_steps(prec, pth, n_o, 3, False, per_call, stages=not staged_path,
                                             noise=noise)
            out = {"value": beads * n_o / (sum(ms_l) * 1e-3), "unit": UNIT, "ms_per_step": float(sum(ms_l) / n_o),
                   "steps_per_call": per_call, "kernels_us": k_l, "path": what}
            if staged_path:
                out["kernels_us_note"] = ("per-kernel times from a second pass with stage events, the noise "
                                          "kernel in line; the timed pass runs it beside the inverse transform")
                out["hbm"] = staged_hbm(k_l, pk)
            return out

        plain = leg(sfp.SFP_FP32_SIMT, sfp.SFP_PATH_STAGED, spc, "plain FP32 CUDA-core path")
        if path == sfp.SFP_PATH_FUSED:
            staged = leg(precision, sfp.SFP_PATH_STAGED, spc, "tcgen05 transforms, one kernel per stage (same precision)")
            # one step per call: every step a launch of its own after an L2 flush
            single = leg(precision, sfp.SFP_PATH_FUSED, 1, "fused step, one step per call and launch")
            # the fused step with the other tensor-core split, same workload and timing
            o_prec = sfp.SFP_FP32 if precision == sfp.SFP_MIXED_BF16 else sfp.SFP_MIXED_BF16
            other = leg(o_prec, sfp.SFP_PATH_FUSED, spc, "fused step")
            other.update({"precision": PREC_NAME[o_prec], "dtype": DTYPE[o_prec],
                          "roofline": roofline(other["kernels_us"], pk, how, o_prec, sfp.SFP_PATH_FUSED, sfp)})
            # the same fused step with mode-keyed noise (Z drawn per mode: no
            # projection, a third fewer MMAs; a different noise stream)
            modes = leg(precision, sfp.SFP_PATH_FUSED, spc, "fused step, mode-keyed noise (sfp_set_noise)",
                        noise=sfp.SFP_NOISE_MODES)
            us_m = modes["kernels_us"].get("inverse_us")
            if us_m and precision in (sfp.SFP_MIXED_BF16, sfp.SFP_FP32):
                peak_m = pk.get("bf16_tflops", 1900.0) if precision == sfp.SFP_MIXED_BF16 else (
                    pk.get("tf32_tflops") or pk.get("bf16_tflops", 1900.0) * 1.1 / 2.25)
                fl = 3 * 12.0 * M_BEADS * beads      # inverse 2M x 3 + forward force half 2M x 3, three passes
                modes["roofline_tensor"] = {"achieved": fl / (us_m * 1e-6) / 1e12, "peak": peak_m,
                                            "frac": fl / (us_m * 1e-6) / 1e12 / peak_m, "kernel_us": us_m,
                                            "flops_per_bead_step": 3 * 12 * M_BEADS}

    # the mixed-precision workload, 16384 chains x 512 bp at dt 15.9 ps: the fused
    # step (a tile per cluster of two CTAs) with each split, the staged
    # tensor-core kernels and the plain path; calls of 20 steps after an L2 flush
    big = None
    if rank == 0 and not args.no_512 and precision != sfp.SFP_FP32_SIMT:
        b.close()
        big = {"workload": "16384 chains x 512 bp, dt 15.9 ps, equilibrium starts, no shear", "chains": 16384,
               "beads": 512}
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        for name, prec, pth in (("fused_bf16x3", sfp.SFP_MIXED_BF16, sfp.SFP_PATH_FUSED),
                                ("fused_bf16x2", sfp.SFP_MIXED_BF16_2, sfp.SFP_PATH_FUSED),
                                ("fused_tf32x3", sfp.SFP_FP32, sfp.SFP_PATH_FUSED),
                                ("staged_bf16x3", sfp.SFP_MIXED_BF16, sfp.SFP_PATH_STAGED),
                                ("plain_fp32", sfp.SFP_FP32_SIMT, sfp.SFP_PATH_STAGED)):
            bb = sfp.Batch([{"n_beads": 512, "dt_ps": DT_PS, "job_id": j} for j in range(16384)], seed=1,
                           precision=prec, stream=stream)
            bb.set_path(pth)
            bb.init_equilibrium(0)
            calls = 5 if pth == sfp.SFP_PATH_FUSED else 2
            for _ in range(2):
                bb.step(20)
            torch.cuda.synchronize()
            t_ms = 0.0
            for _ in range(calls):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                bb.step(20)
                e1.record(stream)
                torch.cuda.synchronize()
                t_ms += e0.elapsed_time(e1)
            n = 20 * calls
            big[name] = {"value": 16384 * 512 * n / (t_ms * 1e-3), "unit": UNIT, "us_per_step": 1e3 * t_ms / n}
            if pth == sfp.SFP_PATH_FUSED:
                bf = prec in (sfp.SFP_MIXED_BF16, sfp.SFP_MIXED_BF16_2)
                passes = 2 if prec == sfp.SFP_MIXED_BF16_2 else 3
                big[name]["kernel"] = "k_fused_pair<%s>" % ({sfp.SFP_MIXED_BF16: "bf16", sfp.SFP_MIXED_BF16_2: "bf16, two passes"}.get(prec, "tf32"))
                big[name]["roofline_tensor_frac"] = (passes * 18 * 512 * 16384 * 512 / (1e-3 * t_ms / n)) / 1e12 / (
                    pk["bf16_tflops"] if bf else pk.get("tf32_tflops") or pk["bf16_tflops"] * 1.1 / 2.25)
            elif prec == sfp.SFP_MIXED_BF16:
                # per-kernel times of the staged step at this size (stage events, noise in line)
                bb.stage_timing(True)
                for _ in range(calls):
                    flush.zero_()
                    bb.step(20)
                big[name]["kernels_us"] = bb.stage_times()
                bb.stage_timing(False)
                big[name]["hbm"] = staged_hbm(big[name]["kernels_us"], pk, 16384 * 512)
            bb.modes()      # raises if a kernel reported an error
            bb.close()
        del flush

    # the other workloads of the benchmark: served jobs (p50/p99 latency), the
    # uneven batch, and the single 64-bp chain in FP64 (one GPU, rank 0 only)
    serving = uneven = config1 = None
    if rank == 0 and world == 1 and not args.no_extra and precision != sfp.SFP_FP32_SIMT:
        b.close()
        config1 = config1_leg(sfp, torch)
        uneven = uneven_leg(sfp, torch, precision, 5000)
        serving = serving_leg(sfp, precision, args.serve_seconds, args.serve_rate, args.serve_budget_mb)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n_c, n_s = 512, 768
        rate, secs, cores = cpu_oracle_rate(n_c, n_s)
        rate1, secs1, _ = cpu_oracle_rate(16, 96, nthreads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
               "sample": f"{n_c} chains x 256 beads x {n_s} steps ({secs:.1f} s)",
               "one_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                              "sample": f"16 chains x 256 beads x 96 steps ({secs1:.1f} s)"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "chains_per_gpu": C_CHAINS, "beads": M_BEADS, "dt_ps": DT_PS,
                       "dtau": dtau, "precision": PREC_NAME[precision],
                       "path": "fused" if (path == sfp.SFP_PATH_FUSED and tensor) else "staged",
                       "steps_per_call": spc,
                       "l2": f"flushed (256 MB write) before every timed sfp_step call of {spc} steps; "
                             "inside a call the state stays in L2, as in a run"},
            "sim_ns_per_s_per_chain": DT_PS * 1e-3 * args.steps / (tot_ms * 1e-3),
            "roofline": roof, "kernels_us": kern, "cpu_baseline": cpu, "e2e": e2e,
            "sustained": sustained, "plain_path": plain, "staged_path": staged,
            "other_split_fused": other, "mode_keyed_noise": modes, "single_step_calls": single,
            "mixed_precision_512bp": big,
            "serving": serving, "uneven": uneven, "config1_fp64": config1,
            "tf32_peak": {"value": pk.get("tf32_tflops"), "unit": "TFLOP/s",
                          "how": "torch.matmul FP32 with TF32 tensor cores, 8192^3, best of 10 (measured live)"},
            "clocks": clocks,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


KERNEL_SOURCES = ("paper_1411_3487_gb300/csrc/sfp_fused.cu", "paper_1411_3487_gb300/csrc/sfp_device.cuh",
                  "paper_1411_3487_gb300/csrc/sfp_ptx.cuh")


def kernel_sha() -> str:
    """First 16 hex digits of the SHA-256 of the fused kernel's sources, in order."""
    import hashlib
    h = hashlib.sha256()
    for src in KERNEL_SOURCES:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(profile: str, source: str = ""):
    """DRAM bytes per launch from a committed ncu summary under profiles/, or None
    when the kernel sources have changed since the counters were taken."""
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        sha = kernel_sha()
    except OSError:
        return None
    got = dict(line.split(":", 1) for line in text.splitlines()
               if line.startswith(("dram_bytes_per_launch:", "kernel_source_sha256_16:")))
    if got.get("kernel_source_sha256_16", "").strip() != sha:
        return None
    try:
        return int(got["dram_bytes_per_launch"].strip())
    except (KeyError, ValueError):
        return None


def roofline(kern, pk, how, precision, path, sfp):
    """Roofline of the dominant kernel from its live CUDA-event time.

    Algorithmic work of the transforms: 18 M flops per bead-step (inverse
    2 M x 3 rows, forward 2 M x 6 rows per chain); the tensor-core kernels
    execute each product as three MMAs (hi/lo split), so the tensor pipe does
    54 M flops per bead-step, compared with the dense peak of the MMA type
    (measured BF16; TF32 from it by the nominal 1.1/2.25 ratio)."""
    if not kern:
        return None
    M, beads = M_BEADS, C_CHAINS * M_BEADS
    if pk.get("tf32_tflops"):
        tf32_peak = pk["tf32_tflops"]
        src = "measured live: torch.matmul TF32 8192^3, best of 10"
    else:
        tf32_peak = pk.get("bf16_tflops", 1900.0) * (1.1 / 2.25)
        src = f"{how} bf16 x 1.1/2.25 (nominal tf32/bf16 dense ratio)"
    if precision == sfp.SFP_MIXED_BF16_2 and path == sfp.SFP_PATH_FUSED:
        us = kern.get("inverse_us")          # the fused kernel is recorded as the first stage
        flops = 2 * 18.0 * M * beads
        peak = pk.get("bf16_tflops", 1900.0)
        return {"bound": "tensor", "kernel": "k_fused_step<256, bf16, two passes> (whole step, bf16x2)",
                "achieved": flops / (us * 1e-6) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops / (us * 1e-6) / 1e12 / peak, "traffic": None,
                "algorithmic_bytes": 24 * beads, "kernel_us": us, "peak_source": f"{how} bf16 dense (burst)"}
    if precision == sfp.SFP_MIXED_BF16 and path == sfp.SFP_PATH_FUSED:
        us = kern.get("inverse_us")          # the fused kernel is recorded as the first stage
        flops = 3 * 18.0 * M * beads
        peak = pk.get("bf16_tflops", 1900.0)
        traffic = measured_traffic("fused_step_bf16_4096x256.md", "paper_1411_3487_gb300/csrc/sfp_fused.cu")
        return {"bound": "tensor", "kernel": "k_fused_step<256, bf16> (whole step, bf16x3)",
                "achieved": flops / (us * 1e-6) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops / (us * 1e-6) / 1e12 / peak, "traffic": traffic,
                "traffic_unit": "DRAM bytes per launch (ncu, profiles/fused_step_bf16_4096x256.md)",
                "algorithmic_bytes": 24 * beads, "kernel_us": us, "peak_source": f"{how} bf16 dense (burst)"}
    if precision == sfp.SFP_FP32 and path == sfp.SFP_PATH_FUSED:
        us = kern.get("inverse_us")          # the fused kernel is recorded as the first stage
        flops = 3 * 18.0 * M * beads
        traffic = measured_traffic("fused_step_4096x256.md", "paper_1411_3487_gb300/csrc/sfp_fused.cu")
        return {"bound": "tensor", "kernel": "k_fused_step<256, tf32> (whole step, tf32x3)",
                "achieved": flops / (us * 1e-6) / 1e12, "peak": tf32_peak, "unit": "TFLOP/s",
                "frac": flops / (us * 1e-6) / 1e12 / tf32_peak, "traffic": traffic,
                "traffic_unit": "DRAM bytes per launch (ncu, profiles/fused_step_4096x256.md)",
                "algorithmic_bytes": 24 * beads, "kernel_us": us, "peak_source": src}
    if precision in (sfp.SFP_FP32, sfp.SFP_MIXED_BF16, sfp.SFP_MIXED_BF16_2):
        # forward transform: DeltaH = chi^T v and Z = phi^T z, 2*rows x M x M, three passes
        bf = precision in (sfp.SFP_MIXED_BF16, sfp.SFP_MIXED_BF16_2)
        peak = pk.get("bf16_tflops", 1900.0) if bf else tf32_peak
        us = kern.get("forward_us")
        flops = 3 * 2.0 * (6 * C_CHAINS) * M * M
        return {"bound": "tensor", "kernel": "k_tc_gemm forward transform (%s)" % ("bf16x3" if bf else "tf32x3"),
                "achieved": flops / (us * 1e-6) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops / (us * 1e-6) / 1e12 / peak, "traffic": None, "kernel_us": us,
                "peak_source": f"{how} bf16 dense (burst)" if bf else src}
    us = kern.get("forward_us")
    flops = 2.0 * (6 * C_CHAINS) * M * M
    peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    return {"bound": "alu", "kernel": "FP32 CUDA-core forward transform",
            "achieved": flops / (us * 1e-6) / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": flops / (us * 1e-6) / 1e12 / peak, "traffic": None, "kernel_us": us,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}


def staged_hbm(kern, pk, beads=None):
    """HBM roofline of the staged step's streaming kernels from their live times:
    bond force 12 B read + 12 B written per bead, bead noise 12 B written (bound
    by its Philox arithmetic, listed for completeness), mode update 36 B read +
    12 B written."""
    beads = beads or C_CHAINS * M_BEADS
    peak = pk.get("hbm_gbs", 6800.0)
    out = {"peak_gbs": peak}
    for name, key, per_bead in (("k_force", "force_us", 24), ("k_noise", "noise_us", 12),
                                ("k_mode_update", "update_us", 48)):
        us = kern.get(key)
        if us:
            gbs = per_bead * beads / (us * 1e-6) / 1e9
            out[name] = {"us": us, "algorithmic_bytes": per_bead * beads, "achieved_gbs": gbs, "frac": gbs / peak}
    return out


def end_to_end(sfp, b, torch, steps, f32=True):
    """Per step: H2D of the mode state from pinned host memory, one sfp_step,
    D2H of the mode state; wall-clock timed.  f32: the state as FP32
    (sfp_set_modes_f32 + SFP_OBS_MODES_F32, the precision the FP32 and mixed
    paths hold it in), else FP64 (sfp_set_modes + SFP_OBS_MODES)."""
    n = 3 * C_CHAINS * M_BEADS
    dt_t, dt_n, width = (torch.float32, np.float32, 4) if f32 else (torch.float64, np.float64, 8)
    hin = torch.empty(n, dtype=dt_t, pin_memory=True)
    hout = torch.empty(n, dtype=dt_t, pin_memory=True)
    a_in, a_out = hin.numpy(), hout.numpy()
    a_in[:] = b.modes().ravel().astype(dt_n)
    L = sfp._lib.load()
    set_modes = L.sfp_set_modes_f32 if f32 else L.sfp_set_modes
    what = sfp.SFP_OBS_MODES_F32 if f32 else sfp.SFP_OBS_MODES

    def one():
        sfp._lib.check(set_modes(b._h, a_in.ctypes.data, n))
        sfp._lib.check(L.sfp_step(b._h, 1))
        sfp._lib.check(L.sfp_observe(b._h, what, a_out.ctypes.data, n * width))

    for _ in range(3):
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    api = "sfp_set_modes_f32 + sfp_step + sfp_observe(SFP_OBS_MODES_F32)" if f32 else \
        "sfp_set_modes + sfp_step + sfp_observe(SFP_OBS_MODES)"
    return {"value": C_CHAINS * M_BEADS * steps / dt, "unit": UNIT, "h2d_bytes_per_step": n * width,
            "d2h_bytes_per_step": n * width, "steps": steps, "api": api}


def bench_precision(sfp, args):
    """The --precision choice as (sfp precision, name)."""
    prec = {"bf16": sfp.SFP_MIXED_BF16, "bf16x2": sfp.SFP_MIXED_BF16_2, "tf32": sfp.SFP_FP32, "tc": sfp.SFP_FP32,
            "simt": sfp.SFP_FP32_SIMT}[args.precision]
    return prec, PREC_NAME.get(prec, str(prec))


def tf32_peak(torch) -> float:
    """Dense TF32 tensor-core throughput of this GPU (TFLOP/s): torch.matmul on
    FP32 8192^3 with TF32 allowed, best of 10 (CUDA events), the way the BF16 peak
    is measured."""
    n = 8192
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        for _ in range(3):
            torch.matmul(a, b)
        best = 1e30
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def config1_leg(sfp, torch):
    """One 64-bp chain, FP64 on the GPU, dt = 1.59 ps (dtau 10), 2e4 steps from an
    equilibrium start (one kernel per chain running the steps of a call); beside it the
    default bead-position Euler scheme of the same chain at dtau = 0.1 (Sec. 3A)."""
    out = {"workload": "1 chain x 64 bp, FP64, dt 1.59 ps (dtau 10), 2e4 steps, equilibrium start"}
    for name, dtau, integ, n in (("mode_space", 10.0, sfp.SFP_INTEGRATOR_MODES, 20000),
                                 ("euler_dtau_0.1", 0.1, sfp.SFP_INTEGRATOR_EULER, 20000)):
        b = sfp.Batch([{"n_beads": 64, "dtau": dtau}], seed=1, precision=sfp.SFP_FP64)
        b.init_equilibrium(0)
        b.set_integrator(integ)
        b.set_graph(True)
        b.step(128)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(n)
        b.modes()                          # synchronises; raises on a kernel error
        dt = time.perf_counter() - t0
        ps = dtau * C_PS
        out[name] = {"value": 64 * n / dt, "unit": UNIT, "steps": n, "dtau": dtau, "dt_ps": ps,
                     "sim_ns_per_s": n * ps * 1e-3 / dt, "wall_s": dt}
        b.close()
    out["value"], out["unit"] = out["mode_space"]["value"], UNIT
    out["sim_ns_per_s_per_chain"] = out["mode_space"]["sim_ns_per_s"]
    return out


def uneven_chains(n=8192, seed=1):
    dt = {64: 10.0, 128: 50.0, 256: 100.0, 512: 100.0}
    rng = np.random.default_rng(seed)
    lengths = rng.choice([64, 128, 256, 512], size=n)
    return [{"n_beads": int(M), "dtau": dt[int(M)], "job_id": i} for i, M in enumerate(lengths)]


def uneven_leg(sfp, torch, prec, steps=5000):
    """8192 chains, lengths uniform over 64/128/256/512 bp at their Table 1 steps,
    FP32 state, equilibrium starts: `steps` steps as calls of 1000 (state in L2
    between the steps of a call), on the tensor-core path (all four lengths in
    one grouped launch of clusters of two CTAs) as created, after the chains-per-tile
    autotuner, and autotuned with CUDA-graph replay; the same with one launch
    per group on its own stream; and the plain FP32 CUDA-core path."""
    chains = uneven_chains()
    beads = sum(c["n_beads"] for c in chains)
    stream = torch.cuda.current_stream()
    res = {}
    for name, p, tune, graph, grouped in (("as_created", prec, False, False, True),
                                          ("autotuned", prec, True, False, True),
                                          ("autotuned_graph", prec, True, True, True),
                                          ("per_group_launches_autotuned_graph", prec, True, True, False),
                                          ("plain_fp32", sfp.SFP_FP32_SIMT, False, True, True)):
        b = sfp.Batch(chains, seed=1, stream=stream, precision=p)
        b.set_grouped(grouped)
        b.init_equilibrium(0)
        tiles = b.autotune(20) if tune else None
        b.set_graph(graph)
        b.step(100)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done = 0
        while done < steps:
            k = min(1000, steps - done)
            b.step(k)
            done += k
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[name] = {"value": beads * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                     "chains_per_tile": tiles, "graph": graph,
                     "launch": "one grouped launch (clusters of two CTAs) for all four lengths"
                     if grouped and p != sfp.SFP_FP32_SIMT else "per group"}
        b.modes()
        b.close()
    best = res["autotuned_graph"]
    return {"workload": "8192 chains, lengths uniform over 64/128/256/512 bp, dtau 10/50/100/100, FP32 state, "
                        f"{steps} steps in calls of 1000", "precision": PREC_NAME.get(prec, str(prec)),
            "beads": beads, "steps": steps, "value": best["value"], "unit": UNIT,
            "vs_plain_fp32": best["value"] / res["plain_fp32"]["value"], "results": res}


def serving_leg(sfp, prec, seconds, rate, budget_mb, seed=1):
    """Continuous-batching serving: Poisson arrivals (`rate` jobs/s for `seconds`)
    of jobs with lengths uniform over 64/128/256/512 bp at their Table 2 steps,
    10^U(3,5) steps, shear 0 with probability 1/2 else U[1e6, 1e8] 1/s; latency
    from submission to the result being on the host; all jobs drained."""
    dt_ps = {64: 1.59, 128: 7.96, 256: 15.9, 512: 15.9}
    rng = np.random.default_rng(seed)
    budget = int(budget_mb * (1 << 20))
    srv = sfp.Server(slots_per_pool=1024, quantum_steps=64, keep_results=False, hbm_budget_bytes=budget,
                     precision=prec)
    clk = ClockSampler(0)
    t0 = time.perf_counter()
    t_next, k, offered = 0.0, 0, 0.0
    while t_next < seconds:
        wait = t0 + t_next - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        M = int(rng.choice([64, 128, 256, 512]))
        n = int(round(10 ** rng.uniform(3, 5)))
        shear = 0.0 if rng.random() < 0.5 else float(rng.uniform(1e6, 1e8))
        srv.submit({"n_beads": M, "dt_ps": dt_ps[M], "n_steps": n, "shear_rate_per_s": shear, "job_id": k})
        offered += M * n
        k += 1
        t_next += rng.exponential(1.0 / rate)
    arrivals_s = time.perf_counter() - t0
    srv.wait_idle(3600)
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    res = srv.poll(k + 16)
    st = srv.stats()
    srv.close()
    lat = np.array([r["latency_s"] for r in res])
    bad = sum(1 for r in res if r["status"] != 0)
    by_len = {}
    for r in res:
        by_len.setdefault(int(r["n_beads"]), []).append(r["latency_s"])
    return {
        "metric": "p50/p99 request latency", "unit": "s", "higher_is_better": False,
        "value": float(np.percentile(lat, 50)), "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)), "max_s": float(lat.max()), "jobs": k, "finished": len(res),
        "failed": bad,
        "p50_s_by_beads": {str(m): float(np.percentile(v, 50)) for m, v in sorted(by_len.items())},
        "workload": "Poisson arrivals, 64/128/256/512 bp at Table 2 steps, 10^U(3,5) steps, half sheared "
                    "U[1e6,1e8]/s, continuous batching",
        "rate_jobs_per_s": rate, "arrival_window_s": seconds, "arrivals_wall_s": arrivals_s,
        "hbm_budget_bytes": budget, "slots_per_pool": 1024, "quantum_steps": 64,
        "precision": PREC_NAME.get(prec, str(prec)),
        "served_bead_steps_per_s": st["bead_steps"] / wall, "offered_bead_steps_per_s": offered / arrivals_s,
        "wall_s": wall, "device_bytes_at_end": st["device_bytes"], "clocks": clocks,
    }


def _names(sfp):
    PREC_NAME.update({sfp.SFP_MIXED_BF16: "SFP_MIXED_BF16", sfp.SFP_FP32: "SFP_FP32",
                      sfp.SFP_FP32_SIMT: "SFP_FP32_SIMT", sfp.SFP_FP64: "SFP_FP64",
                      sfp.SFP_MIXED_BF16_2: "SFP_MIXED_BF16_2"})


def run_serving(args, rank):
    """--workload serving: the serving sub-key on its own."""
    if rank != 0:
        return
    import torch
    sys.path.insert(0, ROOT)
    import paper_1411_3487_gb300 as sfp
    from paper_1411_3487_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    _names(sfp)
    prec, _ = bench_precision(sfp, args)
    line = serving_leg(sfp, prec, args.serve_seconds, args.serve_rate, args.serve_budget_mb)
    line.update({"n_gpus": 1, "data": "synthetic"})
    print(json.dumps(line), flush=True)


def run_precision(args, rank):
    """Error per observable against the FP64 oracle at 16384 x 512 bp (dt 15.9 ps),
    for each GPU precision, with the step time of each (16384 x 512 bp)."""
    if rank != 0:
        return
    import torch
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import paper_1411_3487_gb300 as sfp
    from paper_1411_3487_gb300 import build
    from oracle import oracle as O
    from precision_case import errors
    build.build()
    torch.cuda.set_device(0)
    out = {}
    for name, prec in (("tf32x3_tcgen05", sfp.SFP_FP32), ("bf16x3_tcgen05", sfp.SFP_MIXED_BF16),
                       ("bf16x2_tcgen05", sfp.SFP_MIXED_BF16_2),
                       ("fp32_cuda_cores", sfp.SFP_FP32_SIMT), ("fp64", sfp.SFP_FP64)):
        e = errors(sfp, O, prec, steps=2000, every=20, sub=32)
        b = sfp.Batch([{"n_beads": 512, "dtau": 100.0}] * 16384, seed=1, precision=prec)
        b.init_equilibrium(0)
        b.step(3)
        b.stage_timing(True)
        b.step(20)
        e["step_us"] = b.stage_times()["step_us"]
        b.close()
        out[name] = e
    print(json.dumps({"metric": "error per observable vs FP64 oracle", "workload":
                      "16384 chains x 512 bp, dt 15.9 ps, equilibrium starts; oracle on 32 chains, 2000 steps, "
                      "sums sampled every 20 steps", "errors": out}), flush=True)


def run_uneven(args, rank):
    """--workload uneven: the uneven-batch sub-key on its own (--steps steps)."""
    if rank != 0:
        return
    import torch
    sys.path.insert(0, ROOT)
    import paper_1411_3487_gb300 as sfp
    from paper_1411_3487_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    _names(sfp)
    prec, _ = bench_precision(sfp, args)
    line = uneven_leg(sfp, torch, prec, max(1000, args.steps))
    line.update({"metric": METRIC, "n_gpus": 1, "data": "synthetic"})
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "serving":
        run_serving(args, rank)
        return
    if args.workload == "precision":
        run_precision(args, rank)
        return
    if args.workload == "uneven":
        run_uneven(args, rank)
        return
    run_native(args, rank, world, local)


if __name__ == "__main__":
    main()
