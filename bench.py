"""Benchmark of the FSA apply path (libfsaconv) on GB300.

One step = one solve Phi = T * rho of the headline workload: the 3-D Coulomb
FSA convolution of an 8-Gaussian density on [-16,16]^3 with 256^3 points
(all five passes of the apply path; the spectrum is cached on the device,
as in the paper's Execution phase).  Inputs are resident in HBM when the
timed region starts; each step reads one of 4 rotating rho buffers and
writes one of 4 phi buffers, and one step moves ~0.6 GB (FP32) through
memory, far above the 129 MB L2, so no step finds its inputs in L2.

Prints one JSON line (see --help).  Under torchrun every rank runs its own
replica on its own GPU (solves are independent: replicas only, weak
scaling), the ranks are barrier-synchronised around the timed region, the
time is the max over ranks and the value is all ranks' solves / that time.

--impl reference times the CPU oracle (oracle/, FP64 FFT route) on the host
cores instead: each step is one oracle solve of the same 256^3 density with
the spectrum cached, its FFTs on every host thread (scipy).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/s and HBM-roofline % at 256^3 FP64/FP32; p50/p99 latency under serving"
UNIT = "solves/s"
PASSES = ["r2c_ax0", "row_fwd", "col_mid", "row_inv", "c2r_ax0"]
KERNEL_TEXT = {"coulomb3d": "3-D Coulomb", "biharmonic3d": "3-D biharmonic", "poisson2d": "2-D Poisson",
               "coulomb2d": "2-D Coulomb", "biharmonic2d": "2-D biharmonic", "ddi3d": "3-D DDI (Example 4)",
               "yukawa3d": "3-D Yukawa (Example 4, lam = 1)", "yukawa2d": "2-D Yukawa (Example 4, lam = 1)"}
PLANE_KERNELS = ("poisson2d", "coulomb2d", "biharmonic2d", "yukawa2d")


def plane_pass_bytes(n, s):
    """Algorithmic HBM bytes of the three passes of a plane solve (s = bytes
    per real): R2C reads rho and writes X = (n0+1) n1 complex; the middle pass
    reads and writes X and reads the (n0+1)(n1+1) octant; C2R reads X and
    writes phi."""
    n0, n1 = n
    V = n0 * n1
    X = (n0 + 1) * n1 * 2
    S = (n0 + 1) * (n1 + 1)
    return {"r2c_ax0": (V + X) * s, "row_fwd": 0, "col_mid": (2 * X + S) * s, "row_inv": 0, "c2r_ax0": (X + V) * s}


def pass_bytes(n, s):
    """Algorithmic HBM bytes of each pass for one solve (reads + writes of the
    pass's compulsory input and output; s = bytes per real).  V = n0 n1 n2,
    X = (n0+1) n1 n2 complex, Y = (n0+1) n1 (2 n2) complex, S = octant."""
    n0, n1, n2 = n
    V = n0 * n1 * n2
    X = (n0 + 1) * n1 * n2 * 2
    Y = (n0 + 1) * n1 * 2 * n2 * 2
    S = (n0 + 1) * (n1 + 1) * (n2 + 1)
    return {"r2c_ax0": (V + X) * s, "row_fwd": (X + Y) * s, "col_mid": (2 * Y + S) * s,
            "row_inv": (Y + X) * s, "c2r_ax0": (X + V) * s}


def ddi_grid_pass_bytes(n, s):
    """The DDI grid reading's passes, summed per kind as the profiler does:
    the Coulomb passes, the five unpadded passes of d_n d_m rho (Xn =
    (n0/2+1) n1 n2 complex: R2C reads rho and writes Xn, the row and middle
    passes read and write Xn, C2R reads Xn and writes V reals) and the final
    C2R's read of rho for the local term."""
    n0, n1, n2 = n
    V = n0 * n1 * n2
    Xn = (n0 // 2 + 1) * n1 * n2 * 2
    b = pass_bytes(n, s)
    extra = {"r2c_ax0": (V + Xn) * s, "row_fwd": 2 * Xn * s, "col_mid": 2 * Xn * s, "row_inv": 2 * Xn * s,
             "c2r_ax0": (Xn + V) * s + V * s}
    return {k: b[k] + extra[k] for k in b}


PIPE_LENGTHS = (128, 192, 256, 384, 512)  # transform lengths with the pipelined middle passes


def fused_text(c, M):
    """The outer pass pair in use: separate passes or a cluster configuration."""
    from paper_2504_19410_gb300 import capi
    if not c:
        return "separate passes"
    cs, nt = capi.fsa_fused_configs(M)[c - 1]
    return f"fused, clusters of {cs} CTAs x {nt} threads"


def reference_model_bytes(n, s):
    """Reference 5-pass byte model: E = 2V + 24 n0 n1 (n2+1) + octant reals per solve."""
    n0, n1, n2 = n
    return (2 * n0 * n1 * n2 + 24 * n0 * n1 * (n2 + 1) + (n0 + 1) * (n1 + 1) * (n2 + 1)) * s


# Radix plan of the double-word (first-generation Stockham) line transforms,
# per line length M = 2n; the same factorisation the kernels are built with.
DW_RADICES = {8: [8], 12: [4, 3], 16: [4, 4], 24: [8, 3], 32: [8, 4], 48: [4, 4, 3], 64: [8, 8],
              96: [8, 4, 3], 128: [8, 4, 4], 192: [8, 8, 3], 256: [8, 8, 4], 384: [8, 4, 4, 3],
              512: [8, 8, 8], 768: [8, 8, 4, 3], 1024: [8, 8, 4, 4]}


def dw_mid_ops(n):
    """FP32 operations of the double-word middle pass for one solve (the pass
    is bound by the FP32 pipes, not by HBM).  Costs in FP32 operations: a
    double-word add 8 (TwoSum 6 + 2), multiply 6, complex add 16, complex
    twiddle product 32 (two fused dot products), complex scale 12.  Codelets:
    DFT2/3/4/8 = 32/120/128/440; pruned first stage (zero upper half) of radix
    2/4/8 = 0/64/312; pruned last stage (lower half kept) = 16/96/376.  A
    column line (length M = 2 n1) is: forward transform (first stage pruned),
    multiply by the spectrum (M complex scales), inverse transform (last stage
    pruned), renormalisation of the n1 stored values (12 each); a stage s > 0
    adds R - 1 twiddle products per radix-R group.  At 256^3 this gives 223,232
    per line x 257 x 512 lines, equal to the FADD + FMUL + FFMA thread
    instructions ncu counts for the kernel."""
    n0, n1, n2 = n
    M = 2 * n1
    rad = DW_RADICES[M]
    full = {2: 32, 3: 120, 4: 128, 8: 440}
    half_in = {2: 0, 4: 64, 8: 312}
    half_out = {2: 16, 4: 96, 8: 376}

    def transform(zin, zout):
        ops = 0
        for s, R in enumerate(rad):
            groups = M // R
            last = s == len(rad) - 1
            if zin and s == 0 and R % 2 == 0:
                c = half_in[R]
            elif zout and last and R % 2 == 0:
                c = half_out[R]
            else:
                c = full[R]
            tw = (R - 1) * 32 if s > 0 else 0
            ops += groups * (c + tw)
        return ops

    per_line = transform(True, False) + 12 * M + transform(False, True) + 12 * n1
    return per_line * (n0 + 1) * (2 * n2)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def read_traffic(kernel, workload, dtype):
    """DRAM bytes per launch from the committed ncu summary, if it lists this
    kernel for this workload and dtype (lines: kernel workload dtype bytes)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        for line in f:
            t = line.split("#", 1)[0].split()
            if len(t) >= 4 and t[0] == kernel and t[1] == workload and t[2] == dtype:
                return float(t[3])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                t = [x.strip() for x in line.split(",")]
                if len(t) >= 9:
                    rows.append(t)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def allreduce_max(x, dist, device):
    """Max of a float over all ranks (replicas report the slowest rank's time).
    `device` is where the collective's tensor lives: cuda for NCCL, cpu for gloo."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ ours ----

def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_19410_gb300 as fsa
    from paper_2504_19410_gb300 import capi
    import workloads as W

    capi.fsa_autotune_set({"auto": 1, "1": 2, "2": 3, "3": 4, "4": 5, "6": 6, "8": 7}[args.kernel_gen])
    plane = args.kernel in PLANE_KERNELS
    ddi_kw = ({"dipoles": (W.DDI_N, W.DDI_M), "ddi_derivative": args.ddi_derivative}
              if args.kernel == "ddi3d" else {})
    # 8 Gaussians, [-16,16]^3 at 256^3 (or [-16,16]^2 at 512^2 for a plane kernel), eps = 1
    d = W.gaussian_sum_2d(seed=2504) if plane else W.gaussian_sum(seed=2504, n=args.n)
    n = d.n
    if args.outer_pairs != "auto" and capi.fsa_fused_configs(2 * n[0]):
        capi.fsa_fused_select(2 * n[0], 2, 0 if args.outer_pairs == "separate" else int(args.outer_pairs))
    if args.pipe != "auto" and not plane and n[1] == n[2] and 2 * n[2] in PIPE_LENGTHS:
        capi.fsa_pipe_select(2 * n[2], int(args.pipe))
    rho64 = d.rho()
    hbm_peak, peak_kind = peaks()
    stream = torch.cuda.current_stream()
    out = {}
    # measured ALU peaks of this GPU: the denominators of the ALU rooflines
    f32_rate, f32_ms = capi.fsa_measure_alu_peak(0)
    f64_rate, f64_ms = capi.fsa_measure_alu_peak(1)
    x2_rate, _ = capi.fsa_measure_alu_peak(2)
    alu_peaks = {"fp32_fma_gops": f32_rate / 1e9, "fp64_fma_gops": f64_rate / 1e9,
                 "fp32x2_fma_gops": x2_rate / 1e9,
                 "fp32_tflops": 2 * f32_rate / 1e12, "fp64_tflops": 2 * f64_rate / 1e12,
                 "how": "fsa_measure_alu_peak: every resident thread runs 8 independent FMA chains, "
                        f"best of 3 launches by CUDA events ({f32_ms:.2f} / {f64_ms:.2f} ms); 1 FMA = 1 op = 2 flop"}

    def bench_tier(dt):
        tdt = torch.float32 if dt == "f32" else torch.float64
        s = 4 if dt == "f32" else 8
        t0 = time.perf_counter()
        plan = fsa.Plan(d.L, n, dt, eps=d.eps, generate=False, l2_chunk_mb=args.l2_chunk_mb,
                        kernel=args.kernel, **ddi_kw)  # + autotuner trials
        torch.cuda.synchronize()
        create_ms = (time.perf_counter() - t0) * 1e3
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        plan.generate(stream)  # the paper's Precomp: the kernel tensor's spectrum, FP64 on the device
        g1.record(stream)
        torch.cuda.synchronize()
        precomp_ms = g0.elapsed_time(g1)
        rhos = [torch.from_numpy(rho64).to(tdt).cuda() for _ in range(4)]
        phis = [torch.empty_like(rhos[0]) for _ in range(4)]
        for i in range(args.warmup):
            plan.apply(rhos[i % 4], phis[i % 4])
        prof = capi.fsa_profiler_create(args.steps)
        clk = ClockSampler(local)
        clk.start()
        # untimed applies of the same solve for about 0.6 s, so that the
        # clock samples (every 200 ms) fall under this load and the timed
        # steps start on a busy GPU
        t_soak = time.perf_counter()
        i = 0
        while time.perf_counter() - t_soak < 0.6:
            for _ in range(16):
                plan.apply(rhos[i % 4], phis[i % 4])
                i += 1
            torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        # the timed steps: plain applies, nothing recorded between the passes
        ev0.record(stream)
        for i in range(args.steps):
            plan.apply(rhos[i % 4], phis[i % 4])
        ev1.record(stream)
        torch.cuda.synchronize()
        elapsed = ev0.elapsed_time(ev1)
        # the same steps again with an event after every pass: the per-pass
        # durations of the rooflines (the events cost a little: see step_ms)
        for i in range(args.steps):
            capi.fsa_apply_profiled(plan.handle, rhos[i % 4], phis[i % 4], stream, prof)
        torch.cuda.synchronize()
        clocks = clk.stop()
        barrier()
        elapsed = allreduce_max(elapsed, dist, "cuda")
        pass_ms, step_ms, steps = capi.fsa_profiler_read(prof)
        capi.fsa_profiler_destroy(prof)
        pb = (plane_pass_bytes(n, s) if plane else
              ddi_grid_pass_bytes(n, s) if args.kernel == "ddi3d" and args.ddi_derivative == "grid" else
              pass_bytes(n, s))
        info = plan.info
        if not plane and args.kernel != "ddi3d" and (info.fused_fwd or info.fused_inv):
            # the fused outer pairs (clusters): rho -> Y reported as row_fwd,
            # Y -> phi as row_inv; X never goes to HBM
            pb = dict(pb)
            V = n[0] * n[1] * n[2]
            Yr = (n[0] + 1) * n[1] * 2 * n[2] * 2
            if info.fused_fwd:
                pb["r2c_ax0"], pb["row_fwd"] = 0, (V + Yr) * s
            if info.fused_inv:
                pb["row_inv"], pb["c2r_ax0"] = (Yr + V) * s, 0
        if info.pipe:
            # the pipelined middle passes (one kernel, reported as col_mid):
            # X in, X out and the spectrum; Y stays in L2 between its passes
            pb = dict(pb)
            Xr = (n[0] + 1) * n[1] * n[2] * 2
            pb["row_fwd"], pb["row_inv"] = 0, 0
            pb["col_mid"] = (2 * Xr + (n[0] + 1) * (n[1] + 1) * (n[2] + 1)) * s
        dom = max(range(5), key=lambda i: pass_ms[i])
        kname = PASSES[dom]
        achieved = pb[kname] / (pass_ms[dom] * 1e-3) / 1e9
        # 3-D: the reference 27V byte model; plane: the sum of the three passes' bytes
        model_s = (sum(pb.values()) if plane else reference_model_bytes(n, s)) / (hbm_peak * 1e9)
        arith = ["fp32", "fp64", "double-word"][plan.info.arithmetic]
        hbm_roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm_peak,
                    "unit": "GB/s", "frac": achieved / hbm_peak, "peak_kind": f"of {peak_kind}",
                    "alg_bytes_per_launch": pb[kname],
                    "traffic": (None if plane or args.kernel == "ddi3d" or args.n != 256
                                else read_traffic(kname, "c2_256", dt))}
        roof = hbm_roof
        if arith == "double-word" and kname == "col_mid" and not plane and args.kernel != "ddi3d":
            # The double-word passes run on the FP32 pipes: besides the HBM
            # roofline (the metric's), the pass's FP32 operations per launch
            # over the MEASURED FP32 FMA rate (fsa_measure_alu_peak).
            ops = dw_mid_ops(n)
            alu = ops / (pass_ms[dom] * 1e-3) / 1e9
            alu_peak = alu_peaks["fp32_fma_gops"]
            roof = dict(hbm_roof)
            roof["alu"] = {"bound": "alu", "achieved": alu, "peak": alu_peak,
                           "unit": "Gop/s (FP32 lane operations)", "frac": alu / alu_peak,
                           "peak_kind": "measured FP32 FMA rate (fsa_measure_alu_peak)",
                           "alg_ops_per_launch": ops}
        res = {
            "value": ws * args.steps / (elapsed * 1e-3),
            "ms_per_step": elapsed / args.steps,
            "precomp_ms": precomp_ms,
            "plan_create_ms": create_ms,
            "arithmetic": arith,
            "pass_ms": dict(zip(PASSES, [round(x, 5) for x in pass_ms])),
            "profiled_step_ms": step_ms,
            "roofline": roof,
            "step_roofline_frac_27V_model": model_s * 1e3 / (elapsed / args.steps),
            "clocks": clocks,
            "gpu_launches": plan.info.launches_per_apply * args.steps,
            "launches_per_solve": plan.info.launches_per_apply,
            "outer_pairs": {"forward": fused_text(info.fused_fwd, 2 * n[0]),
                            "inverse": fused_text(info.fused_inv, 2 * n[0])},
            "middle_passes": "pipelined (one kernel)" if info.pipe else "separate passes",
            "pass_hbm_frac": {k: round(pb[k] / (v * 1e-3) / 1e9 / hbm_peak, 4)
                              for k, v in zip(PASSES, pass_ms) if v > 0 and pb[k] > 0},
        }
        # e2e through the C-ABI host-buffer entry point: every step copies its rho
        # from pinned host memory and its phi back (both inside the timed
        # region).  Three plans on three streams rotate -- one solve's input
        # copy, another's kernels and a third's output copy in flight at once,
        # the pipeline a caller streaming solves would run.
        res["e2e"] = None
        if not args.no_e2e:
            NS = 3
            plans = [plan] + [fsa.Plan(d.L, n, dt, eps=d.eps, l2_chunk_mb=args.l2_chunk_mb, kernel=args.kernel,
                                       **ddi_kw) for _ in range(NS - 1)]
            streams = [torch.cuda.Stream() for _ in range(NS)]
            hin = [torch.from_numpy(rho64).to(tdt).pin_memory() for _ in range(NS)]
            hout = [torch.empty_like(hin[0]).pin_memory() for _ in range(NS)]
            for i in range(NS):
                plans[i].apply_host(hin[i], hout[i], streams[i])
            torch.cuda.synchronize()
            barrier()
            k = max(6, args.steps // 2) // NS * NS
            t0 = time.perf_counter()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(k):
                s_i = streams[i % NS]
                s_i.wait_event(e0) if i < NS else None
                plans[i % NS].apply_host(hin[i % NS], hout[i % NS], s_i)
            for s_i in streams:
                stream.wait_stream(s_i)
            e1.record(stream)
            torch.cuda.synchronize()
            et = e0.elapsed_time(e1)
            wall = (time.perf_counter() - t0) * 1e3
            et = allreduce_max(et, dist, "cuda")
            nb = int(np.prod(n)) * s
            res["e2e"] = {"value": ws * k / (et * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nb,
                          "d2h_bytes_per_step": nb, "ms_per_step": et / k, "host_wall_ms_per_step": wall / k,
                          "how": f"fsa_apply_host, pinned host buffers, {NS} plans on {NS} streams rotating"}
            for p in plans[1:]:
                p.close()
        plan.close()
        del rhos, phis
        torch.cuda.empty_cache()
        return res

    tiers = {}
    for dt in args.tiers.split(","):
        tiers[dt] = bench_tier(dt)
    main = tiers.get("f32") or tiers["f64"]

    batched = None if args.no_batched else bench_batched(args, fsa, W, torch, stream)
    many = None if args.no_many else bench_many(args, fsa, W, torch, stream)
    serving = None if args.no_serve else bench_serving(args, fsa, W, torch, rank)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(d, args.kernel)

    if rank == 0:
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if "f32" in tiers else "f64",
            "data": "synthetic",
            "config": {"workload": (f"plane_512: {KERNEL_TEXT[args.kernel]} FSA apply, 8-Gaussian plane density "
                                    "(seed 2504) on [-16,16]^2, 512^2 grid, eps=1, spectrum cached on device")
                                   if args.kernel in PLANE_KERNELS else
                                   (f"{'c2_256' if args.n == 256 else f'gaussian8_{args.n}'}: "
                                    f"{KERNEL_TEXT[args.kernel]} FSA apply, 8-Gaussian density (seed 2504) on "
                                    f"[-16,16]^3, {args.n}^3 grid, eps=1, spectrum cached on device"
                                    + (f"; dipoles n, m of Example 4, {args.ddi_derivative} reading of d_n d_m rho"
                                       if args.kernel == "ddi3d" else "")),
                       "grid": list(n),
                       "l2": ("plane: per-step working set ~12 MB (FP32) < 129 MB L2, L2-resident, not flushed"
                              if args.kernel in PLANE_KERNELS else
                              f"per-step working set ~{reference_model_bytes(n, 4) / 3e9:.3g} GB (FP32) "
                              + ("> 129 MB L2; 4 rotating rho/phi buffers"
                                 if reference_model_bytes(n, 4) / 3 > 129e6 else
                                 "< 129 MB L2: L2-resident, not flushed (a latency-bound small grid)")),
                       "parallelism": f"replicas x{ws}"},
            "roofline": main["roofline"],
            "alu_peaks": alu_peaks,
            "cpu_baseline": cpu,
            "e2e": main["e2e"],
            "gpu_launches": main["gpu_launches"],
            "clocks": main["clocks"],
            "pass_ms": main["pass_ms"],
            "pass_hbm_frac": main["pass_hbm_frac"],
            "outer_pairs": main["outer_pairs"],
            "precomp_ms": main["precomp_ms"],
            "plan_create_ms": main["plan_create_ms"],
            "step_roofline_frac_27V_model": main["step_roofline_frac_27V_model"],
        }
        if batched is not None:
            line["batched"] = batched
        if many is not None:
            line["many"] = many
        if serving is not None:
            line["serving"] = serving
        if "f64" in tiers and main is not tiers["f64"]:
            line["f64"] = {k: tiers["f64"][k] for k in ("value", "ms_per_step", "roofline", "pass_ms", "precomp_ms",
                                                        "plan_create_ms",
                                                        "step_roofline_frac_27V_model", "e2e", "clocks",
                                                        "arithmetic")}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------- batched (C4) ----

def bench_batched(args, fsa, W, torch, stream):
    """64 seeded Gaussian-sum densities, cubic n from {64,96,128,192,256},
    gamma in {1,4,8} (cigar or pancake), FP32, in one batched call (persistent
    launches over all 64 solves' concatenated tile lists, captured in a CUDA
    graph; every scheduling mode of fsa_batched_mode_set timed), against the
    same 64 solves issued one fsa_apply at a time."""
    dens = W.batch_requests(seed=2504, count=64)
    plans = [fsa.Plan(d.L, d.n, "f32", eps=d.eps) for d in dens]
    rhos = [d.rho_torch(torch.float32) for d in dens]
    phis = [torch.empty_like(r) for r in rhos]
    k = max(3, args.steps // 5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    modes = {}
    # fsa_batched_mode_set: 0 auto (the default: times 1 and 2 on the first
    # call, keeps the faster), 1 one mixed launch per pass, 2 per-shape groups
    # on concurrent streams, 3 mixed pipelined in two halves
    for mode in (1, 2, 3, 0):
        fsa.capi.fsa_batched_mode_set(mode)
        for _ in range(2):
            fsa.apply_batched(plans, rhos, phis)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fsa.apply_batched(plans, rhos, phis)
        e1.record(stream)
        torch.cuda.synchronize()
        t_m = e0.elapsed_time(e1) / k
        modes[mode] = {"ms_per_batch": t_m, "solves_per_s": len(dens) / (t_m * 1e-3),
                       "gpu_launches_per_batch": fsa.capi.fsa_apply_batched_launches([p.handle for p in plans])}
    tb = modes[0]["ms_per_batch"]
    for p, r, f in zip(plans, rhos, phis):
        p.apply(r, f)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        for p, r, f in zip(plans, rhos, phis):
            p.apply(r, f)
    e1.record(stream)
    torch.cuda.synchronize()
    ts = e0.elapsed_time(e1) / k
    hist = {}
    for d in dens:
        hist[d.n[0]] = hist.get(d.n[0], 0) + 1
    bytes_model = sum(reference_model_bytes(d.n, 4) for d in dens)
    hbm_peak, kind = peaks()
    out = {"workload": "c4: 64 densities, n in {64,96,128,192,256} (counts " + json.dumps(hist) +
                       "), gamma in {1,4,8}, FP32", "solves_per_batch": len(dens),
           "value": len(dens) / (tb * 1e-3), "unit": UNIT, "ms_per_batch": tb,
           "sequential_solves_per_s": len(dens) / (ts * 1e-3), "ms_sequential": ts,
           "step_roofline_frac_27V_model": bytes_model / (hbm_peak * 1e9) / (tb * 1e-3),
           # the library's own count of the default mode's launches
           "gpu_launches_per_batch": modes[0]["gpu_launches_per_batch"],
           "path": "auto: the faster of the mixed path (one persistent launch per pass over the 64 solves' "
                   "concatenated tile lists) and per-shape groups, timed on the first call",
           "modes": {"0 auto (default)": modes[0], "1 mixed, one launch per pass": modes[1],
                     "2 per-shape groups, concurrent streams": modes[2],
                     "3 mixed, pipelined halves": modes[3]}}
    for p in plans:
        p.close()
    del rhos, phis
    torch.cuda.empty_cache()
    return out


# ------------------------------------------- many densities, one plan ----

def bench_many(args, fsa, W, torch, stream):
    """Many densities through one plan (fsa_apply_many: one launch sequence,
    the middle pass reading each spectrum tile once for all densities) against
    the same solves issued one fsa_apply at a time: 8 densities at 256^3 and
    64 at 64^3, FP32, 8-Gaussian sums (seeds 2504 + k) on [-16,16]^3."""
    out = {}
    for n, K in ((256, 8), (64, 64)):
        dens = [W.gaussian_sum(seed=2504 + k, n=n) for k in range(K)]
        plan = fsa.Plan(dens[0].L, dens[0].n, "f32", eps=dens[0].eps)
        plan.reserve(K)
        rhos = [d.rho_torch(torch.float32) for d in dens]
        phis = [torch.empty_like(r) for r in rhos]
        for _ in range(2):
            plan.apply_many(rhos, phis)
        torch.cuda.synchronize()
        reps = max(3, args.steps // 5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.apply_many(rhos, phis)
        e1.record(stream)
        torch.cuda.synchronize()
        tm = e0.elapsed_time(e1) / reps
        e0.record(stream)
        for _ in range(reps):
            for r, f in zip(rhos, phis):
                plan.apply(r, f)
        e1.record(stream)
        torch.cuda.synchronize()
        ts = e0.elapsed_time(e1) / reps
        out[f"{n}^3 x{K}"] = {"value": K / (tm * 1e-3), "unit": UNIT, "ms_per_call": tm,
                             "sequential_solves_per_s": K / (ts * 1e-3), "ms_sequential": ts,
                             "gpu_launches_per_call": plan.info.launches_per_apply,
                             "outer_pairs": {"forward": fused_text(plan.info.fused_fwd, 2 * n),
                                             "inverse": fused_text(plan.info.fused_inv, 2 * n)}}
        plan.close()
        del rhos, phis
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------- serving (C5) ----

def bench_serving(args, fsa, W, torch, rank):
    """Poisson-arrival request stream through the serving loop (C5): n
    log-uniform in [32,512] rounded to supported sizes, 80 % FP32 / 20 % FP64,
    isotropic [-16,16]^3 8-Gaussian densities; plans cached on the device,
    admission by free HBM.  Capacity is measured closed loop (all requests
    queued at once); the open-loop run offers Poisson arrivals at
    load x capacity and reports p50/p99 latency (submit -> done)."""
    import numpy as np
    reqs = W.serve_requests(seed=2504, count=args.serve_n)
    keys = sorted({(n, dt) for n, dt, _ in reqs})
    inputs, pools = {}, {}
    for n, dt in keys:
        tdt = torch.float32 if dt == "f32" else torch.float64
        inputs[(n, dt)] = W.gaussian_sum(seed=2504 + n, n=n).rho_torch(tdt)
        pools[(n, dt)] = [torch.empty_like(inputs[(n, dt)]) for _ in range(4 if n >= 384 else 8)]
    srv = fsa.Server(max_inflight=32, streams=8, policy=args.serve_policy)

    def run(arrivals):
        free = {k: list(v) for k, v in pools.items()}
        outstanding = {}
        lat, t0 = [], time.perf_counter()

        def reap(block):
            for t in list(outstanding):
                st, tm = srv.poll(t, 0.05 if block else 0.0)
                if st in (2, 3):
                    key, buf = outstanding.pop(t)
                    free[key].append(buf)
                    lat.append((tm.done_s - tm.submit_s) * 1e3)
                    if block:
                        return

        for i, (n, dt, _) in enumerate(reqs):
            if arrivals is not None:
                while time.perf_counter() - t0 < arrivals[i]:
                    reap(False)
            key = (n, dt)
            while not free[key]:
                reap(True)
            buf = free[key].pop()
            t = srv.submit((16.0, 16.0, 16.0), (n, n, n), dt, inputs[key], buf, eps=1.0)
            outstanding[t] = (key, buf)
            reap(False)
        while outstanding:
            reap(True)
        wall = time.perf_counter() - t0
        return wall, lat

    # warm the plan cache and the workspace pool: one request per (n, tier)
    for key in keys:
        t = srv.submit((16.0, 16.0, 16.0), (key[0],) * 3, key[1], inputs[key], pools[key][0], eps=1.0)
        srv.wait(t, timeout=600.0)
    wall, lat = run(None)
    capacity = len(reqs) / wall
    arrivals = W.poisson_arrivals(2504, len(reqs), args.serve_load * capacity)
    wall2, lat2 = run(arrivals)
    # the other offered loads (same stream, same seed for the arrival process)
    per_load = {f"{args.serve_load:g}": {"solves_per_s": len(reqs) / wall2,
                                         "p50_ms": float(np.percentile(lat2, 50)),
                                         "p99_ms": float(np.percentile(lat2, 99))}}
    for f in [float(x) for x in args.serve_other_loads.split(",") if x]:
        w_f, lat_f = run(W.poisson_arrivals(2504, len(reqs), f * capacity))
        per_load[f"{f:g}"] = {"solves_per_s": len(reqs) / w_f, "p50_ms": float(np.percentile(lat_f, 50)),
                              "p99_ms": float(np.percentile(lat_f, 99))}
    st = srv.stats()
    srv.close()
    # the other scheduling policy on the same arrival stream (same offered rate)
    other_policy = 1 - args.serve_policy
    srv = fsa.Server(max_inflight=32, streams=8, policy=other_policy)
    for key in keys:
        srv.wait(srv.submit((16.0, 16.0, 16.0), (key[0],) * 3, key[1], inputs[key], pools[key][0], eps=1.0),
                 timeout=600.0)
    w_o, lat_o = run(arrivals)
    srv.close()
    other = {"policy": other_policy, "offered_load": args.serve_load, "solves_per_s": len(reqs) / w_o,
             "p50_ms": float(np.percentile(lat_o, 50)), "p99_ms": float(np.percentile(lat_o, 99))}
    torch.cuda.empty_cache()
    lat2 = np.array(lat2)

    # The plain FP64 single-solve path on the same request sizes: one FP64 plan
    # per size, every request solved alone (fsa_apply, one stream, no overlap),
    # back to back; a sample of the stream keeps the run short.
    sample = reqs[: args.serve_fp64_sample]
    plans64, in64, out64 = {}, {}, {}
    for n, _, _ in sample:
        if n not in plans64:
            plans64[n] = fsa.Plan((16.0, 16.0, 16.0), (n, n, n), "f64", eps=1.0)
            in64[n] = inputs[(n, "f64")] if (n, "f64") in inputs else \
                W.gaussian_sum(seed=2504 + n, n=n).rho_torch(torch.float64)
            out64[n] = torch.empty_like(in64[n])
    for n in plans64:
        plans64[n].apply(in64[n], out64[n])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for n, _, _ in sample:
        plans64[n].apply(in64[n], out64[n])
    torch.cuda.synchronize()
    fp64_single = len(sample) / (time.perf_counter() - t0)
    for p in plans64.values():
        p.close()
    del in64, out64
    torch.cuda.empty_cache()
    return {"workload": f"c5: {len(reqs)} requests, n log-uniform in [32,512] (supported sizes), "
                        "80% FP32 / 20% FP64, [-16,16]^3 8-Gaussian densities",
            "capacity_solves_per_s": capacity, "offered_load": args.serve_load,
            "value": len(reqs) / wall2, "unit": UNIT,
            "p50_ms": float(np.percentile(lat2, 50)), "p99_ms": float(np.percentile(lat2, 99)),
            "closed_loop_p50_ms": float(np.percentile(lat, 50)),
            "per_load": dict(sorted(per_load.items())),
            "policy": args.serve_policy,
            "policy_text": {0: "size-aware lanes: large requests on low-priority bulk streams, one CTA per tile; "
                               "others on high-priority streams, least-loaded stream per lane",
                            1: "round robin over equal-priority streams, persistent grids"}[args.serve_policy],
            "other_policy_same_arrivals": other,
            "plan_hit_rate": st.plan_hits / max(1, st.plan_hits + st.plan_misses),
            "fp64_single_solve_solves_per_s": fp64_single,
            "fp64_single_solve_sample": f"first {len(sample)} requests, each solved alone in FP64 "
                                        "(the FP64 tier's arithmetic), sequentially",
            "served_capacity_over_fp64_single": capacity / fp64_single}


# -------------------------------------------------------------- oracle ----

def host_cores():
    """Host threads this process may run on (the cgroup / affinity set)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_timing(d, reps, workers_list, kernel="coulomb3d"):
    """The oracle's Execution phase (FFT route with the spectrum cached, FP64,
    numpy / scipy FFT) on density d at its own grid: the spectrum is computed
    once (untimed, on all host threads), then each entry of workers_list
    (None = numpy's single-threaded FFT, k = scipy's FFT on k threads) is
    timed over ``reps`` solves; returns {workers: seconds per solve}."""
    from oracle import fsa as oracle
    rho = d.rho()
    allw = host_cores()
    S = oracle.spectrum(oracle.tensor_T(d.L, d.n, d.eps, kernel=kernel, workers=allw), workers=allw)
    out = {}
    for w in workers_list:
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            oracle.apply_spectrum(S, rho, workers=w)
            ts.append(time.perf_counter() - t0)
        out[w] = min(ts)
    del S
    return out


def cpu_baseline(d, kernel="coulomb3d"):
    """The oracle timed on this host's cores on the benchmarked density and
    grid itself (no scaling): one solve on 1 thread, one on every thread; for
    3-D grids also C1 (32^3) and the cigar (128 x 128 x 512)."""
    import workloads as W
    cores = host_cores()
    n = d.n
    kern = "coulomb3d" if kernel == "ddi3d" else kernel  # the DDI solve's FFT route is Coulomb's
    t = oracle_timing(d, 1, [cores, None], kern)
    three_d = len(n) == 3
    c1 = oracle_timing(W.iso_gaussian(), 5, [cores, None]) if three_d else None
    cig = oracle_timing(W.aniso_gaussian("cigar"), 1, [cores, None]) if three_d else None

    def rate(x):
        return {"all_cores_solves_per_s": 1.0 / x[cores], "one_core_solves_per_s": 1.0 / x[None]}
    return {"value": 1.0 / t[cores], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one oracle solve (FFT route, FP64, spectrum cached) of the same 8-Gaussian density "
                      f"on the same {'x'.join(map(str, n))} grid, measured (not scaled): {t[cores]:.2f} s on "
                      f"{cores} threads (scipy FFT, workers={cores}), {t[None]:.2f} s on 1 thread (numpy FFT)",
            "one_core": {"value": 1.0 / t[None], "unit": UNIT, "cores": 1},
            "configs": ({"benchmarked_grid": rate(t), "c1_32": rate(c1), "cigar_128x128x512": rate(cig)}
                        if three_d else {"benchmarked_grid": rate(t)})}


def run_reference(args):
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    import workloads as W
    from oracle import fsa as oracle
    cores = host_cores()
    d = W.gaussian_sum(seed=2504, n=256)
    rho = d.rho()
    S = oracle.spectrum(oracle.tensor_T(d.L, d.n, d.eps, workers=cores), workers=cores)
    for _ in range(args.warmup):
        oracle.apply_spectrum(S, rho, workers=cores)
    secs = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.apply_spectrum(S, rho, workers=cores)
        secs.append(time.perf_counter() - t0)
    total = sum(secs)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "c2_256: 3-D Coulomb FSA apply, 8-Gaussian density (seed 2504) on "
                               "[-16,16]^3, 256^3 grid, eps=1, spectrum cached",
                   "grid": [256, 256, 256], "parallelism": f"host cores (oracle, {cores} threads)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step one oracle solve (FFT route, FP64, spectrum cached) of the "
                                   f"8-Gaussian density on the 256^3 grid itself, scipy FFT on {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tiers", default="f32,f64", help="apply tiers to time; the first FP32 one is the headline")
    ap.add_argument("--kernel", choices=list(KERNEL_TEXT), default="coulomb3d",
                    help="kernel of Table 1 for the single-solve tiers (batched and serving legs use Coulomb)")
    ap.add_argument("--ddi-derivative", choices=["grid", "kernel"], default="grid",
                    help="--kernel ddi3d: d_n d_m rho on the computational grid (the paper's Table 5) or "
                         "fused into the middle multiply")
    ap.add_argument("--n", type=int, default=256,
                    help="3-D kernels: grid points per axis of the 8-Gaussian workload (default 256, the "
                         "headline workload; smaller grids are L2-resident and latency-bound)")
    ap.add_argument("--outer-pairs", default="auto",
                    help="the outer pass pairs of FP32 cubes: auto (tuned), separate, or a fused cluster "
                         "configuration 1, 2, ... (fsa_fused_configs)")
    ap.add_argument("--pipe", choices=["auto", "0", "1"], default="auto",
                    help="middle passes of FP32 grids with n1 = n2: auto (tuned), 0 separate, 1 pipelined kernel")
    ap.add_argument("--kernel-gen", choices=["auto", "1", "2", "3", "4", "6", "8"], default="auto",
                    help="auto: autotuned per plan; 1 / 2 / 3 / 4 / 6: force one kernel generation "
                         "(FP64: native for 1, double-word otherwise)")
    ap.add_argument("--l2-chunk-mb", type=int, default=0,
                    help="plane-slab size of the middle passes in MB (0 = library default, -1 = one slab)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-many", action="store_true", help="skip the many-densities-one-plan leg")
    ap.add_argument("--serve-other-loads", default="0.5,0.95",
                    help="further offered loads (fractions of the measured capacity) for the serving leg's p50/p99")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-n", type=int, default=10000, help="requests in the serving run")
    ap.add_argument("--serve-fp64-sample", type=int, default=1000,
                    help="requests of the stream re-run through the plain FP64 single-solve path")
    ap.add_argument("--serve-load", type=float, default=0.8, help="offered load as a fraction of capacity")
    ap.add_argument("--serve-policy", type=int, choices=[0, 1], default=0,
                    help="serving policy (fsa_serve_opts.policy): 0 size-aware lanes, 1 round robin")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
