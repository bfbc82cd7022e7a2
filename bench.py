"""Benchmark of the NENO6 Euler right-hand side on GB300.

One step = one third-order SSP Runge-Kutta step of the whole grid: the CFL
reduction and three fused right-hand-side evaluations (the hot path: ghost
cells, Roe characteristic projection, LLF split, classifier, renormalised
combination, back-projection, conservative difference, stage update).

Default workload (N=1): 2D Euler, 4096 x 4096 periodic grid, seeded
four-quadrant states with a sinusoidal density perturbation, mixed-precision
path (fp16 tensor-core classifier with an FP32 guard band, FP32
reconstruction of block-relative deviations, FP64 Roe eigenvectors, reference
fluxes, difference and RK3).  Beside it the FP64 GPU
path on the same state (speed, mask flip rate, L1/Linf error of dU/dt and of
the state after one step).  `--precision fp64 --n 2048` gives the FP64 line.
Metric: Mcell-updates/s (cells x steps / s), higher is better.

`--impl reference` times the FP64 CPU oracle on the same workload's
structure (a bounded periodic crop per step) on this host's cores.

Under torchrun (N > 1) every rank advances its own independent copy of the
workload (weak scaling, no data-path collective); rank 0 prints one JSON
line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D Euler NENO6 RHS Mcell-updates/s: mixed-prec vs FP64 GPU, at stated L1 error"
UNIT = "Mcell-updates/s"
WEIGHTS = os.path.join(ROOT, "weights", "neno6_mlp_6x64x32x16x8x4.bin")
SMS = 152


# --------------------------------------------------------------- flop count
def flops_per_cell_rhs(ndim=2):
    """Algorithmic binary64 flops of one cell's right-hand side, counted from
    the scheme's definition (fma = 2, every other + - * / sqrt = 1; max, |x|
    and ReLU not counted).  Per face: Roe average and eigenvectors, per field
    the projection of six cells (U and F), LLF split, two normalisations, two
    classifier calls, two candidate sets, two renormalised combinations, the
    sum of both sides; back-projection.  Per cell: primitives and fluxes, the
    conservative difference.  2D: two faces per cell (one x, one y)."""
    nv = 4 if ndim == 2 else 3
    mlp = 2 * (6 * 64 + 64 * 32 + 32 * 16 + 16 * 8 + 8 * 4)    # 3104 fma
    roe = 29 if ndim == 2 else 21
    eig = 15 if ndim == 2 else 12
    alpha = 12                                                # u_n -/+ c for the two acoustic fields
    per_field = (6 * 2 * (1 + 2 * (nv - 1))                   # v = L.U_j, g = L.F_j
                 + 6 * 6                                      # split: 2 fma + 2 mul per cell
                 + 2 * 6                                      # 2 x 6 divisions (normalise)
                 + 2 * mlp
                 + 2 * 22                                     # candidates S0..S3, both sides
                 + 2 * (3 + 4 + 8)                            # sum of d, 4 divisions, 4 fma
                 + 1)                                         # g+ + g-
    per_face = roe + eig + alpha + nv * per_field + nv * (1 + 2 * (nv - 1))
    per_cell = 25 + nv * (5 if ndim == 2 else 2)
    return ndim * per_face + per_cell


def fp64_flops_per_cell_rhs_mixed(ndim=2):
    """Algorithmic binary64 flops of one cell's RHS in the mixed path, i.e.
    the parts kept in FP64: per cell the Roe inputs and fluxes (1/rho, u, v,
    q, p, H, sqrt(rho), one flux per direction), per face the Roe average and
    eigenvectors (29 + 15) and the back-projection (4 x 7), per cell the
    difference and the RK3 stage (nv x 9)."""
    nv = 4 if ndim == 2 else 3
    per_cell = 1 + 2 + 3 + 4 + 2 + 1 + ndim * 4
    per_face = 29 + 15 + nv * (1 + 2 * (nv - 1))
    return per_cell + ndim * per_face + nv * 9


def mlp_flops_per_cell_rhs(ndim=2):
    """Algorithmic classifier flops of one cell's RHS: 2 x nv x ndim
    classifier calls (faces per cell x fields x sides) of 3104 multiply-adds."""
    nv = 4 if ndim == 2 else 3
    return 2 * nv * ndim * 2 * (6 * 64 + 64 * 32 + 32 * 16 + 16 * 8 + 8 * 4)


def mlp_grad_flops_per_sample():
    """Algorithmic flops of one sample's loss gradient: the forward pass
    (3104 multiply-adds), the deltas of layers 4..1 (4x8 + 8x16 + 16x32 + 32x64
    multiply-adds) and the weight gradients (3104 multiply-adds)."""
    fwd = 6 * 64 + 64 * 32 + 32 * 16 + 16 * 8 + 8 * 4
    return 2 * (fwd + (4 * 8 + 8 * 16 + 16 * 32 + 32 * 64) + fwd)


def tensor_peak_tflops():
    """Dense 16-bit tensor-core rate (fp16 and bf16 run at the same rate):
    the sustained cuBLAS figure of MEASURED_PEAKS.json (the kernel runs inside
    a long step), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["bf16_tflops_sustained"])
        return v, "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS, seconds-long loop)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback: 1.7 PFLOP/s dense bf16 sustained"


def gpu_numa_cpus(dev_index):
    """(node, CPUs) of the NUMA node next to the GPU from sysfs, or None."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(dev_index)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        with open("/sys/bus/pci/devices/%s/numa_node" % bus) as f:
            node = int(f.read())
        if node < 0:
            return None
        with open("/sys/devices/system/node/node%d/cpulist" % node) as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        return (node, cpus) if cpus else None
    except Exception:
        return None


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[5 + k].lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import torch
    import paper_2207_08500_gb300 as neno6
    import synth

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    n = args.n
    cfl = 0.4
    weights = args.weights
    prec = args.precision
    solver = neno6.Neno6(ndim=2, nx=n, ny=n, bc=("periodic", "periodic"), precision=prec,
                         weights=weights)
    U0 = synth.quadrants_2d(n, n)  # seeded, identical on every rank (weak scaling)
    U = torch.from_numpy(U0).to(dev)
    stream = torch.cuda.current_stream()
    t_dev = torch.zeros(1, dtype=torch.float64, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        solver.step(U, cfl, t=t_dev)
    torch.cuda.synchronize()
    if solver.status():
        raise RuntimeError("non-physical state during warm-up")

    clocks = ClockSampler(dev.index)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        solver.step(U, cfl, t=t_dev)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clock_info = clocks.stop()

    # per-launch duration of the dominant kernel (the fused RHS), same
    # workload and launch configuration, on the launching stream
    dUdt = torch.empty_like(U)
    reps = max(3, args.steps)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for r in range(reps):
        solver.rhs(U, out=dUdt)
        ev[r + 1].record(stream)
    torch.cuda.synchronize()
    rhs_ms = [ev[r].elapsed_time(ev[r + 1]) for r in range(reps)]
    rhs_avg = sum(rhs_ms) / reps

    # end to end through the C ABI with host buffers: every step one
    # neno6_step_host call, which copies the (pinned) host state to the
    # device, steps it, copies the new state back and synchronises
    numa = gpu_numa_cpus(dev.index)
    prev_aff = os.sched_getaffinity(0) if numa else None
    if numa:
        # the pinned buffers' pages are placed by the allocating thread: on
        # the NUMA node next to the GPU
        os.sched_setaffinity(0, numa[1])
    try:
        host = torch.from_numpy(U0.copy()).pin_memory()
        out_host = torch.empty_like(host).pin_memory()
        out_host.copy_(host)
    finally:
        if prev_aff:
            os.sched_setaffinity(0, prev_aff)
    solver.step_host(host, cfl, out=out_host)  # allocates the call's device state
    torch.cuda.synchronize()
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    U.copy_(host, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = host.numel() * 8 / (h0.elapsed_time(h1) * 1e-3) / 1e9
    barrier()
    # two rounds of steps, each timed; the value is over all of them, the
    # rounds and a copy rate taken after them show a slowdown of the host
    # link during the loop (the link is shared with other users' GPUs)
    per_round = max(1, min(args.steps, 5))
    fe = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fe[0].record(stream)
    for r in range(2):
        for _ in range(per_round):
            solver.step_host(host, cfl, out=out_host)
        fe[r + 1].record(stream)
    torch.cuda.synchronize()
    e2e_steps = 2 * per_round
    e2e_ms = fe[0].elapsed_time(fe[2])
    e2e_rounds = [round(fe[r].elapsed_time(fe[r + 1]) / per_round, 3) for r in range(2)]
    h0.record(stream)
    U.copy_(host, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize()
    h2d_after = host.numel() * 8 / (h0.elapsed_time(h1) * 1e-3) / 1e9
    status = solver.status()

    # mixed precision against the FP64 GPU path (itself bit-exact with the
    # oracle) on the same state: decisions, dU/dt, and one RK3 step
    compare = None
    if prec != "fp64" and not args.no_compare:
        ref = neno6.Neno6(ndim=2, nx=n, ny=n, bc=("periodic", "periodic"), precision="fp64",
                          weights=weights)
        S0 = torch.from_numpy(U0).to(dev)
        d64, m64 = ref.rhs(S0, want_mask=True)
        solver.guard_count(reset=True)
        dmx, mmx = solver.rhs(S0, want_mask=True)
        guard_rows = solver.guard_count()
        flips = int(np.unpackbits(torch.bitwise_xor(m64, mmx).cpu().numpy()).sum())
        a, b = dmx.double(), d64
        rhs_l1 = ((a - b).abs().sum() / b.abs().sum()).item()
        rhs_linf = ((a - b).abs().max() / b.abs().max()).item()
        rhs_l1_field = ((a - b).abs().sum(dim=(1, 2)) / b.abs().sum(dim=(1, 2))).tolist()
        del d64, dmx
        A, B = S0.clone(), S0.clone()
        ta = torch.zeros(1, dtype=torch.float64, device=dev)
        tb = torch.zeros(1, dtype=torch.float64, device=dev)
        # one RK3 step of each path from the same state: the state error
        ref.step(A, cfl, t=ta)
        solver.step(B, cfl, t=tb)
        torch.cuda.synchronize()
        st_l1 = ((B - A).abs().sum() / A.abs().sum()).item()
        st_linf = ((B - A).abs().max() / A.abs().max()).item()
        # FP64 path speed: that step was its warm-up; three more timed
        fp64_steps = 3
        ev64 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev64[0].record(stream)
        for _ in range(fp64_steps):
            ref.step(A, cfl, t=ta)
        ev64[1].record(stream)
        torch.cuda.synchronize()
        fp64_ms = ev64[0].elapsed_time(ev64[1]) / fp64_steps
        compare = {
            "fp64_gpu_value": round(n * n / (fp64_ms * 1e-3) / 1e6, 4), "unit": UNIT,
            "fp64_gpu_ms_per_step": round(fp64_ms, 3),
            "fp64_gpu_timing": "mean of %d SSP-RK3 steps after one untimed step" % fp64_steps,
            "mask_flip_rate": flips / (8.0 * m64.numel()),
            "rhs_rel_l1": rhs_l1, "rhs_rel_linf": rhs_linf,
            "rhs_rel_l1_per_field": rhs_l1_field,
            "state_rel_l1_one_step": st_l1, "state_rel_linf_one_step": st_linf,
            "reference": "FP64 GPU path (bit-exact with the FP64 oracle in the parity tests)",
            "guard_tau": solver.config.guard_tau,
            "guard_reevaluated_fraction": guard_rows / (2.0 * m64.numel()),
        }
        ref.close()
        del A, B, S0, m64, mmx

    # secondary rows (outside the timed region): the frozen-mask adjoint at
    # 1024^2 and the classifier backward on 2^20 stencils
    extra = {}
    if not args.no_extra:
        nv_ = 1024
        g64 = neno6.Neno6(ndim=2, nx=nv_, ny=nv_, precision="fp64", weights=weights)
        Uv = torch.from_numpy(synth.smooth_2d(nv_, nv_, seed=11)).to(dev)
        lam = torch.from_numpy(synth.normal((4, nv_, nv_), seed=12)).to(dev)
        _, maskv = g64.rhs(Uv, want_mask=True)
        gv = g64.rhs_vjp(Uv, lam, mask=maskv)
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_a.record(stream)
        for _ in range(2):
            g64.rhs_vjp(Uv, lam, mask=maskv, out=gv)
        e_b.record(stream)
        torch.cuda.synchronize()
        vjp_ms = e_a.elapsed_time(e_b) / 2
        extra["vjp_fp64_1024"] = {"ms_per_vjp": round(vjp_ms, 3),
                                  "Mcell_evals_per_s": round(nv_ * nv_ / vjp_ms / 1e3, 3)}
        Xs = torch.from_numpy(synth.mlp_stencils(1 << 20)).to(dev)
        ys = torch.zeros(1 << 20, dtype=torch.uint8, device=dev)
        ys[1 << 19:] = 0b1011
        g64.mlp_bwd(Xs, ys)
        e_a.record(stream)
        for _ in range(3):
            g64.mlp_bwd(Xs, ys)
        e_b.record(stream)
        torch.cuda.synchronize()
        extra["mlp_bwd_2^20"] = {"ms_per_call": round(e_a.elapsed_time(e_b) / 3, 3),
                                 "arithmetic": "FP32, CUDA cores (FP64 handle)"}
        # the same gradient on the tensor cores (fp16 handle)
        g16 = neno6.Neno6(ndim=1, nx=8, precision="fp16", weights=weights)
        g16.mlp_bwd(Xs, ys)
        e_a.record(stream)
        for _ in range(3):
            g16.mlp_bwd(Xs, ys)
        e_b.record(stream)
        torch.cuda.synchronize()
        tc_ms = e_a.elapsed_time(e_b) / 3
        tfl = (1 << 20) * mlp_grad_flops_per_sample()
        tpeak, tsrc = tensor_peak_tflops()
        extra["mlp_bwd_tc_2^20"] = {
            "ms_per_call": round(tc_ms, 3), "arithmetic": "fp16 operands, FP32 accumulation, tcgen05",
            "speedup_vs_fp32": round(extra["mlp_bwd_2^20"]["ms_per_call"] / tc_ms, 2),
            "tensor": {"achieved": round(tfl / (tc_ms * 1e-3) / 1e12, 2), "peak": tpeak, "unit": "TFLOP/s",
                       "frac": round(tfl / (tc_ms * 1e-3) / 1e12 / tpeak, 4),
                       "flops_per_call": tfl, "peak_source": tsrc}}
        g16.close()
        # the 709 000 samples of Algorithm 1 / Table 9 generated on the GPU
        # from seeded uniform draws, then one training epoch of the Table 2
        # recipe on their 70 % training share: 496 300 samples, batch 175, Adam
        n_all = 709000
        ud = torch.from_numpy(np.random.default_rng(17).random((n_all, 9))).to(dev)
        g64.datagen(ud[:1024])
        e_a.record(stream)
        Xall, yall, _ = g64.datagen(ud)
        e_b.record(stream)
        torch.cuda.synchronize()
        dg_ms = e_a.elapsed_time(e_b)
        extra["datagen_709000"] = {"ms": round(dg_ms, 3), "Msamples_per_s": round(n_all / dg_ms / 1e3, 1)}
        n_tr = 496300
        Xt, yt = Xall[:n_tr], yall[:n_tr]
        perm = torch.randperm(n_tr, generator=torch.Generator().manual_seed(15)).to(dev, torch.int32)
        params = torch.from_numpy(he_init_params(seed=16)).to(dev)
        mom = [torch.zeros_like(params), torch.zeros_like(params)]
        g64.mlp_train(Xt, yt, perm[:1750], params, mom[0], mom[1], 0, 1e-4)
        e_a.record(stream)
        ls = g64.mlp_train(Xt, yt, perm, params, mom[0], mom[1], 10, 1e-4)
        e_b.record(stream)
        torch.cuda.synchronize()
        ep_ms = e_a.elapsed_time(e_b)
        steps_ep = (n_tr + 174) // 175
        extra["mlp_train_epoch"] = {"samples": n_tr, "batch": 175, "steps": steps_ep,
                                    "ms_per_epoch": round(ep_ms, 1),
                                    "us_per_step": round(ep_ms * 1e3 / steps_ep, 2),
                                    "mean_batch_loss": round(ls.item() / steps_ep, 5)}
        g64.close()
        del Uv, lam, gv, maskv, Xs, ys
        # width study: neno6_classify throughput of the paper's network and
        # of the 6-32-32-32-4 network on 2^22 stencils (FP64 and fp16)
        Xw = torch.from_numpy(synth.mlp_stencils(1 << 22, seed=18)).to(dev)
        narrow_w = os.path.join(os.path.dirname(neno6.DEFAULT_WEIGHTS), "neno6_mlp_6x32x32x32x4.bin")
        wst = {}
        for label, wpath in (("6-64-32-16-8-4", neno6.DEFAULT_WEIGHTS), ("6-32-32-32-4", narrow_w)):
            for wprec in ("fp64", "fp16"):
                gw = neno6.Neno6(ndim=1, nx=8, precision=wprec, weights=wpath)
                gw.classify(Xw[:4096])
                e_a.record(stream)
                for _ in range(3):
                    gw.classify(Xw)
                e_b.record(stream)
                torch.cuda.synchronize()
                wst[label + " " + wprec] = round(3 * Xw.shape[0] / e_a.elapsed_time(e_b) / 1e6, 2)
                gw.close()
        extra["classify_Gstencils_per_s"] = wst
        del Xw

    ms, e2e_ms, rhs_avg = max_over_ranks([ms, e2e_ms, rhs_avg], world, dev)

    cells = n * n
    value = cells * args.steps * world / (ms * 1e-3) / 1e6
    e2e_value = cells * e2e_steps * world / (e2e_ms * 1e-3) / 1e6
    if prec == "fp64":
        fl = flops_per_cell_rhs(2) * cells
        kname = "rhs_fp64_kernel"
        fl_note = "all binary64 flops of the scheme (bench.flops_per_cell_rhs)"
        launches_per_step = 4
    else:
        fl = fp64_flops_per_cell_rhs_mixed(2) * cells
        kname = "faces_mixed_kernel + diff_mixed_kernel (one RHS)"
        fl_note = ("binary64 flops of the parts the mixed path keeps in FP64 "
                   "(bench.fp64_flops_per_cell_rhs_mixed); FP32 and tensor-core work not counted")
        launches_per_step = 8
    achieved = fl / (rhs_avg * 1e-3) / 1e12
    # the FP64 and FP32 FMA rates measured on this GPU in the same run: the
    # FP64 one is the roofline's peak
    meas64 = neno6.pipe_peak("fp64") / 1e12
    meas32 = neno6.pipe_peak("fp32") / 1e12
    peak = meas64
    tensor = None
    if prec != "fp64":
        # the classifier's multiply-adds (16 calls per cell and RHS) against
        # the tensor cores' measured dense 16-bit rate
        tfl = mlp_flops_per_cell_rhs() * cells
        tpeak, tsrc = tensor_peak_tflops()
        tach = tfl / (rhs_avg * 1e-3) / 1e12
        tensor = {"achieved": round(tach, 2), "peak": tpeak, "unit": "TFLOP/s",
                  "frac": round(tach / tpeak, 4), "flops_per_launch": tfl, "peak_source": tsrc}
    state_bytes = U.numel() * 8
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "%s+f32+f64" % prec,
        "data": "synthetic (seeded four-quadrant Euler states, trained frozen classifier)",
        "config": {"workload": workload_name(n, prec),
                   "nx": n, "ny": n, "precision": prec, "step": "one SSP-RK3 step = 3 RHS",
                   "l2": "inputs larger than L2 (state %d MB)" % (state_bytes >> 20),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "kernel": kname, "flops_counted": fl_note,
                     "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": traffic_bytes(prec, n),
                     "traffic_source": TRAFFIC_NOTE[prec == "fp64"],
                     "peak_source": "measured in this run: DFMA chains on every SM (neno6_pipe_peak)",
                     "nominal_fp64_tflops": fp64_peak_tflops(),
                     "frac_of_nominal_fp64": round(achieved / fp64_peak_tflops(), 4),
                     "flops_per_launch": fl, "ms_per_launch": round(rhs_avg, 3),
                     "fp32_fma_measured_tflops": round(meas32, 2),
                     "tensor": tensor},
        "e2e": {"value": round(e2e_value, 4), "unit": UNIT,
                "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                "steps": e2e_steps, "ms_per_step_by_round": e2e_rounds,
                "h2d_copy_gbs": round(h2d_gbs, 1), "h2d_copy_gbs_after": round(h2d_after, 1),
                "pinned_host_numa_node": numa[0] if numa else None},
        "gpu_launches": launches_per_step * args.steps,
        "vs_fp64_gpu": compare,
        "precision_note": PRECISION_NOTE.get(prec),
        "secondary": extra,
        "clocks": clock_info,
        "device_status": status,
        "weights_sha256": weights_sha256(weights),
    }
    return line


# What the 100-step accuracy runs (2048^2, against the FP64 path) showed for
# each classifier precision.
PRECISION_NOTE = {
    "fp16": "fp16 (guard tau 0.5) stays within 1e-6 relative L1 of the FP64 state over the 99-step 2048^2 run "
            "(7.1e-7); bf16 does not (6.7e-6 at tau 1.0, 1.24e-6 at tau 4.0, 1.22e-6 with every row in FP32)",
    "bf16": "bf16 does not stay within 1e-6 relative L1 of the FP64 state over the 99-step 2048^2 run "
            "(6.7e-6 at tau 1.0, 1.24e-6 at tau 4.0, 1.22e-6 with every row in FP32); only fp16 does (7.1e-7)",
}


# DRAM bytes (read + write) of one launch of the dominant kernel(s), from one
# ncu capture of the current kernels at the grid named (dram__bytes_read.sum
# + dram__bytes_write.sum, a single-pass capture); other grids: None
TRAFFIC = {True: (2048, 141937152 + 94543104),
           False: (4096, 1212746496 + 1051745536 + 1074054656 + 507911424)}
TRAFFIC_NOTE = {True: "rhs_fp64_kernel at 2048^2, one launch: 141.9 MB read + 94.5 MB written",
                False: "one RHS at 4096^2: faces_mixed_kernel 1212.7 MB read + 1051.7 MB written, "
                       "diff_mixed_kernel 1074.1 MB read + 507.9 MB written"}


def traffic_bytes(prec, n):
    grid, b = TRAFFIC[prec == "fp64"]
    return b if (b is not None and grid == n) else None


def max_over_ranks(values, world, device):
    """Element-wise maximum of `values` (floats) over all ranks of the
    default process group (the job's time is its slowest rank's)."""
    import torch
    vals = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(vals, op=torch.distributed.ReduceOp.MAX)
    return vals.tolist()


def he_init_params(seed):
    """Seeded He-style initial parameters of the 6-64-32-16-8-4 network in
    weights-file order (float32), for the training timing."""
    rng = np.random.default_rng(seed)
    widths = [6, 64, 32, 16, 8, 4]
    parts = []
    for a, b in zip(widths[:-1], widths[1:]):
        parts.append(rng.standard_normal(a * b) * np.sqrt(2.0 / a))
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


def weights_sha256(path):
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def fp64_peak_tflops():
    """FP64-pipe peak: DFMA rate per SM per clock (2 on GB300; ncu reports
    the same sustained peak, 2 DFMA thread instructions per cycle per SM) x
    SMs x 2 flops x maximum SM clock."""
    dfma_per_clk_sm = 2.0
    return round(dfma_per_clk_sm * SMS * 2 * 2070e6 / 1e12, 4)


# ---------------------------------------------------------- oracle arm
def host_cores():
    return len(os.sched_getaffinity(0))


def oracle_timing(crop=64, reps=1, threads=1):
    """The FP64 CPU oracle on a periodic crop of the workload (same
    generator, crop x crop cells): one SSP-RK3 step per rep, on `threads`
    host threads (OpenMP over the faces)."""
    import oracle
    import synth
    from oracle.weights import Net
    net = Net.load(WEIGHTS) if os.path.exists(WEIGHTS) else Net.random()
    oracle.set_threads(threads)
    o = oracle.Oracle(ndim=2, nx=crop, ny=crop, net=net)
    U = synth.quadrants_2d(crop, crop)
    t0 = time.perf_counter()
    for _ in range(reps):
        U, _, _ = o.step(U, 0.4)
    dt = time.perf_counter() - t0
    return crop * crop * reps / dt / 1e6, dt


def oracle_rhs_rate(n, threads):
    """Cell-RHS evaluations per second (millions) of the FP64 oracle on the
    n x n periodic quadrant workload: one full RHS on `threads` threads."""
    import oracle
    import synth
    from oracle.weights import Net
    net = Net.load(WEIGHTS) if os.path.exists(WEIGHTS) else Net.random()
    got = oracle.set_threads(threads)
    o = oracle.Oracle(ndim=2, nx=n, ny=n, net=net)
    U = synth.quadrants_2d(n, n)
    t0 = time.perf_counter()
    o.rhs(U)
    dt = time.perf_counter() - t0
    return n * n / dt / 1e6, dt, got


def cpu_baseline_line(args):
    """The oracle on this host: all cores at each of --cpu-sizes, one core at
    the smallest; the value is the all-core rate at the largest size, as
    cell-updates (one update = three RHS)."""
    cores = host_cores()
    sizes = sorted(int(x) for x in args.cpu_sizes.split(",") if x)
    per, total = {}, 0.0
    for n in sizes:
        r, secs, used = oracle_rhs_rate(n, cores)
        per[str(n)] = {"all_cores_Mcell_rhs_per_s": round(r, 6), "threads": used, "seconds": round(secs, 2)}
        total += secs
    one = [n for n in sizes if n <= 1024] or sizes[:1]
    for n in one:
        r1, secs1, _ = oracle_rhs_rate(n, 1)
        per[str(n)]["one_core_Mcell_rhs_per_s"] = round(r1, 6)
        total += secs1
    top = per[str(sizes[-1])]["all_cores_Mcell_rhs_per_s"]
    return {"value": round(top / 3.0, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "one FP64 oracle RHS of the %d^2 periodic quadrant workload on all %d host cores "
                      "(OpenMP over faces), as cell-updates/s = cell-RHS/s / 3; also %s on all cores and "
                      "%s on one core (%.1f s of wall time in all)" % (
                          sizes[-1], cores, ", ".join("%d^2" % n for n in sizes[:-1]) or "no other size",
                          ", ".join("%d^2" % n for n in one), total),
            "per_size": per}


def workload_name(n, prec):
    return "2D Euler %dx%d periodic, %s NENO6 RHS, SSP-RK3 (CFL 0.4)" % (
        n, n, "FP64" if prec == "fp64" else "mixed-precision (%s classifier)" % prec)


def run_reference(args):
    cores = host_cores()
    oracle_timing(16, 1, cores)  # build + warm the oracle library
    for _ in range(args.warmup):
        oracle_timing(args.ref_crop, 1, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_timing(args.ref_crop, 1, cores)
    dt = time.perf_counter() - t0
    value = args.ref_crop ** 2 * args.steps / dt / 1e6
    sample = ("one FP64 SSP-RK3 step of the oracle on a %dx%d periodic crop of the %d^2 "
              "workload per step, %d host threads (OpenMP over faces)" % (
                  args.ref_crop, args.ref_crop, args.n, cores))
    return {
        "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": 1, "impl": "reference",
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(args.n, args.precision),
                                        "sample": sample},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def run_rhs_only(args):
    """`--rhs-only` / `--vjp-only`: warm-up + `--steps` plain RHS (or
    frozen-mask adjoint) evaluations, a case for profilers; prints one line,
    no timing."""
    import torch
    import paper_2207_08500_gb300 as neno6
    import synth
    n = args.n
    prec = "fp64" if args.vjp_only else args.precision
    g = neno6.Neno6(ndim=2, nx=n, ny=n, precision=prec, weights=args.weights)
    U = torch.from_numpy(synth.quadrants_2d(n, n)).cuda()
    d = torch.empty_like(U)
    if args.vjp_only:
        lam = torch.from_numpy(synth.normal(U.shape, seed=12)).cuda()
        _, mask = g.rhs(U, want_mask=True)
    for _ in range(args.warmup + args.steps):
        if args.vjp_only:
            g.rhs_vjp(U, lam, mask=mask, out=d)
        else:
            g.rhs(U, out=d)
    torch.cuda.synchronize()
    print(json.dumps({"vjp_only" if args.vjp_only else "rhs_only": True, "n": n, "precision": prec,
                      "launches": args.warmup + args.steps, "status": g.status()}))


def run_mlp_bwd_only(args):
    """`--mlp-bwd-only`: warm-up + `--steps` classifier gradients (Eq.
    (Crossentropy)) on 2^20 synthetic stencils with a mixed-precision handle
    (the tensor-core kernel; `--precision fp64` gives the FP32 CUDA-core
    kernel), a case for profilers; prints one line, no timing."""
    import torch
    import paper_2207_08500_gb300 as neno6
    import synth
    n = 1 << 20
    g = neno6.Neno6(ndim=1, nx=8, precision=args.precision, weights=args.weights)
    X = torch.from_numpy(synth.mlp_stencils(n)).cuda()
    y = torch.zeros(n, dtype=torch.uint8, device="cuda")
    y[n // 2:] = 0b1011
    for _ in range(args.warmup + args.steps):
        g.mlp_bwd(X, y)
    torch.cuda.synchronize()
    print(json.dumps({"mlp_bwd_only": True, "n": n, "precision": args.precision,
                      "launches": args.warmup + args.steps, "status": g.status()}))


def run_mlp_train_only(args):
    """`--mlp-train-only`: warm-up + `--steps` calls of the training loop
    (Sec. 3.3, Table 2: Adam, batch 175) over 100 batches of Table 9 samples
    generated on the GPU, a case for profilers; prints one line, no timing."""
    import torch
    import paper_2207_08500_gb300 as neno6
    g = neno6.Neno6(ndim=1, nx=8, weights=args.weights)
    n = 175 * 100
    u = torch.from_numpy(np.random.default_rng(17).random((n, neno6.DATAGEN_DRAWS))).cuda()
    X, y, _ = g.datagen(u)
    perm = torch.randperm(n, generator=torch.Generator().manual_seed(15)).to("cuda", torch.int32)
    params = torch.from_numpy(he_init_params(seed=16)).cuda()
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    for k in range(args.warmup + args.steps):
        g.mlp_train(X, y, perm, params, m, v, 100 * k, 1e-4)
    torch.cuda.synchronize()
    print(json.dumps({"mlp_train_only": True, "samples": n, "batch": 175,
                      "launches": args.warmup + args.steps, "status": g.status()}))


def run_classify_only(args):
    """`--classify-only`: warm-up + `--steps` neno6_classify calls on `--n`
    sine / step stencils with the paper's network, then the same with the
    6-32-32-32-4 network of the width study (`--precision`), a case for
    profilers; prints one line, no timing."""
    import torch
    import paper_2207_08500_gb300 as neno6
    import synth
    X = torch.from_numpy(synth.mlp_stencils(args.n, seed=18)).cuda()
    narrow = os.path.join(os.path.dirname(neno6.DEFAULT_WEIGHTS), "neno6_mlp_6x32x32x32x4.bin")
    status = []
    for wpath in (neno6.DEFAULT_WEIGHTS, narrow):
        g = neno6.Neno6(ndim=1, nx=8, precision=args.precision, weights=wpath)
        for _ in range(args.warmup + args.steps):
            g.classify(X)
        torch.cuda.synchronize()
        status.append(g.status())
        g.close()
    print(json.dumps({"classify_only": True, "n": args.n, "precision": args.precision,
                      "launches_per_network": args.warmup + args.steps, "status": status}))


def run_oblique(args):
    """`--workload oblique`: 8192 x 4096 transmissive oblique-shock state
    (square cells on [0, 2] x [0, 1]), mixed-precision steps replayed from a
    CUDA graph of 100 captured SSP-RK3 steps, and after every 100 steps the
    frozen-mask FP64 adjoint of the RHS at the current state (its mask from
    the mixed-precision RHS, cotangent N(0,1)).  The timed region holds all
    of it; the value counts cell-updates (steps x cells)."""
    import torch
    import paper_2207_08500_gb300 as neno6
    import synth
    nx, ny = 8192, 4096
    kw = dict(ndim=2, nx=nx, ny=ny, dx=1.0 / ny, dy=1.0 / ny, bc=("transmissive", "transmissive"),
              weights=args.weights)
    prec = "bf16" if args.precision == "fp64" else args.precision
    g = neno6.Neno6(precision=prec, **kw)
    g64 = neno6.Neno6(precision="fp64", **kw)
    U = torch.from_numpy(synth.oblique_shock_2d(nx, ny)).cuda()
    lam = torch.from_numpy(synth.normal(tuple(U.shape), seed=12)).cuda()
    grad = torch.empty_like(U)
    dUdt = torch.empty_like(U)
    t_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    per = 100
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(max(1, args.warmup)):
            g.step(U, 0.4, t=t_dev)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(per):
            g.step(U, 0.4, t=t_dev)
    blocks = max(1, args.steps // per)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * blocks + 1)]
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for b in range(blocks):
        graph.replay()
        ev[2 * b + 1].record(stream)
        _, mask = g.rhs(U, want_mask=True, out=dUdt)
        g64.rhs_vjp(U, lam, mask=mask, out=grad)
        ev[2 * b + 2].record(stream)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    ms = ev[0].elapsed_time(ev[-1])
    vjp_ms = sum(ev[2 * b + 1].elapsed_time(ev[2 * b + 2]) for b in range(blocks)) / blocks
    status = g.status() | g64.status()
    steps = blocks * per
    return {
        "metric": METRIC, "value": round(nx * ny * steps / (ms * 1e-3) / 1e6, 4), "unit": UNIT,
        "n_gpus": 1, "steps": steps, "warmup": max(1, args.warmup),
        "ms_per_step": round(ms / steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "%s+f32+f64" % prec, "data": "synthetic (seeded oblique shock)",
        "config": {"workload": "2D Euler %dx%d transmissive oblique shock + density blobs, "
                               "mixed-precision (%s classifier) NENO6, SSP-RK3 (CFL 0.4) replayed "
                               "from a CUDA graph of %d steps, frozen-mask FP64 adjoint every %d "
                               "steps" % (nx, ny, prec, per, per),
                   "l2": "inputs larger than L2 (state %d MB)" % (U.numel() * 8 >> 20)},
        "adjoint_ms_per_call": round(vjp_ms, 3), "t_final": t_dev.item(),
        "gpu_launches": steps * 8 + blocks * 3, "clocks": clock_info, "device_status": status,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--precision", choices=["fp64", "bf16", "fp16"], default="fp16")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--rhs-only", action="store_true")
    ap.add_argument("--vjp-only", action="store_true")
    ap.add_argument("--classify-only", action="store_true")
    ap.add_argument("--mlp-bwd-only", action="store_true")
    ap.add_argument("--mlp-train-only", action="store_true")
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--ref-crop", type=int, default=192)
    ap.add_argument("--cpu-sizes", default="256,1024,2048")
    ap.add_argument("--workload", choices=["quadrants", "oblique"], default="quadrants")
    args = ap.parse_args()
    if args.workload == "oblique" and args.impl == "ours":
        print(json.dumps(run_oblique(args)))
        return
    if args.mlp_bwd_only:
        run_mlp_bwd_only(args)
        return
    if args.mlp_train_only:
        run_mlp_train_only(args)
        return
    if args.classify_only:
        args.n = args.n or (1 << 20)
        run_classify_only(args)
        return
    if args.n is None:
        args.n = 2048 if args.precision == "fp64" else 4096

    if args.rhs_only or args.vjp_only:
        run_rhs_only(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world)
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline_line(args)
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
