#!/usr/bin/env python
"""Fit throughput of Fourier-represented kernel regression on one B300.

Workload: 2-D Sobolev regression, n = 1e8 points X ~ U[-pi, pi)^2 (fp32),
Y = exp(-|X|^2) + N(0, 0.05^2), m = 32 (65 x 65 modes, 129 x 129 moments),
s = 2, lambda = 1e-6, NUFFT eps = 1e-6.  One step is one whole fit through the
C-ABI (fk_fit_sobolev): type-1 spreading of the ones and Y channels, FFT and
deconvolution to the moments T and right-hand side b, penalty assembly and the
FP64 conjugate-gradient solve.  Inputs (1.2 GB) are larger than L2, so no flush
runs between steps.

The same line carries, under "rows", the other hot-path rows at full size, each
timed with its own (smaller) step count, clocks and roofline: the additive model
(d = 8, n = 2e8), the physics-informed fit with its held-out-loss hypergradient
(n = 1e9) and the 1-D sweep (1e10 points, 256 lambdas x 16 targets).  FP32 peaks are
measured on the device (fk_peak_fp32); the mixed result is gated against the FP64
path at eps = 1e-12.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WL = dict(workload="2d-sobolev", d=2, n=100_000_000, m=32, s=2.0, lam=1e-6, eps=1e-6)
METRIC = "fit points/s (NUFFT Gram+RHS+solve)"
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (derived peak, reported beside the measured one)
ACC_DRAM_BYTES_PER_POINT = (241.220096e6 + 6.502656e6) / 2e7  # k_bin_accumulate, 2-D, w = 7
# k_bin_accumulate on the additive model's pair records: one launch serves the 7 partners
# of coordinate 0 (DRAM bytes per point and partner)
ADD_ACC_DRAM_BYTES_PER_POINT_PAIR = (646.954496e6 + 7.005440e6) / (2e7 * 7)
SPREAD1D_DRAM_BYTES_PER_POINT = (5.09e9 + 5.1e6) / 67108864  # k_spread1d_fx, 17 channels


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # a step takes a few ms: 100 steps make the timed region ~0.35 s, long enough that the
    # nvidia-smi clock sampling running during it (each query stalls the GPU ~3 ms) costs ~2 %
    ap.add_argument("--steps", type=int, default=None, help="default: 100 (2d-sobolev), 3 (sweep-1d), 20 (others)")
    ap.add_argument("--warmup", type=int, default=None, help="default: 5 (2d-sobolev), 1 (sweep-1d), 3 (others)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=WL["n"],
                    help="points (default: 1e8 for 2d-sobolev; sweep-1d: total points, default 1e10)")
    ap.add_argument("--spread", default="auto", choices=["auto", "atomic", "binned"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="skip the graph-replay measurements (headline and additive rows)")
    ap.add_argument("--no-rows", action="store_true",
                    help="headline line only (skip the sweep-1d, pik-heat and additive-8d rows)")
    ap.add_argument("--workload", default="2d-sobolev", choices=["2d-sobolev", "sweep-1d", "pik-heat", "additive-8d"],
                    help="2d-sobolev is the headline line; the others time the other hot-path rows")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = {"2d-sobolev": 100, "sweep-1d": 3}.get(a.workload, 20) if a.impl == "ours" else 10
    if a.warmup is None:
        a.warmup = {"2d-sobolev": 5, "sweep-1d": 1}.get(a.workload, 3)
    return a


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp32_peak(fk):
    """Measured FP32 FMA throughput (fk_peak_fp32) and the derived one, in TFLOP/s."""
    import torch
    measured, sms = fk.fk_peak_fp32()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = sms or props.multi_processor_count
    sm_max = measured_peaks().get("sm_max_mhz", 2032.0)
    derived = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    return {"measured": measured, "derived": derived, "sm_count": sms,
            "basis": "of measured: fk_peak_fp32 (FFMA chains, 2048 threads per SM, best of 3 launches); derived = "
                     "%d SMs x %d FP32 lanes x 2 flop x %.0f MHz" % (sms, FP32_LANES_PER_SM, sm_max)}


def host_cores():
    try:
        from threadpoolctl import threadpool_info
        th = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if th:
            return int(max(th))
    except Exception:
        pass
    return os.cpu_count() or 1


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled while the timed region runs:
    every 10 ms through NVML (so that a 40 ms region still gets a few samples), every
    200 ms through nvidia-smi.

    The samples come from NVML (libnvidia-ml, the library nvidia-smi reads) through
    ctypes: an `nvidia-smi -lms 200` process stalled the GPU for ~10 ms per query,
    6.5 % of the measured step, while these queries cost no measurable time.
    Without NVML the sampler falls back to nvidia-smi."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    # NVML clocks-event reason bits
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
            "hw_power_brake_slowdown": 0x80}

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.nvml = None
        self.samples = []
        self.source = None

    def _nvml_open(self):
        import ctypes
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(self.index, ctypes.byref(h)) != 0:
                return None
            return nv, h
        except OSError:
            return None

    def __enter__(self):
        import threading
        self.nvml = self._nvml_open()
        if self.nvml is not None:
            import ctypes
            nv, h = self.nvml
            clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
            nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))  # NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
            self.stop = threading.Event()

            def run():
                while not self.stop.is_set():
                    if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and \
                            nv.nvmlDeviceGetCurrentClocksEventReasons(h, ctypes.byref(rs)) == 0:
                        self.samples.append((float(clk.value), int(rs.value)))
                    self.stop.wait(0.01)

            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            self.source = "nvml"
        else:
            try:
                self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                              "--format=csv,noheader,nounits", "-lms", "200"],
                                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.source = "nvidia-smi"
            except Exception:
                self.proc = None
            time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.nvml is not None:
            self.stop.set()
            self.thread.join(timeout=5)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        if self.nvml is not None:
            mx = self.max_mhz
            for c, r in self.samples:
                sm.append(c)
                for nm, bit in self.BITS.items():
                    if r & bit:
                        reasons.add(nm)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "source": self.source}


def make_inputs(n: int):
    import synthetic as S
    x, y = S.wl2_sobolev_2d(n, dtype=np.float32)
    return np.ascontiguousarray(x), np.ascontiguousarray(y)


def cpu_oracle_fit(x, y, m, s, lam):
    import oracle as O
    t0 = time.perf_counter()
    th = O.fit(x.astype(np.float64), y.astype(np.float64), m, O.penalty_sobolev(2, m, lam, s))
    return time.perf_counter() - t0, th


def run_reference(args, rank):
    """The CPU oracle as it stands, timed on this machine's host cores."""
    if rank != 0:
        return
    n_o = 50_000
    x, y = make_inputs(n_o)
    for _ in range(args.warmup):
        cpu_oracle_fit(x[:, :2000], y[:2000], WL["m"], WL["s"], WL["lam"])
    times = [cpu_oracle_fit(x, y, WL["m"], WL["s"], WL["lam"])[0] for _ in range(args.steps)]
    t = statistics.median(times)
    v = n_o / t
    cores = host_cores()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WL["workload"], "n": n_o, "d": 2, "m": WL["m"], "s": WL["s"], "lambda": WL["lam"],
                       "eps": WL["eps"], "note": "oracle fit on a %d-point sample of the workload" % n_o},
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": cores, "kind": "oracle",
                             "sample": "%d points of the workload; direct sums + dense solve D=4225" % n_o},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _dev_uniform(torch, n, d, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.rand((d, n), generator=g, device="cuda", dtype=torch.float32) * (2 * np.pi) - np.pi


def _dev_normal(torch, n, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.randn(n, generator=g, device="cuda", dtype=torch.float32)


def run_row(args, rank, local, W=None, steps=None, warmup=None, peak=None, n=None):
    """Time one of the other hot-path rows on one GPU (inputs drawn on the device).

    sweep-1d:    1e10 points (2^28-point chunks from the counter-based generator; the
                 generation is outside the timed region), 17 channels on one 1-D grid,
                 then the batched solve for 256 lambdas x 16 targets.
    pik-heat:    n = 1e9 (t, x) points, heat prior, fit + held-out loss and its
                 gradient (autograd) on 1e7 validation points.
    additive-8d: n = 2e8 points in d = 8, m = 64: 8 1-D and 28 2-D transforms,
                 block Gram and dense FP64 solve.
    n overrides the point count (smaller cases for profiling); --no-autotune keeps
    the spreaders' default shapes.  Returns the row's JSON object."""
    import torch
    import paper_2509_02649_b300 as fk
    torch.cuda.set_device(local)
    tune = 0 if args.no_autotune else 1
    st = torch.cuda.current_stream()
    W = W or args.workload
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    peak = peak or fp32_peak(fk)
    p32 = peak["measured"]
    if W == "sweep-1d":
        n_total = n or 10_000_000_000
        chunk, m, nt = min(1 << 28, (n_total + 3) // 4 * 4), 1000, 16
        lams = list(np.logspace(-12, -2, 256))
        x = torch.empty((1, chunk), dtype=torch.float32, device="cuda")
        y = torch.empty((nt, chunk), dtype=torch.float32, device="cuda")
        amax = torch.empty(nt, dtype=torch.int32, device="cuda")
        acc = fk.Accumulator(1, m, nt, 1e-6, "mixed", opts=fk.default_opts(autotune=tune))

        def step():
            ev = []
            first = 0
            while first < n_total:
                c = min(chunk, n_total - first)
                xs, ys = (x, y) if c == chunk else (torch.empty((1, c), dtype=torch.float32, device="cuda"),
                                                    torch.empty((nt, c), dtype=torch.float32, device="cuda"))
                fk.generate_sweep_1d(first, c, nt, out=(xs, ys, amax))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                acc.add(xs, ys, amax)
                e1.record(st)
                ev.append((e0, e1))
                first += c
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(st)
            th = acc.fit_sobolev(1.0, lams)
            f1.record(st)
            torch.cuda.synchronize()
            acc.reset()
            ms_add = sum(a.elapsed_time(b) for a, b in ev)
            return ms_add + f0.elapsed_time(f1), ms_add, th

        n, f_pt = n_total, 7 * (2 * (1 + nt))
        cfg = {"workload": W, "n": n_total, "d": 1, "m": m, "s": 1.0, "n_lambda": 256, "n_targets": nt, "eps": 1e-6,
               "chunk": chunk, "timed": "spreading of every chunk + transform + batched solve; generation excluded"}
        kern = "k_spread1d_fx (fixed-point shared-memory spreading, 17 channels)"
        traffic = SPREAD1D_DRAM_BYTES_PER_POINT * chunk
        traffic_note = ("ncu capture of k_spread1d_fx at n = 2^26 (5.09 GB read + 5.1 MB written), scaled to one "
                        "launch (one 2^28-point chunk)")
    elif W == "pik-heat":
        n, nv, m = (n or 1_000_000_000), 10_000_000, 25
        x = _dev_uniform(torch, n, 2, 11)
        y = torch.exp(-0.1 * x[0]) * torch.sin(x[1]) + 0.1 * _dev_normal(torch, n, 12)
        xv = _dev_uniform(torch, nv, 2, 13)
        yv = torch.exp(-0.1 * xv[0]) * torch.sin(xv[1]) + 0.1 * _dev_normal(torch, nv, 14)
        alpha = [[1, 0], [0, 2]]

        def step():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            lt = torch.tensor(1e-8, dtype=torch.float64, requires_grad=True)
            mt = torch.tensor(1e-2, dtype=torch.float64, requires_grad=True)
            at = torch.tensor([1.0, -0.1], dtype=torch.float64, requires_grad=True)
            L = fk.heldout_loss(y, lt, torch.tensor(1.0, dtype=torch.float64), mt, at, x, xv, yv, m, alpha, 1e-6)
            L.backward()
            e1.record(st)
            torch.cuda.synchronize()
            _, rep = fk.fk_fit_pik(x, y, m, 1.0, 1e-8, 1e-2, alpha, [1.0, -0.1], 1e-6, "mixed", report=True,
                                   opts=fk.default_opts(autotune=tune))
            return e0.elapsed_time(e1), rep["ms_kernel"], (L.item(), lt.grad.item(), mt.grad.item())

        f_pt = 49 * (2 * 2 + 1)
        cfg = {"workload": W, "n": n, "n_val": nv, "d": 2, "m": m, "s": 1.0, "lambda": 1e-8, "mu": 1e-2,
               "operator": "d_t - 0.1 d_xx", "eps": 1e-6,
               "timed": "fit + held-out loss + hypergradient (autograd forward and backward)"}
        kern = "k_bin_accumulate (register-accumulation spreading, training fit)"
        traffic = ACC_DRAM_BYTES_PER_POINT * n
        traffic_note = ("ncu capture of k_bin_accumulate at n = 2e7 (2-D sobolev, the same 256^2 grid and w = 7), "
                        "scaled to one launch by points")
    else:
        n, d, m = (n or 200_000_000), 8, 64
        lam = n ** (-0.8)
        x = _dev_uniform(torch, n, d, 41)
        y = 0.1 * _dev_normal(torch, n, 42)
        for j in range(d):
            y += torch.sin((j + 1) * x[j]) / (j + 1)

        def step():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            th, rep = fk.fk_fit_additive(x, y, m, [lam], 1e-6, "mixed", report=True, opts=fk.default_opts(autotune=tune))
            e1.record(st)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1), rep["ms_spread"], rep

        f_pt = 8 * 7 * 3 + 28 * 49 * 3  # 8 1-D transforms (ones + y) and 28 2-D transforms of ones
        cfg = {"workload": W, "n": n, "d": d, "m": m, "lambda": lam, "eps": 1e-6,
               "timed": "8 1-D + 28 2-D type-1 transforms, block Gram, dense FP64 solve"}
        kern = "all spreading kernels of the 36 transforms"
        traffic = ADD_ACC_DRAM_BYTES_PER_POINT_PAIR * n * (d - 1)
        traffic_note = ("ncu capture of the pair accumulation (k_bin_accumulate on row-owner records) for the "
                        "%d partners of coordinate 0 at n = 2e7 (647.0 MB read + 7.0 MB written), scaled to that "
                        "launch at this n" % (d - 1))
    for _ in range(max(1, warmup)):
        step()
    torch.cuda.synchronize()
    launches0 = fk.fk_launch_count()
    res = []
    with ClockSampler(local) as clk:
        for _ in range(steps):
            res.append(step())
    launches = (fk.fk_launch_count() - launches0) // max(1, steps)
    ms = statistics.median(r[0] for r in res)
    mk = statistics.median(r[1] for r in res)
    achieved = f_pt * n / (mk / 1e3) / 1e12
    line = {"metric": "fit points/s (" + W + ")", "value": n / (ms / 1e3), "unit": "points/s", "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (drawn on the device)",
            "config": cfg, "gpu_launches_per_step": launches,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": p32, "unit": "TFLOP/s", "frac": achieved / p32,
                         "traffic": traffic, "traffic_basis": traffic_note, "kernel": kern, "flop_per_point": f_pt,
                         "ms_kernel": mk, "peak_basis": peak["basis"], "peak_derived": peak["derived"],
                         "frac_of_derived": achieved / peak["derived"]},
            "clocks": clk.summary()}
    if W == "sweep-1d":
        # the spreader is bound by its shared-memory atomics (one 32-bit add per tap and
        # channel): its rate against the measured peaks of that operation
        dist, rnd = fk.fk_peak_smem_atomics()
        ops = 7 * (1 + nt) * n / (mk / 1e3) / 1e9
        line["atomic_view"] = {"achieved": ops, "unit": "G lane ops/s", "atomics_per_point": 7 * (1 + nt),
                               "peak_distinct_banks": dist, "frac_distinct_banks": ops / dist,
                               "peak_random_windows": rnd, "frac_random_windows": ops / rnd,
                               "basis": "of measured: fk_peak_smem_atomics (32-bit adds with returned value, "
                                        "windows of 7 words, two 1024-thread CTAs per SM)"}
    line["autotune"] = fk.fk_autotune_table().strip() or None
    if W == "pik-heat":
        line["loss_and_grads"] = {"L": res[-1][2][0], "dL/dlambda": res[-1][2][1], "dL/dmu": res[-1][2][2]}
    if W == "additive-8d":
        line["report"] = res[-1][2]
        # a grid search over 300 lambdas (the paper's Sec. 5 experiment) from one transform
        # pass: one eigendecomposition for all lambdas against one Cholesky solve per lambda
        lams300 = list(np.logspace(-6, -1, 300))
        sweep = {}
        for name, solver in (("eigen", fk.FK_SOLVER_EIG), ("cholesky", fk.FK_SOLVER_CHOL)):
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(st)
            th300, rep300 = fk.fk_fit_additive(x, y, m, lams300, 1e-6, "mixed", report=True,
                                               opts=fk.default_opts(autotune=tune, solver=solver))
            s1.record(st)
            torch.cuda.synchronize()
            sweep[name] = {"ms": s0.elapsed_time(s1), "ms_solve": rep300["ms_solve"], "theta": th300}
        # what the estimator determines: the coefficients with k != 0 and the sum of the d
        # intercepts (their differences are fixed by lambda alone, condition ~ d / lambda)
        def unique(t):
            t = t.reshape(len(lams300), d, 2 * m + 1)
            return torch.cat([torch.cat([t[:, :, :m], t[:, :, m + 1:]], dim=2).reshape(len(lams300), -1),
                              t[:, :, m].sum(dim=1, keepdim=True)], dim=1)
        ue, uc = unique(sweep["eigen"]["theta"]), unique(sweep["cholesky"]["theta"])
        diff = float(((ue - uc).abs().pow(2).sum(1).sqrt() / uc.abs().pow(2).sum(1).sqrt()).max())
        line["lambda_sweep_300"] = {k: {"ms": v["ms"], "ms_solve": v["ms_solve"]} for k, v in sweep.items()}
        line["lambda_sweep_300"]["lambdas"] = "300 log-spaced in [1e-6, 1e-1]"
        line["lambda_sweep_300"]["max_rel_diff_eigen_vs_cholesky"] = diff
        del sweep
    if W == "additive-8d" and not args.no_graph:
        # the same fit recorded once into a CUDA graph and replayed: one launch per step
        gst = torch.cuda.Stream()
        gst.wait_stream(st)
        out = torch.empty((1, 1, d, 2 * m + 1), dtype=torch.complex128, device=x.device)
        with fk.capture(gst) as graph:
            fk.fk_fit_additive(x, y, m, [lam], 1e-6, "mixed", out=out)
        graph.launch(gst)
        graph.status()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(gst)
        for _ in range(steps):
            graph.launch(gst)
        g1.record(gst)
        graph.status()
        line["graph"] = {"ms_per_step": g0.elapsed_time(g1) / steps, "graph_launches_per_step": 1,
                         "what": "fk_capture_begin/end of one fit, replayed with fk_graph_launch"}
        graph.close()
    return line


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload != "2d-sobolev":
        print(json.dumps(run_row(args, rank, local, n=(args.n if args.n != WL["n"] else None))), flush=True)
        return

    import torch
    import paper_2509_02649_b300 as fk

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    n, d, m, s, lam, eps = args.n, WL["d"], WL["m"], WL["s"], WL["lam"], WL["eps"]
    x_np, y_np = make_inputs(n)
    x_h = torch.from_numpy(x_np).pin_memory()
    y_h = torch.from_numpy(y_np).pin_memory()
    x = x_h.cuda()
    y = y_h.cuda()
    peak = fp32_peak(fk)
    spread = {"auto": fk.FK_SPREAD_AUTO, "atomic": fk.FK_SPREAD_ATOMIC, "binned": fk.FK_SPREAD_BINNED}[args.spread]
    # the first warm-up step times the spreader's tunable shapes and keeps the fastest
    opts = fk.default_opts(spread=spread, autotune=0 if args.no_autotune else 1)
    st = torch.cuda.current_stream()

    def step():
        return fk.fk_fit_sobolev(x, y, m, s, [lam], eps, "mixed", opts=opts, report=True)

    for _ in range(args.warmup):
        theta, rep = step()
    torch.cuda.synchronize()

    reps = []
    launches0 = fk.fk_launch_count()
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            theta, rep = step()
            reps.append(rep)
        e1.record(st)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = fk.fk_launch_count() - launches0
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    value = world * n * args.steps / (ms / 1e3)

    # the same fit recorded once into a CUDA graph (fk_capture_*) and replayed: one graph
    # launch per fit, the spreading kernel timed by the graph's event record nodes
    graph_line = None
    if not args.no_graph:
        gst = torch.cuda.Stream()
        gst.wait_stream(st)
        theta_g = torch.empty_like(theta)
        c0 = fk.fk_launch_count()
        with fk.capture(gst) as graph:
            fk.fk_fit_sobolev(x, y, m, s, [lam], eps, "mixed", opts=opts, out=theta_g)
        kernels_per_replay = fk.fk_launch_count() - c0  # kernels recorded (launched at each replay)
        graph.launch(gst)
        graph.status()
        kms = []
        with ClockSampler(local) as gclk:
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(gst)
            for _ in range(args.steps):
                graph.launch(gst)
                kms.append(graph.kernel_ms())  # waits for this replay's spreading kernel only
            g1.record(gst)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
        graph.status()
        gms = g0.elapsed_time(g1)
        if dist:
            t = torch.tensor([gms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            gms = float(t.item())
        err = float((theta_g - theta).abs().norm() / theta.abs().norm())
        graph_line = {"value": world * n * args.steps / (gms / 1e3), "unit": "points/s",
                      "ms_per_step": gms / args.steps, "ms_kernel": statistics.mean(kms),
                      "gpu_launches": kernels_per_replay * args.steps, "graph_launches_per_step": 1,
                      "theta_rel_diff_vs_direct": err, "clocks": gclk.summary()}
        graph.close()

    # dominant kernel: the register-accumulation spreading kernel, timed by CUDA events
    # recorded on its own stream inside the library (fk_report.ms_kernel)
    ms_kernel = statistics.mean(r["ms_kernel"] for r in reps)
    ms_spread = statistics.mean(r["ms_spread"] for r in reps)
    direct = {"value": value, "ms_per_step": ms_step, "ms_kernel": ms_kernel, "gpu_launches": launches,
              "clocks": clk.summary(), "what": "one fk_fit_sobolev call per fit (stage times from its report)"}
    launch_mode = "direct"
    if graph_line is not None:
        # headline: the graph-replayed fit (same kernels on the same resident inputs, no
        # host work between fits); the direct calls stay in "direct"
        launch_mode = "graph"
        value, ms_step, ms_kernel = graph_line["value"], graph_line["ms_per_step"], graph_line["ms_kernel"]
        launches = graph_line["gpu_launches"]
    w = reps[-1]["kernel_width"]
    C = 2
    f_pt = (w ** d) * (2 * C + (d - 1))
    peaks = measured_peaks()
    peak_tflops = peak["measured"]
    achieved = f_pt * n / (ms_kernel / 1e3) / 1e12
    # DRAM bytes of one k_bin_accumulate launch: ncu capture of this kernel at n = 2e7
    # (dram__bytes_read.sum 241.2 MB + dram__bytes_write.sum 6.5 MB), scaled by points
    # (the reads are the 8-byte partition records and the strengths, the writes the flush)
    traffic = ACC_DRAM_BYTES_PER_POINT * n if (d == 2 and w == 7) else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic,
                "kernel": "k_bin_accumulate (register-accumulation spreading)",
                "flop_per_point": f_pt, "kernel_width": w, "ms_kernel": ms_kernel,
                "peak_basis": peak["basis"], "peak_derived": peak["derived"],
                "frac_of_derived": achieved / peak["derived"], "sm_count": peak["sm_count"],
                "stage": {"ms_spread_all_kernels": ms_spread,
                          "achieved_TFLOPs": f_pt * n / (ms_spread / 1e3) / 1e12,
                          "frac": f_pt * n / (ms_spread / 1e3) / 1e12 / peak_tflops,
                          "ms_fft": statistics.mean(r["ms_fft"] for r in reps),
                          "ms_solve": statistics.mean(r["ms_solve"] for r in reps), "cg_iters": reps[-1]["cg_iters"]},
                "hbm_view": {"bytes_per_point_input": 12, "achieved_GBs": 12 * n / (ms_spread / 1e3) / 1e9,
                             "peak_GBs": peaks.get("hbm_gbs"), "of": "measured"}}
    # the whole fit against the slower of the point bytes over HBM and the spreading
    # arithmetic at the FP32 peak (points/s)
    hbm = peaks.get("hbm_gbs") or 6400.0
    bound_pts = min(hbm * 1e9 / 12.0, peak_tflops * 1e12 / f_pt)
    roofline["fit_view"] = {"bound_points_per_s": bound_pts, "achieved_points_per_s": value / world,
                            "frac": value / world / bound_pts,
                            "basis": "min(measured HBM / 12 B, measured FP32 peak / %d flop) per GPU" % f_pt}

    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WL["workload"], "n": n, "d": d, "m": m, "s": s, "lambda": lam, "eps": eps,
                       "precision": "mixed (fp32 spread/FFT, fp64 assembly/solve)",
                       "l2": "inputs (%.1f GB) larger than L2, no flush" % (12 * n / 1e9), "parallelism": "replicas" if world > 1 else "1 GPU",
                       "launch": ("one CUDA graph per fit (fk_capture_begin/end once, fk_graph_launch per fit)"
                                  if launch_mode == "graph" else "one fk_fit_sobolev call per fit")},
            "gpu_launches": launches, "roofline": roofline,
            "clocks": graph_line["clocks"] if launch_mode == "graph" else clk.summary(),
            "direct": direct if launch_mode == "graph" else None,
            "autotune": fk.fk_autotune_table().strip() or None}

    if rank == 0 and not args.no_e2e:
        # end to end through the public API with host buffers: every step hands the pinned
        # host inputs to fk_accum_add_host, which copies them in chunks of 2^22 points on
        # the accumulator's copy stream and spreads each chunk once it has landed, so the
        # spreading hides under the host link (~54 GB/s); the last chunk's spreading, the
        # transform and the solve (fk_accum_fit_sobolev) follow the copy, and theta is
        # read back.
        theta_h = torch.empty(theta.shape, dtype=theta.dtype).pin_memory()
        y_h2 = y_h.reshape(1, -1)
        acc = fk.Accumulator(2, m, 1, eps, "mixed", opts=opts)

        def e2e_step():
            acc.reset()
            acc.add_host(x_h, y_h2)
            th = acc.fit_sobolev(s, [lam])
            theta_h.copy_(th, non_blocking=True)
            return th

        th_e = e2e_step()
        torch.cuda.synchronize()
        k = max(2, min(args.steps, 5))
        ee0 = torch.cuda.Event(enable_timing=True)
        ee1 = torch.cuda.Event(enable_timing=True)
        ee0.record(st)
        for _ in range(k):
            th_e = e2e_step()
        ee1.record(st)
        torch.cuda.synchronize()
        ems = ee0.elapsed_time(ee1) / k
        err_e = float((th_e - theta).abs().norm() / theta.abs().norm())
        acc.close()
        line["e2e"] = {"value": n / (ems / 1e3), "unit": "points/s", "h2d_bytes_per_step": 12 * n,
                       "d2h_bytes_per_step": int(theta.numel() * 16), "ms_per_step": ems,
                       "what": "pinned host inputs passed to fk_accum_add_host (chunks of 2^22 points "
                               "copied on its copy stream, each spread on arrival), then "
                               "fk_accum_fit_sobolev and theta read back",
                       "theta_rel_diff_vs_resident": err_e}

    if rank == 0 and not args.no_fp64:
        # the plain FP64 GPU path on the same points (fp64 copies) and the mixed result's error against it
        x64 = x.double()
        y64 = y.double()
        fk.fk_fit_sobolev(x64, y64, m, s, [lam], eps, "fp64")
        torch.cuda.synchronize()
        k = 2
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(st)
        for _ in range(k):
            th64 = fk.fk_fit_sobolev(x64, y64, m, s, [lam], eps, "fp64")
        f1.record(st)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1) / k
        err = float(torch.linalg.norm(theta - th64) / torch.linalg.norm(th64))
        # accuracy reference: the FP64 path at eps = 1e-12 (itself gated <= 1e-10 against the
        # oracle at small n); the metric's gate is rel err <= 1e-5 for the mixed path
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(st)
        th_acc = fk.fk_fit_sobolev(x64, y64, m, s, [lam], 1e-12, "fp64")
        a1.record(st)
        torch.cuda.synchronize()
        err_acc = float(torch.linalg.norm(theta - th_acc) / torch.linalg.norm(th_acc))
        line["fp64_path"] = {"value": n / (fms / 1e3), "unit": "points/s", "ms_per_step": fms,
                             "mixed_speedup": (n / (ms_step / 1e3)) / (n / (fms / 1e3)),
                             "theta_rel_err_mixed_vs_fp64": err, "eps": eps,
                             "accuracy_reference": {"eps": 1e-12, "precision": "fp64",
                                                    "ms": a0.elapsed_time(a1),
                                                    "theta_rel_err_mixed": err_acc,
                                                    "theta_rel_err_fp64_eps1e-6": float(
                                                        torch.linalg.norm(th64 - th_acc) / torch.linalg.norm(th_acc)),
                                                    "gate": 1e-5, "pass": err_acc <= 1e-5}}
        del x64, y64

    if rank == 0 and not args.no_cpu_baseline:
        n_o = 50_000
        t_cpu, _ = cpu_oracle_fit(x_np[:, :n_o], y_np[:n_o], m, s, lam)
        line["cpu_baseline"] = {"value": n_o / t_cpu, "unit": "points/s", "cores": host_cores(), "kind": "oracle",
                                "sample": "first %d points of the workload: direct sums + dense solve D=4225" % n_o}
    if rank == 0 and not args.no_rows:
        # the other hot-path rows, each at full size with its own step count, clocks and
        # roofline (the headline's inputs are released first)
        del x, y
        torch.cuda.empty_cache()
        rows = {}
        for wl, k, w0 in (("additive-8d", 5, 2), ("pik-heat", 5, 2), ("sweep-1d", 2, 1)):
            rows[wl] = run_row(args, rank, local, W=wl, steps=k, warmup=w0, peak=peak)
            torch.cuda.empty_cache()
        line["rows"] = rows
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
