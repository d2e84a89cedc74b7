"""Benchmark: Fourier-accelerated Landau gauge fixing of a 64^4 SU(3) configuration on GB300.

Metric: site-iterations/s and time-to-theta < 1e-15 at 64^4, mixed FP32->FP64 vs FP64, and the HBM
roofline of the kernels.

A step is one complete gauge fixing (Algorithm 1 of Cardoso et al., run until theta < 1e-15) of the
64^4 configuration (eps = 0.6, seed 4; links 9.66 GB in double precision), with the mixed-precision
schedule: float links, FFTs and updates with double reductions until theta <= 1e-11, then the double
handover and double precision to theta < 1e-15. The input stays resident in HBM and is never
modified (load -> iterate -> store into a separate output buffer), so every step repeats the same
work. `value` = V * iterations / time (site-iterations per second over whole fixes); `ms_per_step`
is the time to theta < 1e-15. Beside it: the same field fixed in the double path, per-kernel device times
from CUDA events recorded on the working stream during the timed steps, the end-to-end figure through
the C ABI from pinned host buffers (copies included), and the CPU oracle timed on a bounded sample.

Multi-GPU (torchrun): one independent replica per rank (seed 4 + rank); no collective on the data
path; value = all ranks' site-iterations / max over ranks of the time.

--impl reference runs the FP64 CPU oracle on the host cores instead (rank 0 only): each step is one
iteration of Algorithm 1 on the same 64^4 configuration.
"""
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

METRIC = "site-iterations/s & time-to-θ≤1e-15 at 64^4, FP32→FP64 vs FP64; % HBM peak"
UNIT = "site-iterations/s"

# Nominal FP64 rate derived from the unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop
# x 2.07 GHz = 1.259 TFLOP/s (GB300 FP64 is 1.25 TFLOP/s nominal).
FP64_FLOP_PER_CLK = 152 * 2 * 2      # 152 SMs x 2 DFMA per clock x 2 flop
FP32_OPS_PER_CLK = 152 * 128         # 152 SMs x 128 FP32 lanes (one FADD, FMUL or FFMA each per clock)
# DRAM bytes (read + write) per launch of a kernel at 64^4, from one ncu capture of
# dram__bytes_read.sum + dram__bytes_write.sum; valid only for the kernel versions that were captured.
TRAFFIC_64 = {"gauge_update_fused.f32": 4.79e9 + 4.11e9, "update_residual.f32": 9.96e9 + 6.25e9}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


# Flops (multiply and add = 1 each, an FMA = 2) of the SU(3) arithmetic, counted from the source:
# the projection onto SU(3) (two row norms 11 each, two row scalings 6 each, the overlap <r0, r1> 24, its
# removal 24, the row-2 cross product 42; the two reciprocal square roots are not counted), and the
# product g U g^+ kept as rows 0-1 of g U (132) and of (g U) g^+ (144) plus the row-2 cross product (42).
PROJECTION_FLOP = 11 + 6 + 24 + 24 + 11 + 6 + 42
LINK_PRODUCT_FLOP = 132 + 144 + 42


def work_model(kernel, dims):
    """Algorithmic bytes and arithmetic per launch of each kernel (each datum counted once), and the
    precision of the kernel: (bytes, count, prec). es = bytes per complex number. The count is in the units
    of algorithmic(): FP64 flops (FMA = 2), FP32-pipe operations, or, for the FFT passes, the flop
    convention of the paper (5 N log2 N per axis, field and direction)."""
    V = int(np.prod(dims))
    name, prec = kernel.rsplit(".", 1)
    es = 16 if prec == "f64" else 8
    nx, ny, nz, nt = dims
    lg = {k: np.log2(n) for k, n in zip("xyzt", dims)}
    lp = 9 if prec == "f64" else 6  # planes per link: float links keep rows 0-1 (row 2 rebuilt on load)
    table = {
        # 4 links read (the backward neighbours are the same data), 4 packed Delta written
        "delta_theta": ((4 * lp + 4) * es, 190),
        # read + write 4 packed fields; FFT flops 5 N log2 N per field per axis per direction
        "fft_xy_fwd": (8 * es, 4 * 5 * (lg["x"] + lg["y"])),
        "fft_xy_inv": (8 * es, 4 * 5 * (lg["x"] + lg["y"])),
        "fft_x_fwd": (8 * es, 4 * 5 * lg["x"]), "fft_x_inv": (8 * es, 4 * 5 * lg["x"]),
        "fft_y_fwd": (8 * es, 4 * 5 * lg["y"]), "fft_y_inv": (8 * es, 4 * 5 * lg["y"]),
        "fft_z_fwd": (8 * es, 4 * 5 * lg["z"]), "fft_z_inv": (8 * es, 4 * 5 * lg["z"]),
        "fft_zt_filter": (8 * es, 4 * (2 * 5 * (lg["z"] + lg["t"]) + 6)),
        "fft_t_filter": (8 * es, 4 * (2 * 5 * lg["t"] + 6)),
        # packed Delta-tilde read, g written (double path: also a = g - 1 in double-float, 9 x 16 B)
        "gauge_g": ((4 + 9 + (9 if prec == "f64" else 0)) * es, 160),
        # links read and written, g read (neighbours are the same data). Double: the small-step form,
        # which every warp of the double stage takes: per link, rows 0-1 of two 3x3 complex products in
        # double-float, 6 outputs x 3 terms x 4 real products x 2 = 144 multiply-accumulates of 12 FP32
        # operations each (Dot2 step); row 2 by an FP64 cross product (not counted). Float (plain FP32
        # schedule): rows 0-1 of g U (132 flop) and of (g U) g^+ (144), row 2 by a cross product (42).
        "gauge_update": ((4 * lp * 2 + 9) * es, 4 * 144 * 12 if prec == "f64" else 4 * LINK_PRODUCT_FLOP),
        # float stage: links read and written, G read and written (rows 0-1), packed Delta-tilde read (g is
        # rebuilt in registers); the _reunit variant also projects G and the new links onto SU(3) in float
        "gauge_update_fused": ((4 * lp * 2 + 12 + 4) * es, 0),
        "gauge_update_fused_reunit": ((4 * lp * 2 + 12 + 4) * es, 0),
        "gacc_to_double": (6 * 8 + 9 * 16, PROJECTION_FLOP),
        "handover_transform": (36 * 16 * 2 + 9 * 16 + 4 * 6 * 8, 4 * LINK_PRODUCT_FLOP),
        "to_planes": (4 * lp * 16 + 4 * lp * es, 0),  # the float load reads rows 0-1 of each link only
        "from_planes": (4 * lp * es + 36 * 16, 0),
        "set_identity": (6 * 8, 0),
        # residual stage of the mixed schedule: Delta from the residual R (4 x 9 float planes read) plus the
        # base's packed Delta (4 x 16 B) into the float packed field; the update reads the base links (rows
        # 0-1, float), reads and writes R and K = H - 1 (9 float planes) and reads the packed Delta-tilde;
        # at the end H is projected in FP64 (K read, H and a = H - 1 written) and the double links are
        # rebuilt by the double update (the same counts as gauge_update.f64); the base (only when the stage
        # restarts from rebuilt links) is the double links narrowed to float rows 0-1.
        "delta_residual": (4 * 9 * 8 + 4 * 16 + 4 * 8, 0),
        "update_residual": (4 * 6 * 8 + 2 * 4 * 9 * 8 + 2 * 9 * 8 + 4 * 8, 0),
        "residual_gauge": (9 * 8 + 9 * 16 + 9 * 16, PROJECTION_FLOP),
        "residual_rebuild": ((4 * 9 * 2 + 9) * 16, 4 * 144 * 12),
        "residual_base": (4 * 6 * 16 + 4 * 6 * 8, 0),
    }
    b, f = table[name]
    return b * V, f * V, prec


def algorithmic(kernel, dims):
    """Bytes and arithmetic per launch for the roofline: (bytes, count, kind) with kind "fp64" (FP64 flops,
    FMA = 2), "fp32" (FP32-pipe operations: FADD, FMUL, FFMA = 1 each) or None (the kernel is modelled by
    its bytes only; count 0)."""
    b, f, prec = work_model(kernel, dims)
    name = kernel.rsplit(".", 1)[0]
    if prec == "f64":
        # (the handover transform runs in 61-bit fixed point on the integer pipe: bytes only)
        kind = {"gauge_update": "fp32", "residual_rebuild": "fp32", "gacc_to_double": "fp64",
                "residual_gauge": "fp64"}.get(name)
    else:
        kind = None
    return b, (f if kind else 0), kind


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(seed, rank):
    """Each rank fixes its own configuration, a replica: the generator seed is offset by the rank."""
    return seed + rank


def reduce_over_ranks(ms, work, ws, device):
    """Whole-job figures over independent replicas: the slowest rank's time and the summed work
    (site-iterations). The only collective of the bench; none is on the data path."""
    if ws == 1:
        return ms, work
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t[0]), float(w[0])


def run_reference(args, dims, rank, ws):
    """The FP64 CPU oracle on the host cores: each step is one iteration of Algorithm 1 on the 64^4
    configuration (the untimed part loads the configuration and its initial Delta)."""
    if rank != 0:
        return
    import oracle
    import synth
    cores = os.cpu_count()
    U = synth.config(dims, args.seed, args.eps)
    V = int(np.prod(dims))
    for _ in range(args.warmup):
        U, _, _, _, _ = oracle.fix(U, 0.08, 0.0, 1)
    t0 = time.perf_counter()
    U, it, th, F, _ = oracle.fix(U, 0.08, 0.0, args.steps)
    dt = time.perf_counter() - t0
    # oracle.fix also evaluates Delta/theta/F of the input once before its loop (a 1/(K+1) share)
    value = V * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args, dims, args.precision),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d iterations of Algorithm 1 (FP64 CPU oracle) on the %s configuration"
                                       % (args.steps, "x".join(map(str, dims)))},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def schedule_of(args):
    """What the headline schedule does, stage by stage."""
    if args.precision == "fp64":
        return {"stages": "double path: FP64 links and sums (exact fixed-point Delta, double-float filter and "
                          "small-step forms at FP64 rounding level) to theta < 1e-15"}
    if args.precision == "fp32":
        return {"stages": "float links, FFTs and updates with FP64 reductions throughout"}
    return {"float_stage": "float links (rows 0-1), FFTs and updates; theta and F sums in FP64",
            "handover": "theta <= %g (or when a chunk of float iterations stops lowering theta)" % args.theta_switch,
            "reprojection": "float links and accumulated transformation G projected onto SU(3) in float every 16 "
                            "float iterations",
            "handover_links": "U = G U0 G^+(x+mu) from the saved FP64 input, two directions per site in FP64 and two in "
                              "61-bit fixed point (both exact to FP64 rounding)",
            "final_approach": "float iterations on the residual R of U = U_h + R, then the double links rebuilt "
                              "exactly by the double update; theta < 1e-15 checked in FP64"}


def config_of(args, dims, path):
    return {"workload": "%s SU(3) lattice, U=h exp(i eps A) h^+(x+mu), eps=%g, seed %d; alpha=0.08, "
                        "theta<1e-15; %s" % ("^".join(["64", "4"]) if dims == (64, 64, 64, 64) else "x".join(map(str, dims)),
                                             args.eps, args.seed, path),
            "lattice": list(dims), "precision": args.precision, "theta_switch": args.theta_switch,
            "schedule": schedule_of(args),
            "step": "one complete gauge fixing (Algorithm 1 until theta < 1e-15)",
            "l2": ("no flush: links %.3g GB per step >> 129 MB L2" % (int(np.prod(dims)) * 576 / 1e9)
                   if np.prod(dims) >= 2 ** 20 else "small lattice"),
            "parallelism": "replicas"}


def load_golden(dims, seed, eps):
    """The FP64 oracle's complete fix of this configuration, stored in tests/golden/ by a script that calls
    only the oracle (None when no stored fix matches)."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_fix_%s_s%d.json" % ("x".join(map(str, dims)), seed))
    if not os.path.exists(path):
        return None
    g = json.load(open(path))
    if tuple(g["dims"]) != tuple(dims) or g["seed"] != seed or abs(g["eps"] - eps) > 1e-12:
        return None
    return g


def error_vs_oracle(res, golden):
    """Errors of one schedule's result against the oracle's fix of the same configuration: F (both are the
    same maximum, relative), the plaquette (gauge invariant: the fixed links against the input), theta (both
    final values are below 1e-15; reported side by side), the iteration count and, for the double path, the
    largest per-iteration deviation of theta and F along the whole trajectory."""
    if golden is None:
        return None
    out = {"reference": "FP64 CPU oracle, complete fix of the same configuration (%d iterations)" % golden["iters"],
           "F_rel_err": abs(res["F"] - golden["F"]) / abs(golden["F"]),
           "plaquette_err_vs_input": abs(res["plaquette"] - golden["plaquette_in"]),
           "plaquette_err_vs_oracle_output": abs(res["plaquette"] - golden["plaquette_out"]),
           "theta": res["theta"], "theta_oracle": golden["theta"],
           "iters": res["iters"], "iters_oracle": golden["iters"]}
    if "history" in res:
        h, ho = np.asarray(res["history"]), np.asarray(golden["history"])
        n = min(len(h), len(ho))
        out["history_theta_max_rel_err"] = float(np.max(np.abs(h[:n, 0] - ho[:n, 0]) / ho[:n, 0]))
        out["history_F_max_rel_err"] = float(np.max(np.abs(h[:n, 1] - ho[:n, 1]) / np.abs(ho[:n, 1])))
    return out


def spec_lattice(lgf, dims):
    """A context whose float stage reprojects in double and which runs double iterations after the handover
    (the switches are read when the context is created)."""
    saved = {k: os.environ.get(k) for k in ("LGF_REUNIT_FP64", "LGF_RESIDUAL")}
    os.environ["LGF_REUNIT_FP64"], os.environ["LGF_RESIDUAL"] = "1", "0"
    try:
        return lgf.Lattice(dims)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def kernel_table(ktimes, dims, hbm, alu_peak):
    """Per kernel: launches, time, share, and achieved algorithmic GB/s (and ALU rate) against the peaks."""
    kernels = {}
    total_ms = sum(v[1] for v in ktimes.values()) or 1.0
    for name, (n, kms) in ktimes.items():
        b, f, kind = algorithmic(name, dims)
        per = kms / max(n, 1) / 1e3
        gbs = b / per / 1e9 if per > 0 else 0.0
        d = {"launches": n, "ms_total": round(kms, 3), "share": round(kms / total_ms, 4),
             "ms_per_launch": round(kms / max(n, 1), 4), "GB_s": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}
        if kind and per > 0:
            d["alu_kind"] = kind
            d["alu_frac"] = round(f / per / alu_peak[kind][0], 4)
        kernels[name] = d
    return kernels


def cpu_baseline(dims, args, V_gpu, golden=None, gpu_iters=None):
    """The oracle as it stands on the host cores, on a bounded sample: one iteration of Algorithm 1 on
    the same configuration (falls back to a 32^4 configuration when host memory is short). The time to
    theta < 1e-15 is extrapolated: the per-iteration time times the oracle's own iteration count on this
    configuration (stored by the oracle's complete fix), or else the GPU's."""
    import oracle
    import synth
    need = int(np.prod(dims)) * 4 * 144 * 3.2
    avail = 0
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable"):
                avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    cdims = dims if avail > need else (32, 32, 32, 32)
    U = synth.config(cdims, args.seed, args.eps)
    Vc = int(np.prod(cdims))
    t0 = time.perf_counter()
    oracle.fix(U, 0.08, 0.0, 1)
    dt = time.perf_counter() - t0
    out = {"value": Vc / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": "one iteration of Algorithm 1 (plus the initial Delta/theta/F) on the %s configuration, "
                     "%.1f s" % ("x".join(map(str, cdims)), dt)}
    n_it = golden["iters"] if golden else gpu_iters
    if n_it:
        out["time_to_theta_extrapolated_s"] = dt * (V_gpu / Vc) * n_it
        out["time_to_theta_note"] = ("extrapolated: per-iteration time x %d iterations (%s)%s"
                                     % (n_it, "the oracle's own count on this configuration" if golden
                                        else "the GPU's count", "" if cdims == dims else
                                        " x the volume ratio %d/%d" % (V_gpu, Vc)))
    return out


def _timed(torch, fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def run_batch(args):
    """The batched ensemble: 48 configurations (16 each of 16^4, 24^3x48, 32^3x64), eps_i ~ U[0.4, 0.7]
    (seed 99), configuration i from seed 100 + i; fixed together in FP64 and in the mixed schedule
    (grouped launches, CUDA-graph replay, autotuned FFT passes). Links stay on the device. Each schedule:
    W untimed fixes of the whole ensemble (the first also tunes the FFT passes on a cold cache), then K
    timed fixes; the copy of the inputs into the working buffers precedes each fix, outside its timing."""
    import torch
    import paper_1210_8018_gb300 as lgf
    import synth
    shapes = [(16, 16, 16, 16)] * 16 + [(24, 24, 24, 48)] * 16 + [(32, 32, 32, 64)] * 16
    rng = np.random.default_rng(99)
    eps_list = rng.uniform(0.4, 0.7, len(shapes))
    inputs = []
    for i, (d, e) in enumerate(zip(shapes, eps_list)):
        inputs.append(torch.from_numpy(synth.config(d, 100 + i, float(e))).cuda())
    work = [torch.empty_like(u) for u in inputs]
    sites = sum(int(np.prod(d)) for d in shapes)
    out = {"metric": "site-iterations/s, batched ensemble of uneven lattices", "unit": UNIT,
           "config": {"workload": "16 x 16^4 + 16 x 24^3x48 + 16 x 32^3x64, eps ~ U[0.4,0.7], alpha=0.08, theta<1e-15",
                      "sites": sites, "l2": "no flush: 26 GB of links per fix >> 129 MB L2"},
           "data": "synthetic", "steps": args.steps, "warmup": args.warmup}
    schedules = [p for p in args.batch_schedules.split(",") if p]
    with lgf.Batch(shapes) as b:
        for prec in schedules:
            def run():
                for w, u in zip(work, inputs):
                    w.copy_(u)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = b.fix(work, 0.08, 1e-15, prec)
                torch.cuda.synchronize()
                return res, time.perf_counter() - t0
            for _ in range(args.warmup):
                run()
            times = []
            for _ in range(args.steps):
                res, dt = run()
                times.append(dt)
            dt = statistics.median(times)
            its = [r["iters"] for r in res]
            siters = sum(int(np.prod(d)) * r["iters"] for d, r in zip(shapes, res))
            out[prec] = {"time_to_theta_s": dt, "samples_s": [round(t, 4) for t in times],
                         "site_iterations_per_s": siters / dt,
                         "converged": sum(r["status"] == 0 for r in res), "iters_min": min(its),
                         "iters_max": max(its), "describe": b.describe()}
    # the same 48 configurations fixed one after another, each by a single-configuration context (one
    # context per shape, reused): what grouping and graph replay save, or cost, against separate fixes
    for prec in ([] if args.no_sequential else schedules):
        lats = {d: lgf.Lattice(d) for d in sorted(set(shapes))}
        for d, lat in lats.items():
            lat.set_stream(torch.cuda.current_stream())
        for w, u in zip(work, inputs):
            w.copy_(u)
        for lat, w in ((lats[d], w) for d, w in zip(shapes, work)):  # warm-up: one fix per context
            lat.fix(w, 0.08, 1e-15, prec)
        for w, u in zip(work, inputs):
            w.copy_(u)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        siters = 0
        for d, w in zip(shapes, work):
            r = lats[d].fix(w, 0.08, 1e-15, prec)
            siters += int(np.prod(d)) * r["iters"]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        for lat in lats.values():
            lat.close()
        out[prec]["sequential_single_contexts"] = {"time_to_theta_s": dt, "site_iterations_per_s": siters / dt}
    out["value"] = out[schedules[0]]["site_iterations_per_s"]
    return out


def run_scan(args):
    """The paper's tuning sweep over 32^3 x n (n = 8, 16, 32, 64): site-iterations/s of complete fixes in FP64
    and in the mixed schedule (W untimed, then K timed fixes, CUDA events on the working stream), with the
    per-kernel roofline of each."""
    import torch
    import paper_1210_8018_gb300 as lgf
    import synth
    hbm, sm_max, which = peaks()
    clk_hz = sm_max * 1e6
    alu_peak = {"fp64": (FP64_FLOP_PER_CLK * clk_hz, "TFLOP/s", ""), "fp32": (FP32_OPS_PER_CLK * clk_hz, "Tops/s", "")}
    rows = []
    for n in (8, 16, 32, 64):
        dims = (32, 32, 32, n)
        V = int(np.prod(dims))
        U = torch.from_numpy(synth.config(dims, 2, args.eps)).cuda()
        W = torch.empty_like(U)
        row = {"lattice": "32^3x%d" % n, "sites": V}
        with lgf.Lattice(dims) as lat:
            stream = torch.cuda.current_stream()
            lat.set_stream(stream)
            for prec in ("fp64", "mixed"):
                def run():
                    lat.load(U, prec)
                    r = lat.iterate(1 << 30, 0.08, 1e-15)
                    lat.store(W)
                    return r
                for _ in range(args.warmup):
                    run()
                lat.enable_timing(True)
                lat.kernel_times()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                its = 0
                for _ in range(args.steps):
                    r = run()
                    its += r["iters"]
                e1.record(stream)
                torch.cuda.synchronize()
                kt = lat.kernel_times()
                lat.enable_timing(False)
                dt = e0.elapsed_time(e1) / 1e3
                kern = kernel_table(kt, dims, hbm, alu_peak)
                dom = max(kern, key=lambda k: kern[k]["ms_total"])
                row[prec] = {"iters": r["iters"], "time_s": dt / args.steps, "site_iterations_per_s": V * its / dt,
                             "dominant_kernel": dom, "dominant_hbm_frac": kern[dom]["hbm_frac"],
                             "kernels": {k: {"share": v["share"], "hbm_frac": v["hbm_frac"]} for k, v in kern.items()}}
        rows.append(row)
    return {"metric": "site-iterations/s over 32^3 x n", "unit": UNIT, "scan": rows, "steps": args.steps,
            "warmup": args.warmup, "value": rows[-1]["mixed"]["site_iterations_per_s"], "data": "synthetic",
            "peak_source": "%s HBM %g GB/s" % (which, hbm)}


def run_autograd(args):
    """F_U[exp(i omega)] on 24^4 (eps = 0.5, seed 5; omega ~ N(0, 0.05^2) per generator, seed 6): forward
    and backward kernel times, then torch optimisers over omega until theta <= 1e-10: Adam on the
    Fourier-preconditioned gradient (re-based every 5 steps, moments carried over), plain Adam (bounded
    number of steps: it slows down critically), and SGD on the preconditioned gradient (Algorithm 1's step)."""
    import torch
    import paper_1210_8018_gb300 as lgf
    import synth
    dims = (24, 24, 24, 24)
    V = int(np.prod(dims))
    U = torch.from_numpy(synth.config(dims, 5, 0.5)).cuda()
    om = torch.from_numpy(synth.normals(6, 0, V * 8, 0.05).reshape(V, 8)).cuda()
    grad = torch.empty_like(om)
    out = {"metric": "F_U[exp(i omega)] forward/backward and Adam to theta<=1e-10", "config":
           {"workload": "24^4, eps=0.5, omega~N(0,0.05^2)"}, "data": "synthetic"}
    with lgf.Lattice(dims) as lat:
        for _ in range(3):
            lat.functional(U, om)
            lat.functional_grad(U, om, grad)
        n = 20
        _, tf = _timed(torch, lambda: [lat.functional(U, om) for _ in range(n)])
        _, tb = _timed(torch, lambda: [lat.functional_grad(U, om, grad) for _ in range(n)])
    out["forward_ms"] = 1e3 * tf / n
    out["backward_ms"] = 1e3 * tb / n
    runs = (("adam_fourier_preconditioned",
             dict(optimizer="adam", lr=0.05, precondition=True, rebase_every=5, check_every=5, patience=2,
                  max_steps=5000)),
            ("adam_plain", dict(optimizer="adam", lr=3e-2, check_every=20, max_steps=3000)),
            ("sgd_fourier_preconditioned",
             dict(optimizer="sgd", precondition=True, lr=0.08, rebase_every=1, check_every=1, max_steps=500)))
    for name, kw in runs:
        Uc = U.clone()
        res, dt = _timed(torch, lambda: lgf.adam_fix(Uc, target=1e-10, omega0=om, **kw))
        out[name] = {k: v for k, v in res.items() if k != "history"}
        out[name]["time_s"] = dt
        out[name]["reached_target"] = res["theta"] <= 1e-10
        out[name]["theta_trace"] = [(h[0], h[1]) for h in res["history"][::max(1, len(res["history"]) // 20)]]
    out["value"] = out["adam_fourier_preconditioned"]["theta"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lgf", choices=["lgf", "reference"])
    ap.add_argument("--lattice", type=int, nargs=4, default=[64, 64, 64, 64])
    ap.add_argument("--eps", type=float, default=0.6)
    ap.add_argument("--seed", type=int, default=4)
    # (the float-only schedule stops at the float floor, far above theta < 1e-15: not a bench schedule)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--theta-switch", type=float, default=1e-11)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 comparison fix")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batch", action="store_true",
                    help="the batched ensemble: 16 each of 16^4, 24^3x48, 32^3x64, eps ~ U[0.4, 0.7]")
    ap.add_argument("--batch-schedules", default="mixed,fp64",
                    help="schedules of the ensemble leg, comma-separated (mixed, fp64, fp32)")
    ap.add_argument("--no-sequential", action="store_true",
                    help="ensemble leg: skip fixing the configurations one by one for comparison")
    ap.add_argument("--scan", action="store_true", help="site-iterations/s over 32^3 x n, n = 8..64")
    ap.add_argument("--autograd", action="store_true",
                    help="F_U[exp(i omega)] forward/backward at 24^4 and Adam over omega to theta <= 1e-10")
    ap.add_argument("--fft32-final", action="store_true",
                    help="also time the mixed variant whose double stage runs the Fourier filter in float")
    args = ap.parse_args()
    assert args.warmup >= 3 or args.impl == "reference", "at least 3 warm-up steps"
    dims = tuple(args.lattice)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, dims, rank, ws)
        return

    import torch
    import synth
    torch.cuda.set_device(local)
    if args.batch or args.scan or args.autograd:
        if rank == 0:
            with ClockSampler(local) as clk:
                out = run_batch(args) if args.batch else run_scan(args) if args.scan else run_autograd(args)
            out["clocks"] = clk.summary()
            print(json.dumps(out), flush=True)
        return
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_1210_8018_gb300 as lgf

    V = int(np.prod(dims))
    seed = replica_seed(args.seed, rank)
    host = torch.empty(synth.links_shape(dims), dtype=torch.complex128).pin_memory()
    synth.config(dims, seed, args.eps, out=host.numpy())
    U_in = host.to("cuda", non_blocking=False)
    U_out = torch.empty_like(U_in)
    stream = torch.cuda.current_stream()
    golden = load_golden(dims, seed, args.eps)

    lat = lgf.Lattice(dims)
    lat.set_stream(stream)
    # (name, context, precision, iterate() keywords): the headline schedule first
    schedules = [(args.precision, lat, args.precision, dict(theta_switch=args.theta_switch))]
    lat_s = None
    if args.precision == "mixed" and not args.no_fp64:
        schedules.append(("fp64", lat, "fp64", {}))
        lat_s = spec_lattice(lgf, dims)
        lat_s.set_stream(stream)
        schedules.append(("mixed_as_specified", lat_s, "mixed", dict(theta_switch=1e-8)))
    if args.fft32_final and args.precision == "mixed":
        schedules.append(("mixed_fft32_final", lat, "mixed", dict(theta_switch=args.theta_switch, fft32_final=True)))

    def one_fix(ctx, prec, kw):
        ctx.load(U_in, prec)
        r = ctx.iterate(1 << 30, 0.08, 1e-15, **kw)
        ctx.store(U_out)
        return r

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # Every schedule: W untimed warm-up fixes, then K fixes timed with CUDA events on the working stream (one
    # event pair per fix) inside the clock sampler; then, untimed, the output's plaquette and (double path)
    # the per-iteration history against the oracle's stored fix of the same configuration.
    results = {}
    with ClockSampler(local) as clk:
        for name, ctx, prec, kw in schedules:
            for _ in range(args.warmup):
                one_fix(ctx, prec, kw)
            ctx.enable_timing(True)
            ctx.kernel_times()  # reset counters
            barrier()
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
            iters = []
            evs[0].record(stream)
            for i in range(args.steps):
                r = one_fix(ctx, prec, kw)
                iters.append(r["iters"])
                evs[i + 1].record(stream)
                if not r["converged"]:
                    raise SystemExit("%s fix did not converge: %r" % (name, r))
            barrier()
            ktimes = ctx.kernel_times()
            ctx.enable_timing(False)
            ms = evs[0].elapsed_time(evs[-1])
            per = [evs[i].elapsed_time(evs[i + 1]) / 1e3 for i in range(args.steps)]
            plaq = ctx.measure(U_out)["plaquette"]
            res = {"time_to_theta_s": ms / args.steps / 1e3, "time_to_theta_samples_s": [round(t, 5) for t in per],
                   "iters": iters[-1], "site_iterations_per_s": V * sum(iters) / (ms / 1e3),
                   "theta": r["theta"], "F": r["F"], "plaquette": plaq, "ms_total": ms, "iters_all": iters,
                   "ktimes": ktimes}
            if prec == "fp64":
                ctx.load(U_in, prec)
                rh = ctx.iterate(1 << 30, 0.08, 1e-15, history_len=4096, **kw)
                res["history"] = rh["history"][: rh["iters"] + 1]
            res["error_vs_oracle"] = error_vs_oracle(res, golden)
            results[name] = res
    clocks = clk.summary()

    head = results[args.precision]
    t_max, site_iters = reduce_over_ranks(head["ms_total"], V * sum(head["iters_all"]), ws, "cuda")
    value = site_iters / (t_max / 1e3)

    # roofline of every kernel of the headline schedule; the dominant kernel (largest share) is reported
    hbm, sm_max, which = peaks()
    clk_hz = (clocks["sm_mhz"] or sm_max) * 1e6
    alu_peak = {"fp64": (FP64_FLOP_PER_CLK * clk_hz, "TFLOP/s", "152 SMs x 4 FP64 flop/clk"),
                "fp32": (FP32_OPS_PER_CLK * clk_hz, "Tops/s (FP32-pipe operations)", "152 SMs x 128 FP32 ops/clk")}
    kernels = kernel_table(head["ktimes"], dims, hbm, alu_peak)
    dom = max(kernels, key=lambda k: kernels[k]["ms_total"])
    dk = kernels[dom]
    b, f, kind = algorithmic(dom, dims)
    per = dk["ms_per_launch"] / 1e3
    traffic = TRAFFIC_64.get(dom) if tuple(dims) == (64, 64, 64, 64) else None
    if kind and dk["alu_frac"] > dk["hbm_frac"]:
        pk, unit, src = alu_peak[kind]
        roof = {"bound": "alu", "achieved": round(f / per / 1e12, 4), "peak": round(pk / 1e12, 4),
                "unit": unit, "frac": round(f / per / pk, 4), "traffic": traffic,
                "kernel": dom, "peak_source": "derived: %s x median SM clock under load" % src}
    else:
        roof = {"bound": "hbm", "achieved": round(b / per / 1e9, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(b / per / 1e9 / hbm, 4), "traffic": traffic, "kernel": dom,
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % which}

    # end to end through the C ABI from pinned host buffers (H2D + fix + D2H inside the timed region):
    # one untimed call, then five timed calls; the median is reported
    e2e = None
    if not args.no_e2e:
        work = torch.empty_like(host).pin_memory()
        samples = []
        for rep in range(6):
            work.copy_(host)
            barrier()
            t0 = time.perf_counter()
            r = lat.fix(work.numpy(), 0.08, 1e-15, args.precision, theta_switch=args.theta_switch)
            dt = time.perf_counter() - t0
            if rep > 0:
                samples.append((dt, r["iters"]))
        dt, it = sorted(samples)[len(samples) // 2]
        dt_max, work_all = reduce_over_ranks(dt, V * it, ws, "cuda")
        nbytes = 4 * V * 144 * ws  # every rank copies its own links in and out
        e2e = {"value": work_all / dt_max, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "time_to_theta_s": dt_max, "samples_s": [round(d, 4) for d, _ in samples],
               "step": "one lgf_fix call on pinned host links (median of 5 timed calls after 1 untimed)"}

    if rank == 0:
        gpu_launches = sum(v[0] for v in head["ktimes"].values())
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"mixed": "f32+f64", "fp64": "f64", "fp32": "f32"}[args.precision],
                "data": "synthetic", "config": config_of(args, dims, args.precision),
                "iters_per_step": head["iters"], "time_to_theta_s": {}, "theta": head["theta"], "F": head["F"],
                "roofline": roof, "gpu_launches": gpu_launches, "clocks": clocks, "e2e": e2e, "kernels": kernels}
        notes = {"mixed_as_specified": "theta_switch 1e-8, float-stage reprojection in double, double iterations "
                                       "after the handover",
                 "mixed_fft32_final": "double stage with the Fourier filter in float; links, Delta, g, update and "
                                      "sums in double"}
        for name, res in results.items():
            line["time_to_theta_s"][name] = res["time_to_theta_s"]
            out = {k: res[k] for k in ("time_to_theta_s", "time_to_theta_samples_s", "iters", "site_iterations_per_s",
                                       "theta", "F", "plaquette", "error_vs_oracle")}
            if name != args.precision:
                out["kernels_ms"] = {k: round(v[1], 3) for k, v in
                                     sorted(res["ktimes"].items(), key=lambda kv: -kv[1][1])}
            if name in notes:
                out["note"] = notes[name]
            line[name] = out
        line["error_vs_oracle"] = head["error_vs_oracle"]
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(dims, args, V, golden, head["iters"])
        print(json.dumps(line), flush=True)
    lat.close()
    if lat_s is not None:
        lat_s.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
