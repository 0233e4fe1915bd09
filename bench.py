#!/usr/bin/env python3
"""Throughput of the Clenshaw-Curtis spherical-harmonic transform on GB300.

One step = one transform pair (synthesis then analysis) of every
field-level of the workload (default T639: N=639, J=1281, I=2560, 256
field-levels) with inputs resident in HBM.  ``value`` is field-level
transform pairs per second over all ranks.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Multi-GPU: one process per GPU (torchrun); every rank transforms its own
batch of field-levels (independent columns, no collective on the data
path), timing is the max over ranks ("weak" scaling).  ``--impl reference``
times the CPU oracle on the host cores instead (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "T639 transform pairs/s per field-level"
UNIT = "field-level transform pairs/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="T639",
                    help="T31, T159, T319, T639 (one JSON line in the bench contract), "
                         "or ensemble / ladder (the grouped ensemble and the nested "
                         "restriction ladder, timed with CUDA events)")
    ap.add_argument("--grid", default="cc", choices=["cc", "fejer1", "reduced"],
                    help="latitude grid: Clenshaw-Curtis, the reduced Clenshaw-Curtis "
                         "grid of the 1e-16 reduction rule (Sec. 6), or the shifted grid of "
                         "Fejer's first rule")
    ap.add_argument("--reduced-rule", default="fast", choices=["fast", "smooth"],
                    help="longitude counts of --grid reduced: lengths with compile-time "
                         "FFT kernels (fast) or any 2-3-5-smooth count (smooth)")
    ap.add_argument("--precision", default="auto",
                    help="auto (headline path), fp64, bf16x3, ...")
    ap.add_argument("--fields", type=int, default=0,
                    help="field-levels per GPU (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--reduced", action="store_true",
                    help="the reduced transform of Sec. 4.1 (|P~| < 1e-16 "
                         "neglected per tile)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the plan's default launch shapes")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the FP64 comparison path")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def dist_init(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend=backend)
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def job_throughput(world, fields_per_rank, steps, ms):
    """Whole-job field-level pairs per second: every rank transforms its own
    fields_per_rank field-levels per step (replicas, weak scaling), and the
    job's time is the slowest rank's."""
    return world * fields_per_rank * steps / (ms / 1000.0)


def max_over_ranks(dist, value, device):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# algorithmic work per launch
# ---------------------------------------------------------------------------
def legendre_flops(w, F):
    """Folded contraction: 2 flops per (coefficient, northern node, real column)."""
    ncoef = (w.N + 1) * (w.N + 2) // 2
    Jh = (w.J + 1) // 2
    return 2.0 * ncoef * Jh * 2 * F


def fft_bytes(w, F, real_bytes, npts=None):
    """Grid read (or written) once + Fourier workspace written (or read) once;
    npts: grid points per field (default J I; fewer on a reduced grid)."""
    Jh = (w.J + 1) // 2
    npts = w.J * w.I if npts is None else npts
    return F * npts * real_bytes + (w.N + 1) * 2 * Jh * F * 2 * real_bytes


# DRAM traffic per launch of the kernels that dominate a step, from ncu
# captures (dram__bytes_read.sum + dram__bytes_write.sum) of the same kernel
# code at the T639 shape with 64 field-levels (the same per-CTA work as the
# 256-field workload), scaled by the field count.  Writes still held in L2
# when a launch ends are not counted by the capture.  Keyed by (stage, path,
# workload, field-levels); an entry is removed whenever its kernel changes
# and re-added from a new capture.
_FFT_INV_T639x64 = (419.860 + 786.732) * 1e6   # bytes, fft_inverse<float, 1280>
MEASURED_TRAFFIC = {}
for _p in ("bf16x3", "bf16x2", "fp16x3", "fp16x2"):   # the same FP32 inverse FFT
    MEASURED_TRAFFIC[("fft_inverse", _p, "T639", 256)] = _FFT_INV_T639x64 * 256 / 64



def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
            "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample(w, mstep):
    """One field-level pair (synthesis then analysis) restricted to the zonal
    wavenumbers m = 0, mstep, 2 mstep, ...; returns (seconds, fraction of the
    full pair's Legendre work this sample covers)."""
    import oracle as O
    from paper_1711_11296_gb300 import workloads as W
    a = W.workload_spectrum(w, F=1)
    ms = list(range(0, w.N + 1, mstep))
    ncoef = (w.N + 1) * (w.N + 2) // 2
    frac = sum(w.N - m + 1 for m in ms) / ncoef
    spec = np.zeros_like(a)
    for m in ms:
        r0 = O.coef_offset(w.N, m)
        spec[r0:r0 + w.N - m + 1] = a[r0:r0 + w.N - m + 1]
    t0 = time.perf_counter()
    X = np.zeros((1, w.J, len(ms)), dtype=np.complex128)
    for k, m in enumerate(ms):
        r0 = O.coef_offset(w.N, m)
        X[:, :, k] = O.legendre_inverse_m(spec[r0:r0 + w.N - m + 1],
                                          O.pnm_cc(w.N, w.J, m, m))
    grid = O.dft_inverse(X, w.I, ms=ms)
    O.analysis(grid, w.N, ms=ms)
    return time.perf_counter() - t0, frac


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_baseline(w, mstep=4):
    sec, frac = oracle_sample(w, mstep)
    return {"value": frac / sec, "unit": UNIT, "cores": host_cores(),
            "kind": "oracle",
            "sample": ("1 field-level pair of %s, zonal wavenumbers m = 0 mod %d "
                       "(%.1f%% of the Legendre work), %.1f s, binary128 P table "
                       "build included; plain CPU oracle (direct DFT + direct "
                       "Legendre sums), not an optimised CPU SHT"
                       % (w.name, mstep, 100 * frac, sec))}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1711_11296_gb300 import workloads as W
    w = W.WORKLOADS[args.workload]
    mstep = 16
    for _ in range(args.warmup):
        oracle_sample(w, mstep)
    tot, frac = 0.0, 0.0
    for _ in range(args.steps):
        s, frac = oracle_sample(w, mstep)
        tot += s
    value = frac * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "J": w.J, "I": w.I,
                   "field_levels": 1, "sample": "m = 0 mod %d" % mstep},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(),
                         "kind": "oracle",
                         "sample": "each step: 1 field-level pair, zonal "
                                   "wavenumbers m = 0 mod %d (%.1f%% of the "
                                   "Legendre work)" % (mstep, 100 * frac)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
def split_gemm_bytes(w, F, prec, inverse):
    """Algorithmic HBM bytes of one split Legendre launch: the FP32 operand
    read once, the 16-bit term planes of the P table read once (rows padded
    to 8, K to 16), the FP32 result written once."""
    terms = 2 if prec.endswith("x2") else 3
    Jh = (w.J + 1) // 2
    C = 2 * F
    ncoef = (w.N + 1) * (w.N + 2) // 2
    work = (w.N + 1) * 2 * Jh * C * 4
    spec = ncoef * C * 4
    tab = 0
    for m in range(w.N + 1):
        for q in range(2):
            d = w.N - m - q
            R = d // 2 + 1 if d >= 0 else 0
            if inverse:
                tab += ((Jh - 1 + 7) // 8 * 8) * ((R + 15) // 16 * 16) * 2
            elif R:
                tab += ((R + 7) // 8 * 8) * ((Jh + 15) // 16 * 16) * 2
    tab *= terms
    return (spec + tab + work)


def roofline_for(name, tot_ms, n, w, F, prec, pk, pk_src, npts=None, grid="cc"):
    per_launch_s = tot_ms / n / 1000.0
    real_bytes = 8 if prec == "fp64" else 4
    if name.startswith("legendre") and prec == "fp64":
        fl = legendre_flops(w, F)
        roof = {"kernel": name + "_fp64", "bound": "alu",
                "achieved": fl / per_launch_s / 1e12, "peak": 1.25,
                "unit": "TFLOP/s", "traffic": None,
                "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (no measured "
                               "FP64 peak in MEASURED_PEAKS.json)"}
    elif name.startswith("legendre"):
        # tensor-core products per split: x_a y_b with a + b < terms, less
        # x_2 y_2 for FP16 (weight 2^-22)
        products = {"bf16x2": 3, "fp16x2": 3, "bf16x3": 6, "fp16x3": 5}[prec]
        fl = legendre_flops(w, F) * products
        by = split_gemm_bytes(w, F, prec, name.endswith("inverse"))
        t_frac = fl / per_launch_s / 1e12 / pk["bf16_tflops_sustained"]
        h_frac = by / per_launch_s / 1e9 / pk["hbm_gbs"]
        if h_frac >= t_frac:
            roof = {"kernel": name + "_" + prec, "bound": "hbm",
                    "achieved": by / per_launch_s / 1e9, "peak": pk["hbm_gbs"],
                    "unit": "GB/s", "traffic": None,
                    "peak_source": "%s hbm_gbs" % pk_src,
                    "tensor_frac": t_frac}
        else:
            roof = {"kernel": name + "_" + prec, "bound": "tensor",
                    "achieved": fl / per_launch_s / 1e12,
                    "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                    "traffic": None,
                    "peak_source": "%s bf16_tflops_sustained" % pk_src,
                    "hbm_frac": h_frac}
    else:
        b = fft_bytes(w, F, real_bytes, npts)
        if prec == "fp64":
            roof = {"kernel": name + "_f64", "bound": "alu",
                    "achieved": b / per_launch_s / 1e9, "peak": None,
                    "unit": "GB/s", "traffic": None,
                    "peak_source": "FP64 pipe bound; HBM figure for context"}
        else:
            roof = {"kernel": name + "_f32", "bound": "hbm",
                    "achieved": b / per_launch_s / 1e9, "peak": pk["hbm_gbs"],
                    "unit": "GB/s", "traffic": None,
                    "peak_source": "%s hbm_gbs" % pk_src}
    if roof["peak"]:
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof["ms_per_launch"] = 1000 * per_launch_s
    t = MEASURED_TRAFFIC.get((name, prec, w.name, F)) if grid != "reduced" else None
    if t is not None:
        roof["traffic"] = t
        roof["traffic_note"] = ("ncu DRAM bytes of the T639 x 64 capture scaled by the "
                                "field count; writes still in L2 at the end of a launch "
                                "are not counted")
    return roof


def run_path(args, w, F, prec, device, dist, local, rank, world, e2e_wanted):
    import torch
    from paper_1711_11296_gb300 import sht, workloads as W
    if args.grid == "reduced":
        # longitudes per latitude by the reduction rule, from an FP64 plan's
        # P~ table (plan setup, untimed)
        sizes = sht.Plan(w.N, w.J, w.I, 1, "fp64",
                         device=device).reduced_grid_sizes(args.reduced_rule)
        plan = sht.Plan(w.N, w.J, w.I, F, prec, device=device, grid="reduced",
                        lat_points=sizes)
    else:
        plan = sht.Plan(w.N, w.J, w.I, F, prec, device=device, grid=args.grid)
    if args.reduced:
        plan.set_reduced(True)
    # launch shapes picked by the library's autotuner (plan setup, untimed)
    tuning = plan.tuning if args.no_autotune else plan.autotune(reps=2)
    a = W.workload_spectrum(w, F=F, field0=rank * F)
    spec_in = torch.from_numpy(a).to(device=device, dtype=plan.complex_dtype)
    grid = plan.empty_grid()
    spec_out = plan.empty_spec()

    def step():
        plan.inverse(spec_in, out=grid)
        plan.forward(grid, out=spec_out)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    barrier(dist, local)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(device)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    plan.profile(True)
    sampler.start()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    plan.profile(False)
    prof3 = plan.profile_read(kernels=True)
    prof = {k: (v[0], v[1]) for k, v in prof3.items()}
    plan.status()
    # NaN/Inf guard: a step that produced non-finite output is not a result
    if not bool(torch.isfinite(torch.view_as_real(spec_out)).all()):
        raise RuntimeError("the transform pair produced non-finite values")
    ms_local = ev0.elapsed_time(ev1)
    barrier(dist, local)
    ms = max_over_ranks(dist, ms_local, device)
    res = {"ms": ms, "prof": prof, "clocks": clocks, "npts": plan.npts,
           "launches": sum(v[2] for v in prof3.values()),
           "kernels": {k: v[2] for k, v in prof3.items()},
           "tuning": {k: v for k, v in tuning.items() if k != "ms_per_pair"}}

    if e2e_wanted:
        # End to end through the public API with host buffers: every step
        # uploads its input spectrum from pinned host memory, runs the
        # inverse and forward transforms and downloads the resulting
        # spectrum.  Copies run on their own streams, double-buffered, so that
        # step i+1's upload and step i-1's download overlap step i's compute.
        host_in = [torch.from_numpy(a).to(plan.complex_dtype).pin_memory() for _ in range(2)]
        host_out = [torch.empty_like(host_in[0]).pin_memory() for _ in range(2)]
        dev_in = [torch.empty_like(spec_in) for _ in range(2)]
        dev_out = [torch.empty_like(spec_out) for _ in range(2)]
        up, down = torch.cuda.Stream(device), torch.cuda.Stream(device)
        computed = [torch.cuda.Event() for _ in range(2)]
        uploaded = [torch.cuda.Event() for _ in range(2)]
        downloaded = [torch.cuda.Event() for _ in range(2)]
        for e in computed + downloaded:
            e.record(stream)

        def upload(i):
            b = i % 2
            up.wait_event(computed[b])            # step i-2 no longer reads dev_in[b]
            with torch.cuda.stream(up):
                dev_in[b].copy_(host_in[b], non_blocking=True)
                uploaded[b].record(up)

        def e2e_steps(n):
            up.wait_stream(stream)                # nothing starts before the timer
            upload(0)
            for i in range(n):
                b = i % 2
                if i + 1 < n:
                    upload(i + 1)
                stream.wait_event(uploaded[b])
                stream.wait_event(downloaded[b])  # step i-2's result is out of dev_out[b]
                plan.inverse(dev_in[b], out=grid)
                plan.forward(grid, out=dev_out[b])
                computed[b].record(stream)
                down.wait_event(computed[b])
                with torch.cuda.stream(down):
                    host_out[b].copy_(dev_out[b], non_blocking=True)
                    downloaded[b].record(down)
            stream.wait_stream(down)

        e2e_steps(max(args.warmup, 1))
        torch.cuda.synchronize()
        barrier(dist, local)
        ev0.record(stream)
        e2e_steps(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(dist, ev0.elapsed_time(ev1), device)
        nbytes = host_in[0].numel() * host_in[0].element_size()
        res["e2e"] = {"value": job_throughput(world, F, args.steps, e2e_ms),
                      "unit": UNIT, "h2d_bytes_per_step": nbytes,
                      "d2h_bytes_per_step": nbytes,
                      "copies": "pinned host buffers, double-buffered on copy streams "
                                "overlapping the neighbouring steps' compute"}
    plan.close()
    del spec_in, grid, spec_out
    torch.cuda.empty_cache()
    return res


def native_arm(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    device = torch.device("cuda", local)

    from paper_1711_11296_gb300 import workloads as W
    w = W.WORKLOADS[args.workload]
    prec = "bf16x3" if args.precision == "auto" else args.precision
    F = args.fields if args.fields > 0 else w.F
    pk, pk_src = peaks()

    head = run_path(args, w, F, prec, device, dist, local, rank, world,
                    not args.no_e2e)
    value = job_throughput(world, F, args.steps, head["ms"])
    prof = head["prof"]
    name, (tot_ms, n) = max(prof.items(), key=lambda kv: kv[1][0])
    npts = head["npts"]
    roof = roofline_for(name, tot_ms, n, w, F, prec, pk, pk_src, npts, args.grid)
    stages = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1],
                  "kernels": head["kernels"].get(k),
                  "roofline": roofline_for(k, v[0], v[1], w, F, prec, pk, pk_src, npts,
                                           args.grid)}
              for k, v in prof.items()}

    other = None
    if prec != "fp64" and args.precision == "auto" and not args.no_fp64:
        import copy
        a64 = copy.copy(args)
        a64.steps = min(args.steps, 10)      # the FP64 path is ~40x slower
        r64 = run_path(a64, w, F, "fp64", device, dist, local, rank, world, False)
        n64, (t64, c64) = max(r64["prof"].items(), key=lambda kv: kv[1][0])
        other = {"path": "fp64", "steps": a64.steps,
                 "value": job_throughput(world, F, a64.steps, r64["ms"]),
                 "ms_per_step": r64["ms"] / a64.steps,
                 "roofline": roofline_for(n64, t64, c64, w, F, "fp64", pk, pk_src, npts,
                                          args.grid),
                 "gpu_launches": r64["launches"]}
        other["split_speedup"] = value / other["value"]

    cpu = None
    # (the oracle sample times the full grid; a reduced grid has no CPU leg)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.grid != "reduced":
        cpu = cpu_baseline(w)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32+" + prec,
            "data": "synthetic",
            "config": {"workload": w.name, "N": w.N, "J": w.J, "I": w.I,
                       "field_levels_per_gpu": F, "path": prec, "grid": args.grid,
                       "grid_points_per_field": npts,
                       "reduced_rule": args.reduced_rule if args.grid == "reduced" else None,
                       "reduced_transform": bool(args.reduced),
                       "parallelism": "replicas" if world > 1 else "single",
                       "launch_shapes": head.get("tuning"),
                       "l2": "inputs larger than L2 (grid %.1f GB)"
                             % (F * npts * (8 if prec == "fp64" else 4) / 1e9)},
            "roofline": dict(roof, note=("algorithmic work of the full transform; the "
                                         "reduced transform skips part of it")
                             if args.reduced else roof.get("note")),
            "stages": stages, "fp64_path": other,
            "cpu_baseline": cpu, "e2e": head.get("e2e"),
            "clocks": head["clocks"], "gpu_launches": head["launches"],
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def batch_arm(args):
    """The two batched configurations that are not the headline: the uneven
    ensemble (16 members x {T63, T127, T255, T511} x 64 field-levels) as one
    group per stage, eagerly and as a CUDA-graph replay, and the nested
    restriction ladder (a T511 grid of 64 fields to T255 and T127 spectra).
    Timed with CUDA events after warm-up; one JSON line."""
    import torch
    from paper_1711_11296_gb300 import sht, workloads as W
    torch.cuda.set_device(0)
    prec = "bf16x3" if args.precision == "auto" else args.precision
    steps = min(args.steps, 5) if prec == "fp64" else args.steps

    def timeit(fn, n, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    line = {"metric": None, "unit": None, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "dtype": "f64" if prec == "fp64" else "f32+" + prec,
            "data": "synthetic"}
    if args.workload == "ensemble":
        members = W.ENSEMBLE
        plans = [sht.Plan(w.N, w.J, w.I, w.F, prec) for w in members]
        grp = sht.Group(plans)
        specs = [torch.from_numpy(W.workload_spectrum(w)).to(device="cuda",
                                                            dtype=plans[0].complex_dtype)
                 for w in members]
        grids = [p.empty_grid() for p in plans]
        outs = [p.empty_spec() for p in plans]

        def pair():
            grp.inverse(specs, out=grids)
            grp.forward(grids, out=outs)

        ms = timeit(pair, steps, args.warmup)
        nfl = sum(w.F for w in members)
        line.update({"metric": "ensemble field-level transform pairs/s", "unit": UNIT,
                     "value": nfl / (ms / 1e3), "ms_per_step": ms,
                     "config": {"workload": "ensemble",
                                "members": ["%s (N=%d, J=%d, I=%d, F=%d)"
                                            % (w.name, w.N, w.J, w.I, w.F) for w in members],
                                "field_levels": nfl, "path": prec, "grouped": True}})
        if prec != "fp64":
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                pair()
            torch.cuda.current_stream().wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                pair()
            msg = timeit(graph.replay, steps, args.warmup)
            line["graph"] = {"value": nfl / (msg / 1e3), "ms_per_step": msg}
        for p in plans:
            p.status()
    else:
        fine = W.LADDER[0]
        dt = torch.float64 if prec == "fp64" else torch.float32
        gen = torch.Generator(device="cuda").manual_seed(171111296)
        x = torch.randn(fine.F, fine.J, fine.I, device="cuda", dtype=dt, generator=gen)
        res = {}
        for k, coarse in ((1, W.LADDER[1]), (2, W.LADDER[2])):
            p = sht.Plan(coarse.N, coarse.J, coarse.I, coarse.F, prec)
            out = p.empty_spec()
            ms = timeit(lambda: p.restrict_nested(x, k, out=out), steps, args.warmup)
            res["k%d" % k] = {"to": coarse.name, "ms": ms,
                              "field_levels_per_s": coarse.F / (ms / 1e3)}
            p.status()
        line.update({"metric": "nested restriction field-levels/s",
                     "unit": "field-levels/s", "value": res["k1"]["field_levels_per_s"],
                     "ms_per_step": res["k1"]["ms"], "results": res,
                     "config": {"workload": "ladder", "fine": fine.name, "path": prec,
                                "field_levels": fine.F}})
    print(json.dumps(line))
    return 0


def main():
    args = parse_args()
    if args.workload in ("ensemble", "ladder") and args.impl == "reference":
        print(json.dumps({"impl": "reference", "unavailable":
                          "the oracle arm times the single-plan workloads only"}))
        return 0
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload in ("ensemble", "ladder"):
        return batch_arm(args)
    return native_arm(args)


if __name__ == "__main__":
    sys.exit(main())
