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


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="T639",
                    help="T31, T159, T319, T639 (one JSON line in the bench contract), "
                         "or ensemble / ladder / alias (the grouped ensemble, the nested "
                         "restriction ladder and the aliasing products of Sec. 4.2, "
                         "timed with CUDA events)")
    ap.add_argument("--grid", default="cc",
                    choices=["cc", "fejer1", "reduced", "octahedral", "icositetrahedral"],
                    help="latitude grid: Clenshaw-Curtis, the reduced Clenshaw-Curtis "
                         "grid of the 1e-16 reduction rule (Sec. 6), the octahedral or "
                         "icositetrahedral Clenshaw-Curtis grid (Sec. 6), or the shifted "
                         "grid of Fejer's first rule")
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
    ap.add_argument("--adjoint", action="store_true",
                    help="time the adjoint pair (adjoint of the analysis, spectrum -> "
                         "grid, then adjoint of the synthesis, grid -> spectrum) "
                         "instead of the transform pair")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the FP64/FP32 pipe probes (the FP64 roofline then uses "
                         "the nominal peak)")
    return ap.parse_args(argv)


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
                 "--format=csv,noheader,nounits", "-lms", "50"],
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
_FFT_INV_T639x64 = (419.963 + 786.312) * 1e6   # bytes, fft_inverse<float, 1280>
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


def measure_pipe_peaks(device):
    """FP64 and FP32 ceilings measured in this process: the library's FMA
    throughput probe (DFMA, FFMA, paired FFMA; best of 5 launches of ~20 ms)
    and cuBLAS GEMMs through torch.matmul (FP64 4096^3, FP32 8192^3 with TF32
    off, best of 3).  TFLOP/s, 2 flops per FMA."""
    import ctypes
    import torch
    from paper_1711_11296_gb300 import _native
    out = {}
    stream = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    for kind, name in ((0, "dfma_probe"), (1, "ffma_probe"), (2, "ffma2_probe")):
        v = ctypes.c_double()
        _native.check(_native.lib.sht_measure_fma_peak(kind, 5, stream, ctypes.byref(v)))
        out[name] = v.value
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for dt, n, name in ((torch.float64, 4096, "dgemm"), (torch.float32, 8192, "sgemm")):
            a = torch.randn(n, n, dtype=dt, device=device)
            b = torch.randn(n, n, dtype=dt, device=device)
            c = a @ b
            torch.cuda.synchronize()
            best = None
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
            out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    torch.cuda.empty_cache()
    out["fp64_tflops"] = max(out["dfma_probe"], out["dgemm"])
    out["fp32_tflops"] = max(out["ffma_probe"], out["ffma2_probe"], out["sgemm"])
    return out


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_tables(w, mstep):
    """The oracle's P~ tables of the sampled zonal wavenumbers m = 0, mstep,
    2 mstep, ... (built once, outside every timed region, as the GPU plan
    builds its tables at plan creation)."""
    import oracle as O
    ms = list(range(0, w.N + 1, mstep))
    return ms, O.pnm_tables(w.N, w.J, ms)


def oracle_sample(w, ms, tables):
    """One field-level pair (synthesis then analysis) restricted to the zonal
    wavenumbers ``ms`` with prebuilt P~ tables; returns (seconds, fraction
    of the full pair's Legendre work this sample covers)."""
    import oracle as O
    from paper_1711_11296_gb300 import workloads as W
    a = W.workload_spectrum(w, F=1)
    ncoef = (w.N + 1) * (w.N + 2) // 2
    frac = sum(w.N - m + 1 for m in ms) / ncoef
    t0 = time.perf_counter()
    X = np.zeros((1, w.J, len(ms)), dtype=np.complex128)
    for k, m in enumerate(ms):
        r0 = O.coef_offset(w.N, m)
        X[:, :, k] = O.legendre_inverse_m(a[r0:r0 + w.N - m + 1], tables[m])
    grid = O.dft_inverse(X, w.I, ms=ms)
    O.analysis(grid, w.N, ms=ms, pnm=tables)
    return time.perf_counter() - t0, frac


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_baseline(w, mstep=4):
    ms, tables = oracle_tables(w, mstep)
    oracle_sample(w, ms, tables)                     # warm-up
    sec, frac = oracle_sample(w, ms, tables)
    return {"value": frac / sec, "unit": UNIT, "cores": host_cores(),
            "kind": "oracle",
            "sample": ("1 field-level pair of %s, zonal wavenumbers m = 0 mod %d "
                       "(%.1f%% of the Legendre work), %.1f s; P~ tables built before "
                       "the timer (as the GPU plan's); plain CPU oracle (direct DFT + "
                       "direct Legendre sums), not an optimised CPU SHT"
                       % (w.name, mstep, 100 * frac, sec))}


def workload_config(w, F, args, npts, real_bytes, world):
    """The workload as both arms name it (sizes, grid, field-levels)."""
    return {"workload": w.name, "N": w.N, "J": w.J, "I": w.I,
            "field_levels_per_gpu": F, "grid": args.grid,
            "grid_points_per_field": npts,
            "reduced_rule": args.reduced_rule if args.grid == "reduced" else None,
            "longitudes": ("16 + 4 j on the j-th latitude from either pole"
                           if args.grid == "octahedral" else
                           "6 min(j, j30), tropical rows alternately shifted by half a "
                           "spacing" if args.grid == "icositetrahedral" else None),
            "reduced_transform": bool(args.reduced),
            "step": "adjoint pair" if args.adjoint else "transform pair",
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (grid %.1f GB)" % (F * npts * real_bytes / 1e9)}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1711_11296_gb300 import workloads as W
    w = W.WORKLOADS[args.workload]
    if args.grid != "cc" or args.adjoint or args.reduced:
        print(json.dumps({"impl": "reference", "unavailable":
                          "the oracle arm times the plain transform pair on the full "
                          "Clenshaw-Curtis grid only"}))
        return 0
    mstep = 16
    ms, tables = oracle_tables(w, mstep)             # untimed, as the GPU plan tables
    for _ in range(args.warmup):
        oracle_sample(w, ms, tables)
    tot, frac = 0.0, 0.0
    for _ in range(args.steps):
        s, frac = oracle_sample(w, ms, tables)
        tot += s
    value = frac * args.steps / tot
    F = args.fields if args.fields > 0 else w.F
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(w, F, args, w.J * w.I, 4, args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(),
                         "kind": "oracle",
                         "sample": "each step: 1 field-level pair of the workload, zonal "
                                   "wavenumbers m = 0 mod %d (%.1f%% of the Legendre "
                                   "work), scaled to the whole pair; P~ tables built "
                                   "before the timer" % (mstep, 100 * frac)},
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
        if pk.get("fp64_tflops"):
            peak = pk["fp64_tflops"]
            src = ("measured in this run: max of the DFMA probe (%.3f) and cuBLAS DGEMM "
                   "(%.3f) TFLOP/s" % (pk.get("dfma_probe", 0.0), pk.get("dgemm", 0.0)))
        else:
            peak = 1.25
            src = "nominal GB300 FP64 1.25 TFLOP/s (no FP64 probe in this run)"
        roof = {"kernel": name + "_fp64", "bound": "alu",
                "achieved": fl / per_launch_s / 1e12, "peak": peak,
                "unit": "TFLOP/s", "traffic": None, "peak_source": src}
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
    t = MEASURED_TRAFFIC.get((name, prec, w.name, F)) if grid in ("cc", "fejer1") else None
    if t is not None:
        roof["traffic"] = t
        roof["traffic_note"] = ("ncu DRAM bytes of the T639 x 64 capture scaled by the "
                                "field count; writes still in L2 at the end of a launch "
                                "are not counted")
    return roof


def step_bytes(w, F, prec, npts=None):
    """Algorithmic HBM bytes of one split-path step (transform or adjoint
    pair): both FFT stages and both Legendre contractions."""
    return (2 * fft_bytes(w, F, 4, npts) + split_gemm_bytes(w, F, prec, False)
            + split_gemm_bytes(w, F, prec, True))


def run_path(args, w, F, prec, device, dist, local, rank, world, e2e_wanted,
             a_host=None, sample_fields=8):
    """Plan, autotune, warm up and time ``args.steps`` steps of one path;
    optionally the end-to-end variant.  a_host: the input spectrum (complex,
    [ncoef][F]); default the workload's seeded spectrum of this rank's
    fields.  Returns timings, per-stage profile, clocks and the first
    ``sample_fields`` columns of the last step's output (host)."""
    import torch
    from paper_1711_11296_gb300 import sht, workloads as W
    if args.grid == "reduced":
        # longitudes per latitude by the reduction rule, from an FP64 plan's
        # P~ table (plan setup, untimed)
        sizes = sht.Plan(w.N, w.J, w.I, 1, "fp64",
                         device=device).reduced_grid_sizes(args.reduced_rule)
        plan = sht.Plan(w.N, w.J, w.I, F, prec, device=device, grid="reduced",
                        lat_points=sizes)
    elif args.grid in ("octahedral", "icositetrahedral"):
        sizes, shift = ((sht.octahedral_grid_sizes(w.J), None) if args.grid == "octahedral"
                        else sht.icositetrahedral_grid_sizes(w.J))
        plan = sht.Plan(w.N, w.J, w.I, F, prec, device=device, grid="reduced",
                        lat_points=sizes, half_shift=shift)
    else:
        plan = sht.Plan(w.N, w.J, w.I, F, prec, device=device, grid=args.grid)
    if args.reduced:
        plan.set_reduced(True)
    # launch shapes picked by the library's autotuner (plan setup, untimed)
    tuning = plan.tuning if args.no_autotune else plan.autotune(reps=2)
    a = W.workload_spectrum(w, F=F, field0=rank * F) if a_host is None else a_host
    spec_in = torch.from_numpy(a).to(device=device, dtype=plan.complex_dtype)
    grid = plan.empty_grid()
    spec_out = plan.empty_spec()

    if args.adjoint:
        def pair(src, dst):
            plan.adjoint(0, src, out=grid)        # spectrum -> grid
            plan.adjoint(1, grid, out=dst)        # grid -> spectrum
    else:
        def pair(src, dst):
            plan.inverse(src, out=grid)
            plan.forward(grid, out=dst)

    for _ in range(max(args.warmup, 0)):
        pair(spec_in, spec_out)
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
        pair(spec_in, spec_out)
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
           "tuning": {k: v for k, v in tuning.items() if k != "ms_per_pair"},
           "sample": spec_out[:, :sample_fields].to(torch.complex128).cpu().numpy()}

    if e2e_wanted:
        res["e2e"] = e2e_run(args, plan, pair, a, spec_in, spec_out, stream, device, dist,
                             local, world, F)
    plan.close()
    del spec_in, grid, spec_out
    torch.cuda.empty_cache()
    return res


def e2e_run(args, plan, pair, a, spec_in, spec_out, stream, device, dist, local, world, F):
    """End to end through the public API with host buffers: every step
    uploads its input spectrum from pinned host memory, runs the pair and
    downloads the resulting spectrum.  Copies run on their own streams,
    double-buffered, so that step i+1's upload and step i-1's download
    overlap step i's compute; only the first upload (fill) and the last
    download (drain) cannot overlap compute.  Also measures each copy
    direction alone, and the fill, drain and steady-state step times."""
    import torch
    host_in = [torch.from_numpy(a).to(plan.complex_dtype).pin_memory() for _ in range(2)]
    host_out = [torch.empty_like(host_in[0]).pin_memory() for _ in range(2)]
    dev_in = [torch.empty_like(spec_in) for _ in range(2)]
    dev_out = [torch.empty_like(spec_out) for _ in range(2)]
    up, down = torch.cuda.Stream(device), torch.cuda.Stream(device)
    computed = [torch.cuda.Event() for _ in range(2)]
    uploaded = [torch.cuda.Event() for _ in range(2)]
    downloaded = [torch.cuda.Event() for _ in range(2)]
    first = torch.cuda.Event(enable_timing=True)
    last = torch.cuda.Event(enable_timing=True)
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
            if i == 0:
                first.record(stream)
            pair(dev_in[b], dev_out[b])
            computed[b].record(stream)
            if i == n - 1:
                last.record(stream)
            down.wait_event(computed[b])
            with torch.cuda.stream(down):
                host_out[b].copy_(dev_out[b], non_blocking=True)
                downloaded[b].record(down)
        stream.wait_stream(down)

    def copy_alone(dst, src, st):
        st.wait_stream(stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        best = None
        for _ in range(3):
            e0.record(st)
            with torch.cuda.stream(st):
                dst.copy_(src, non_blocking=True)
            e1.record(st)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best

    nbytes = host_in[0].numel() * host_in[0].element_size()
    h2d_ms = copy_alone(dev_in[0], host_in[0], up)
    d2h_ms = copy_alone(host_out[0], dev_out[0], down)
    e2e_steps(max(args.warmup, 1))
    torch.cuda.synchronize()
    barrier(dist, local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    e2e_steps(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    local_ms = ev0.elapsed_time(ev1)
    e2e_ms = max_over_ranks(dist, local_ms, device)
    # the last step's download must hold the same spectrum as the device
    # result (copies complete and in order)
    b = (args.steps - 1) % 2
    if not torch.equal(host_out[b], dev_out[b].cpu()):
        raise RuntimeError("end-to-end download does not match the device result")
    fill = ev0.elapsed_time(first)
    drain = last.elapsed_time(ev1)
    steady = first.elapsed_time(last) / args.steps
    return {"value": job_throughput(world, F, args.steps, e2e_ms),
            "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "ms_per_step": e2e_ms / args.steps,
            "copies": "pinned host buffers, double-buffered on copy streams "
                      "overlapping the neighbouring steps' compute",
            "h2d_gbs_alone": nbytes / (h2d_ms * 1e-3) / 1e9,
            "d2h_gbs_alone": nbytes / (d2h_ms * 1e-3) / 1e9,
            "fill_ms": fill, "drain_ms": drain, "steady_ms_per_step": steady,
            "steady_value": job_throughput(world, F, 1, steady)}


def transform_errors(w, prec, a, device, args, nf):
    """Relative L2 of each split transform against the FP64 path on the same
    input values, on plans of the first nf field-levels (columns are
    independent, so these are the timed plan's errors on those columns):
    the grid of the synthesis (or of the adjoint of the analysis), and the
    spectrum of the analysis (or of the adjoint of the synthesis) of the
    split path's own grid."""
    import torch
    from paper_1711_11296_gb300 import sht
    if args.grid not in ("cc", "fejer1"):
        return None
    kw = dict(device=device, grid=args.grid)
    p32 = sht.Plan(w.N, w.J, w.I, nf, prec, **kw)
    p64 = sht.Plan(w.N, w.J, w.I, nf, "fp64", **kw)
    a64 = torch.from_numpy(np.ascontiguousarray(a[:, :nf])).to(device)
    a32 = a64.to(p32.complex_dtype)
    if args.adjoint:
        g32, g64 = p32.adjoint(0, a32), p64.adjoint(0, a64)
        s32, s64 = p32.adjoint(1, g32), p64.adjoint(1, g32.double())
        names = ("adjoint_of_analysis", "adjoint_of_synthesis")
    else:
        g32, g64 = p32.inverse(a32), p64.inverse(a64)
        s32, s64 = p32.forward(g32), p64.forward(g32.double())
        names = ("synthesis", "analysis")

    def rel(x, y):
        x = torch.view_as_real(x) if x.is_complex() else x
        y = torch.view_as_real(y) if y.is_complex() else y
        return float((x.double() - y.double()).norm() / y.double().norm())

    out = {names[0]: rel(g32, g64), names[1]: rel(s32, s64)}
    p32.close()
    p64.close()
    return out


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
    if not args.no_peaks:
        pk = dict(pk, **measure_pipe_peaks(device))

    # the split path's input values (FP32) are the FP64 comparison's input too
    a = W.workload_spectrum(w, F=F, field0=rank * F)
    if prec != "fp64":
        a = a.astype(np.complex64).astype(np.complex128)
    head = run_path(args, w, F, prec, device, dist, local, rank, world,
                    not args.no_e2e, a_host=a)
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
    accuracy = None
    if prec != "fp64" and args.precision == "auto" and not args.no_fp64:
        import copy
        a64 = copy.copy(args)
        a64.steps = min(args.steps, 10)      # the FP64 path is ~50x slower
        r64 = run_path(a64, w, F, "fp64", device, dist, local, rank, world, False,
                       a_host=a)
        n64, (t64, c64) = max(r64["prof"].items(), key=lambda kv: kv[1][0])
        other = {"path": "fp64", "steps": a64.steps,
                 "value": job_throughput(world, F, a64.steps, r64["ms"]),
                 "ms_per_step": r64["ms"] / a64.steps,
                 "roofline": roofline_for(n64, t64, c64, w, F, "fp64", pk, pk_src, npts,
                                          args.grid),
                 "gpu_launches": r64["launches"]}
        other["split_speedup"] = value / other["value"]
        # accuracy of the timed split pair: its output against the FP64 GPU
        # path's output of the same pair on the same input values (the FP64
        # path matches the oracle to 1e-12 in the tests), and of each of its
        # two transforms alone
        s, d = head["sample"], r64["sample"]
        per = [float(np.linalg.norm(s[:, k] - d[:, k]) / np.linalg.norm(d[:, k]))
               for k in range(s.shape[1])]
        accuracy = {"pair_rel_l2_vs_fp64_path": float(np.linalg.norm(s - d)
                                                      / np.linalg.norm(d)),
                    "pair_max_field_rel_l2": max(per), "fields": s.shape[1],
                    "per_transform": transform_errors(w, prec, a, device, args,
                                                      s.shape[1]),
                    "what": ("relative L2 against the FP64 GPU path on the same input "
                             "values, first %d field-levels: the timed %s pair's "
                             "spectral output, and each transform alone (the "
                             "synthesis's grid, the analysis's spectrum of the split "
                             "synthesis's grid); target <= 1e-6 per transform"
                             % (s.shape[1], "adjoint" if args.adjoint else "transform"))}

    cpu = None
    # (the oracle sample times the full grid; a reduced grid has no CPU leg)
    if (rank == 0 and world == 1 and not args.no_cpu_baseline and args.grid == "cc"
            and not args.adjoint and not args.reduced):
        cpu = cpu_baseline(w)

    if rank == 0:
        real_bytes = 8 if prec == "fp64" else 4
        sb = step_bytes(w, F, prec, npts) if prec != "fp64" else None
        line = {
            "metric": ("T639 adjoint pairs/s per field-level" if args.adjoint else METRIC),
            "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32+" + prec,
            "dtype_note": (None if prec == "fp64" else
                           "FP32 FFTs; Legendre contractions as %s split products on the "
                           "tensor cores with FP32 accumulation into two accumulators, "
                           "recombined in FP32 (the result is stored as FP32); FP64 for "
                           "the P~ recurrence, weights and tables" % prec),
            "data": "synthetic",
            "path": prec,
            "config": workload_config(w, F, args, npts, real_bytes, world),
            "launch_shapes": head.get("tuning"),
            "roofline": dict(roof, note=("algorithmic work of the full transform; the "
                                         "reduced transform skips part of it")
                             if args.reduced else roof.get("note")),
            "step_roofline": (None if sb is None else
                              {"bound": "hbm", "bytes": sb,
                               "achieved": sb / (head["ms"] / args.steps * 1e-3) / 1e9,
                               "peak": pk["hbm_gbs"], "unit": "GB/s",
                               "frac": sb / (head["ms"] / args.steps * 1e-3) / 1e9
                               / pk["hbm_gbs"],
                               "what": "algorithmic bytes of the whole step (both FFTs "
                                       "and both contractions) over the step time"}),
            "accuracy": accuracy,
            "peaks": {k: v for k, v in pk.items()
                      if k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained",
                               "dfma_probe", "ffma_probe", "ffma2_probe", "dgemm",
                               "sgemm", "fp64_tflops", "fp32_tflops")},
            "stages": stages, "fp64_path": other,
            "cpu_baseline": cpu, "e2e": head.get("e2e"),
            "clocks": head["clocks"], "gpu_launches": head["launches"],
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def group_pair_bytes(members, prec):
    """Algorithmic HBM bytes of one grouped transform pair over the members."""
    return sum(step_bytes(w, w.F, prec) for w in members)


def restriction_bytes(coarse, F, prec):
    """Algorithmic HBM bytes of one nested restriction to the coarse plan:
    the coarse sub-grid's points read once (strided in the fine grid; at
    stride 2^k a 32-byte sector holds at most 8 / 2^k of them, so DRAM
    reads whole fine rows), the Fourier workspace written and read, the
    contraction's tables and the spectrum written."""
    return fft_bytes(coarse, F, 4) + split_gemm_bytes(coarse, F, prec, False)


def alias_step_bytes(w, F, prec):
    """Algorithmic HBM bytes of one aliasing-product step (Sec. 4.2): three
    syntheses and two analyses, plus, inside W's inverse FFT, the U and V
    grids read and the U V and U V W grids written in place of W's grid."""
    inv = fft_bytes(w, F, 4) + split_gemm_bytes(w, F, prec, True)
    fwd = fft_bytes(w, F, 4) + split_gemm_bytes(w, F, prec, False)
    return 3 * inv + 2 * fwd + 3 * F * w.J * w.I * 4


def alias_arm(args, pk, pk_src):
    """The aliasing experiment of Sec. 4.2 at Tc479: one step is the five
    transforms of the quadratic and cubic terms of F field-levels per field
    (syntheses of U, V, W; products inside W's inverse FFT; analyses of U V
    and U V W), timed with CUDA events.  Beside the timing: the split
    path's error against the FP64 GPU path on the same inputs, and the
    paper's normalised aliasing errors of the cubic CC grid measured with the
    FP64 path against an alias-free reference on the J = 4N+3 CC grid (the
    CC rule with J >= 4N+1 nodes and I > 4N longitudes integrates the cubic
    term's projections exactly)."""
    import torch
    from paper_1711_11296_gb300 import sht, workloads as W
    w = W.ALIAS
    prec = "bf16x3" if args.precision == "auto" else args.precision
    F = args.fields if args.fields > 0 else w.F
    host = [W.random_spectrum(w.N, F, w.envelope, seed=W.SEED_BASE + 1000 * w.index + 100 * k)
            for k in range(3)]
    p = sht.Plan(w.N, w.J, w.I, F, prec)
    specs = [torch.from_numpy(h).to(device="cuda", dtype=p.complex_dtype) for h in host]
    grids = [p.empty_grid(), p.empty_grid()]
    outs = [p.empty_spec(), p.empty_spec()]
    steps = min(args.steps, 5) if prec == "fp64" else args.steps

    def step():
        p.alias_products(*specs, grids=grids, out=outs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    p.status()
    checks = {"finite": all(bool(torch.isfinite(torch.view_as_real(o)).all()) for o in outs)}
    line = {"metric": "Tc479 aliasing-product steps: field-levels per second",
            "unit": "field-levels/s", "value": F / (ms / 1e3), "ms_per_step": ms,
            "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "dtype": "f64" if prec == "fp64" else "f32+" + prec, "data": "synthetic",
            "config": {"workload": "alias", "N": w.N, "J": w.J, "I": w.I,
                       "field_levels_per_field": F, "path": prec,
                       "spectra": "Re, Im uniform in [1, 2] (n+1)^-1/3 (Sec. 4.2)"}}
    if prec != "fp64":
        by = alias_step_bytes(w, F, prec)
        line["roofline"] = {"bound": "hbm", "bytes": by, "achieved": by / (ms * 1e-3) / 1e9,
                            "peak": pk["hbm_gbs"], "unit": "GB/s",
                            "frac": by / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                            "peak_source": "%s hbm_gbs" % pk_src}
    # FP64: the split path's error, and the aliasing errors of the cubic grid
    S = min(F, 4)
    p64 = sht.Plan(w.N, w.J, w.I, S, "fp64")
    sub = [np.ascontiguousarray(h[:, :S]) for h in host]
    if prec != "fp64":
        sub = [a.astype(np.complex64).astype(np.complex128) for a in sub]
    t64 = [torch.from_numpy(a).cuda() for a in sub]
    q64, c64 = p64.alias_products(*t64)
    if prec != "fp64":
        errs = {}
        for nm, got, ref in (("quadratic", outs[0], q64), ("cubic", outs[1], c64)):
            g = got[:, :S].to(torch.complex128)
            errs[nm] = float((g - ref).norm() / ref.norm())
        checks["rel_l2_vs_fp64"] = errs
        checks["accuracy_ok"] = max(errs.values()) <= 2e-6
    Jr = 4 * w.N + 3
    pref = sht.Plan(w.N, Jr, w.I, S, "fp64")
    qr, cr = pref.alias_products(*t64)
    stats = {}
    for nm, test, ref, thr in (("quadratic", q64, qr, 1e-5), ("cubic", c64, cr, 1e-8)):
        e = ((test - ref).abs() / ref.abs()).cpu().numpy()
        stats[nm] = {"median": float(np.median(e)), "p90": float(np.quantile(e, 0.9)),
                     "max": float(e.max()), "threshold": thr,
                     "fraction_below": float((e < thr).mean())}
    line["aliasing_errors"] = {
        "grid": "cubic CC Tc479 (J = %d, I = %d), FP64 path" % (w.J, w.I),
        "reference": "alias-free CC grid J = %d, I = %d, FP64 path" % (Jr, w.I),
        "fields": S, "terms": stats,
        "paper": "Sec. 4.2: below 1e-5 (quadratic) and 1e-8 (cubic) for most (n, m)"}
    for q_ in (p64, pref):
        q_.status()
        q_.close()
    line["checks"] = checks
    bad = [k for k in ("finite", "accuracy_ok") if k in checks and not checks[k]]
    if bad:
        raise RuntimeError("aliasing workload failed its checks %s: %s" % (bad, checks))
    print(json.dumps(line))
    return 0


def batch_arm(args):
    """The two batched configurations that are not the headline: the uneven
    ensemble (16 members x {T63, T127, T255, T511} x 64 field-levels) as one
    group per stage, eagerly and as a CUDA-graph replay, and the nested
    restriction ladder (a T511 grid of 64 fields to T255 and T127 spectra).
    Timed with CUDA events after warm-up; the outputs are checked (finite;
    sampled fields against an FP64 plan on the same inputs within the split
    tolerance; graph replay equal to the eager launches) and the line is
    refused if a check fails.  One JSON line."""
    import torch
    from paper_1711_11296_gb300 import sht, workloads as W
    torch.cuda.set_device(0)
    prec = "bf16x3" if args.precision == "auto" else args.precision
    steps = min(args.steps, 5) if prec == "fp64" else args.steps
    pk, pk_src = peaks()
    if args.workload == "alias":
        return alias_arm(args, pk, pk_src)
    tol = 1e-6 if prec in ("bf16x3", "fp16x3", "fp16x2") else 5e-5
    sample = 8

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

    def finite(ts):
        return all(bool(torch.isfinite(torch.view_as_real(t) if t.is_complex() else t).all())
                   for t in ts)

    line = {"metric": None, "unit": None, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "dtype": "f64" if prec == "fp64" else "f32+" + prec,
            "data": "synthetic"}
    checks = {}
    if args.workload == "ensemble":
        members = W.ENSEMBLE
        plans = [sht.Plan(w.N, w.J, w.I, w.F, prec) for w in members]
        grp = sht.Group(plans)
        host = [W.workload_spectrum(w).astype(np.complex64).astype(np.complex128)
                for w in members]
        specs = [torch.from_numpy(h).to(device="cuda", dtype=plans[0].complex_dtype)
                 for h in host]
        grids = [p.empty_grid() for p in plans]
        outs = [p.empty_spec() for p in plans]

        def pair():
            grp.inverse(specs, out=grids)
            grp.forward(grids, out=outs)

        ms = timeit(pair, steps, args.warmup)
        nfl = sum(w.F for w in members)
        eager = [o.clone() for o in outs]
        checks["finite"] = finite(outs) and finite(grids)
        line.update({"metric": "ensemble field-level transform pairs/s", "unit": UNIT,
                     "value": nfl / (ms / 1e3), "ms_per_step": ms,
                     "config": {"workload": "ensemble",
                                "members": ["%s (N=%d, J=%d, I=%d, F=%d)"
                                            % (w.name, w.N, w.J, w.I, w.F) for w in members],
                                "field_levels": nfl, "path": prec, "grouped": True}})
        if prec != "fp64":
            by = group_pair_bytes(members, prec)
            line["roofline"] = {"bound": "hbm", "bytes": by,
                                "achieved": by / (ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                                "unit": "GB/s",
                                "frac": by / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                                "what": "algorithmic bytes of both FFTs and both "
                                        "contractions of every member, per grouped pair",
                                "peak_source": "%s hbm_gbs" % pk_src}
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
            checks["graph_equals_eager"] = all(torch.equal(o, e) for o, e in zip(outs, eager))
            # one member (the first `sample` field-levels) per truncation
            # against an FP64 plan on the same input values
            errs = {}
            for w, h, o in zip(members, host, eager):
                p64 = sht.Plan(w.N, w.J, w.I, sample, "fp64")
                a64 = torch.from_numpy(np.ascontiguousarray(h[:, :sample])).cuda()
                ref = p64.forward(p64.inverse(a64)).cpu().numpy()
                got = o[:, :sample].to(torch.complex128).cpu().numpy()
                errs[w.name] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
                p64.close()
            checks["rel_l2_vs_fp64"] = errs
            checks["accuracy_ok"] = max(errs.values()) <= tol
        for p in plans:
            p.status()
    else:
        fine = W.LADDER[0]
        dt = torch.float64 if prec == "fp64" else torch.float32
        gen = torch.Generator(device="cuda").manual_seed(171111296)
        x = torch.randn(fine.F, fine.J, fine.I, device="cuda", dtype=dt, generator=gen)
        res = {}
        errs = {}
        for k, coarse in ((1, W.LADDER[1]), (2, W.LADDER[2])):
            p = sht.Plan(coarse.N, coarse.J, coarse.I, coarse.F, prec)
            out = p.empty_spec()
            ms = timeit(lambda: p.restrict_nested(x, k, out=out), steps, args.warmup)
            res["k%d" % k] = {"to": coarse.name, "ms": ms,
                              "field_levels_per_s": coarse.F / (ms / 1e3)}
            if prec != "fp64":
                by = restriction_bytes(coarse, coarse.F, prec)
                res["k%d" % k]["roofline"] = {
                    "bound": "hbm", "bytes": by, "achieved": by / (ms * 1e-3) / 1e9,
                    "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": by / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                    "what": "algorithmic bytes: the coarse sub-grid once, the Fourier "
                            "workspace, the contraction's tables and spectrum; DRAM "
                            "sectors make the strided reads cover whole fine rows",
                    "peak_source": "%s hbm_gbs" % pk_src}
                p64 = sht.Plan(coarse.N, coarse.J, coarse.I, coarse.F, "fp64")
                ref = p64.restrict_nested(x.double(), k).cpu().numpy()
                got = out.to(torch.complex128).cpu().numpy()
                errs[coarse.name] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
                p64.close()
            checks.setdefault("finite", True)
            checks["finite"] = checks["finite"] and finite([out])
            p.status()
        if errs:
            checks["rel_l2_vs_fp64"] = errs
            checks["accuracy_ok"] = max(errs.values()) <= tol
        line.update({"metric": "nested restriction field-levels/s",
                     "unit": "field-levels/s", "value": res["k1"]["field_levels_per_s"],
                     "ms_per_step": res["k1"]["ms"], "results": res,
                     "config": {"workload": "ladder", "fine": fine.name, "path": prec,
                                "field_levels": fine.F}})
    line["checks"] = checks
    bad = [k for k in ("finite", "graph_equals_eager", "accuracy_ok")
           if k in checks and not checks[k]]
    if bad:
        raise RuntimeError("batched workload failed its checks %s: %s" % (bad, checks))
    print(json.dumps(line))
    return 0


def main():
    args = parse_args()
    if args.workload in ("ensemble", "ladder", "alias") and args.impl == "reference":
        print(json.dumps({"impl": "reference", "unavailable":
                          "the oracle arm times the single-plan workloads only"}))
        return 0
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload in ("ensemble", "ladder", "alias"):
        return batch_arm(args)
    return native_arm(args)


if __name__ == "__main__":
    sys.exit(main())
