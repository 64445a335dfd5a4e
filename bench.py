#!/usr/bin/env python
"""Benchmark of the Brillouin-kernel overlap hot path on GB300.

One step = one application of the massless overlap operator
D_ov = rho (1 + gamma5 f_16,16(H)), H = gamma5 D_bri(-rho), to a batch of
right-hand sides on a 24^3 x 48 lattice: multi-shift CG on D^dagger D + sigma_i
(Kenney-Laub order 16) in FP32 with FP64 reductions and FP64 defect-correction
refinement of every shift to a true relative residual of 1e-10, then one FP64
application of D.  Inputs (stout-smeared synthetic SU(3) field, complex
Gaussian sources) are resident in HBM when the timed region starts.

Printed (rank 0, one JSON line): D_ov applies per second over all ranks, the
stencil's roofline figures measured with CUDA events inside the timed region
(against FMA and copy peaks measured on this GPU), an end-to-end figure
through the same C ABI call with host buffers, and the FP64 CPU oracle timed
on a bounded sample on all host cores and on one.  After the timed region, on
rank 0: the FP64 true residual of every shift of the timed step (an untimed
repeat that reproduces the timed output bit for bit), the single-rhs stencil
in FP32, BF16-link and FP64 form against its HBM and FP64 rooflines, and the
plain FP64 GPU solve with the mixed-over-FP64 ratio.  ``--impl reference``
times the oracle alone.

Multi-GPU (torchrun): every rank runs an independent replica (own gauge field
and sources), there is no data-path collective; the per-step time is the
maximum over ranks and the value counts the applications of all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D_ov applies/s at 24^3x48 (mixed vs FP64, 1e-10); bri_apply HBM GB/s vs roofline"
UNIT = "D_ov applies/s"
DIMS = (24, 24, 24, 48)
KL_ORDER = 16
RHO = 1.0
C_SW = 1.0
TOL = 1e-10
GAUGE_SEED = 1
FALLBACK_HBM_GBS = 6800.0
# algorithmic bytes of one FP32 Brillouin stencil launch: per site the 40
# stored links (40 x 72 B) and the clover blocks (72 floats) once, and per site
# and right-hand side one spinor read and one written (2 x 96 B) (App. C)
LINK_BYTES = {1: 40 * 72, 2: 40 * 36}
CLOVER_BYTES = 72 * 4
SPINOR_BYTES = 2 * 96
# algorithmic flops of the Brillouin matvec per site and right-hand side (App. C)
FLOPS_PER_SITE = 30168
# algorithmic bytes of one FP64 stencil launch per site: links 40 x 144, clover 72 doubles,
# and per site and rhs one spinor read and one written (2 x 192 B)
F64_LINK_CLOVER_BYTES = 40 * 144 + 72 * 8
F64_SPINOR_BYTES = 2 * 192
# oracle sample lattices (one D_ov of the workload's settings per process): the
# cpu_baseline of the GPU arm, and the smaller per-step sample of the reference
# arm, which runs warmup + steps rounds and has to end within a few minutes
CPU_SAMPLE = (4, 4, 4, 4)
REF_SAMPLE = (4, 4, 2, 2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)  # x ~9 s per step at 4 rhs
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nrhs", type=int, default=4)
    ap.add_argument("--links", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain FP64 D_ov (1 rhs) timed after the timed region")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the post-timed checks (true residuals, single-rhs stencils, FMA probes)")
    ap.add_argument("--stencil-probe", default=None, metavar="LX,LY,LZ,LT",
                    help="profiling helper: only launch the FP32 Brillouin stencil on this lattice and print "
                         "its CUDA-event time (used for the ncu captures under profiles/)")
    ap.add_argument("--batch-c4", action="store_true",
                    help="time the batched workload instead: 12 point sources on 16^3x32 plus 8 uneven lattices, "
                         "KL order 12, mixed precision, one concurrent batch vs lattice after lattice")
    ap.add_argument("--c2", action="store_true",
                    help="time the FP64 cascaded massive solve on 16^3x32 (KL order 16, cascade order 4, c_SW=1) "
                         "for the Brillouin and Wilson kernels instead")
    ap.add_argument("--c2-masses", default="0.1", help="comma-separated am values of --c2")
    ap.add_argument("--c2-tol", type=float, default=1e-10, help="outer relative residual of --c2")
    ap.add_argument("--c5-grad", action="store_true",
                    help="time the mixed-precision backward (overlap_grad, KL order 12) on 32^3x64 instead")
    ap.add_argument("--probe-nrhs", type=int, default=1)
    ap.add_argument("--probe-launches", type=int, default=4)
    ap.add_argument("--probe-prec", choices=("f32", "dw", "f64"), default="f32",
                    help="stencil probe precision: FP32, double-word FP32 (complex128 in/out) or FP64")
    return ap.parse_args()


def stencil_probe(args):
    import torch

    import synthetic_fields as sf
    from paper_1701_00726_gb300 import Lattice
    dims = tuple(int(v) for v in args.stencil_probe.split(","))
    vol = dims[0] * dims[1] * dims[2] * dims[3]
    lat = Lattice(dims)
    lat.build_links(torch.from_numpy(sf.gauge_field(dims, 1, eps=0.5, device="cuda")).cuda(), C_SW)
    dt = torch.complex64 if args.probe_prec == "f32" else torch.complex128
    dw = args.probe_prec == "dw"
    x = torch.randn((args.probe_nrhs, vol * 12), dtype=dt, device="cuda")
    y = torch.empty_like(x)
    lat.bri_apply(x, -RHO, out=y, double_word=dw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.probe_launches):
        lat.bri_apply(x, -RHO, out=y, double_word=dw)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.probe_launches
    if args.probe_prec == "f32":
        byt = vol * (LINK_BYTES[1] + CLOVER_BYTES + SPINOR_BYTES * args.probe_nrhs)
    else:
        byt = vol * (F64_LINK_CLOVER_BYTES + F64_SPINOR_BYTES * args.probe_nrhs)
    print(json.dumps({"stencil_probe": list(dims), "prec": args.probe_prec, "nrhs": args.probe_nrhs, "ms": ms,
                      "alg_GBps": byt / ms / 1e6, "alg_TFLOPs": vol * args.probe_nrhs * FLOPS_PER_SITE / ms / 1e9}),
          flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    v = d[k]
                    return float(v["value"] if isinstance(v, dict) else v), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def stencil_traffic():
    """dram bytes per launch of the FP32 stencil from the committed ncu summary,
    valid only while the stencil source is unchanged (hash match)."""
    p = os.path.join(ROOT, "profiles", "bri_stencil_traffic.txt")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        if d.get("stencil_source_sha256_16") != stencil_source_hash():
            return None
        return d
    except Exception:
        return None


def stencil_traffic_per_launch(traffic, vol, nlaunch, units, prec):
    """DRAM bytes per launch of the step's FP32 stencil launches from the committed
    ncu capture: per-site link and clover bytes plus per-site-and-rhs spinor bytes
    (both measured on a smaller lattice, scaled by the sites and rhs processed)."""
    if traffic is None or prec != 1 or nlaunch <= 0:  # FP32 links (PREC_F32) only
        return None
    try:
        per_site = float(traffic["links_clover_bytes_per_site"])
        per_site_rhs = float(traffic["spinor_bytes_per_site_rhs"])
    except (KeyError, TypeError, ValueError):
        return None
    return int(vol * per_site + units / nlaunch * per_site_rhs)


def stencil_source_hash():
    """Hash of the FP32 stencil's sources (kernel header and shared helpers)."""
    h = hashlib.sha256()
    for f in ("bri_kernel.cuh", "bri_c2.cuh", "hops.cuh", "stencil.cuh", "cplx.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1701_00726_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.proc = None
        self.out = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")
        try:
            self.fh = open(self.out, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.out):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.out)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def oracle_sample(dims, n, tol, nrhs=1):
    """Time the FP64 oracle's D_ov on a small lattice (same generator, same
    solver settings); returns (seconds, site count)."""
    import synthetic_fields as sf
    from oracle import dirac, overlap
    u = sf.gauge_field(dims, GAUGE_SEED, 0.1, 3)
    x = sf.gaussian_source(dims, nrhs, GAUGE_SEED + 1000)
    t0 = time.perf_counter()
    kern = dirac.DiracOperator(u, "bri", m0=-RHO, c_sw=C_SW)
    overlap.overlap_apply(kern, x, RHO, n, tol)
    return time.perf_counter() - t0, dims[0] * dims[1] * dims[2] * dims[3] * nrhs


def _oracle_task(dims):
    return oracle_sample(tuple(dims), KL_ORDER, TOL)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The FP64 oracle on every host core: one single-threaded oracle D_ov per
    worker process, the workers started with 'spawn' (never forked from a
    process that holds a CUDA context)."""

    def __init__(self, cores):
        import multiprocessing as mp
        self.cores = cores
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        self.pool = mp.get_context("spawn").Pool(cores)
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        self.pool.map(int, range(cores))  # workers up before any timing

    def step(self, dims):
        """One oracle D_ov on the lattice dims per core, concurrently; (wall seconds, applications)."""
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_task, [dims] * self.cores)
        return time.perf_counter() - t0, len(res)

    def close(self):
        self.pool.close()
        self.pool.join()


def sample_fraction(dims):
    """One application on the lattice dims as a fraction of one 24^3x48 application (by volume)."""
    vs = dims[0] * dims[1] * dims[2] * dims[3]
    return vs / float(DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3])


def cpu_baseline_measure():
    """cpu_baseline: the oracle on all host cores (one concurrent round) and on one core."""
    cores = host_cores()
    dt1, _ = oracle_sample(CPU_SAMPLE, KL_ORDER, TOL)
    pool = OraclePool(cores)
    try:
        dtn, napp = pool.step(CPU_SAMPLE)
    finally:
        pool.close()
    frac = sample_fraction(CPU_SAMPLE)
    return {"value": napp * frac / dtn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "one_core": {"value": frac / dt1, "cores": 1, "seconds": round(dt1, 2)},
            "sample": (f"FP64 numpy oracle, one D_ov (KL order {KL_ORDER}, tol {TOL:g}, c_SW {C_SW:g}, stout field) on "
                       f"{'x'.join(map(str, CPU_SAMPLE))} per process, {cores} processes at once ({dtn:.1f} s) and "
                       f"one alone ({dt1:.1f} s); applications scaled by volume to 24^3x48")}


def workload_config(nrhs, world, inner):
    """The `config` of both arms' JSON lines (the same workload; `inner` names the arithmetic)."""
    return {"workload": f"24^3x48 massless overlap apply, {nrhs} rhs per step, stout 3x0.1, c_SW=1, "
                        f"rho=1, KL order {KL_ORDER}, final true residual {TOL:g} per shift",
            "lattice": list(DIMS), "nrhs": nrhs, "kl_order": KL_ORDER, "tol": TOL, "inner": inner,
            "l2": "inputs larger than L2 (links 1.9 GB FP32)", "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The oracle as the reference arm: each step is one concurrent round of
    oracle D_ov applications on CPU_SAMPLE, one per host core."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = host_cores()
    pool = OraclePool(cores)
    try:
        for _ in range(args.warmup):
            pool.step(REF_SAMPLE)
        t = 0.0
        napp = 0
        for _ in range(args.steps):
            dt, k = pool.step(REF_SAMPLE)
            t += dt
            napp += k
    finally:
        pool.close()
    value = napp * sample_fraction(REF_SAMPLE) / t  # 24^3x48-equivalent D_ov applications per second
    desc = (f"FP64 numpy oracle: per step one D_ov (KL order {KL_ORDER}, tol {TOL:g}, c_SW {C_SW:g}, stout field) "
            f"on {'x'.join(map(str, REF_SAMPLE))} in each of {cores} processes at once; applications scaled by "
            f"volume to 24^3x48")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.nrhs, world, "fp64 numpy oracle on the host cores (volume-scaled sample)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def batch_c4(args):
    import torch

    import synthetic_fields as sf
    from paper_1701_00726_gb300 import PREC_F32, Lattice, overlap_apply_batch
    shapes = [(16, 16, 16, 32), (8, 8, 8, 8), (8, 8, 8, 16), (12, 12, 12, 24), (16, 16, 16, 16), (12, 12, 12, 12),
              (12, 12, 12, 12), (8, 8, 8, 24), (8, 8, 8, 24)]
    lats, xs = [], []
    for i, dims in enumerate(shapes):
        lat = Lattice(dims)
        lat.build_links(torch.from_numpy(sf.gauge_field(dims, 10 + i, 0.1, 3, device="cuda")).cuda(), C_SW)
        lats.append(lat)
        src = sf.point_sources(dims) if i == 0 else sf.gaussian_source(dims, 1, 1010 + i)
        xs.append(torch.from_numpy(src).cuda())
    applies = sum(x.shape[0] for x in xs)
    for _ in range(max(1, args.warmup)):
        overlap_apply_batch(lats, xs, n=12, tol=TOL, prec=PREC_F32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        overlap_apply_batch(lats, xs, n=12, tol=TOL, prec=PREC_F32)
    torch.cuda.synchronize()
    tb = (time.perf_counter() - t0) / args.steps
    t0 = time.perf_counter()
    for lat, x in zip(lats, xs):
        lat.overlap_apply(x, n=12, tol=TOL, prec=PREC_F32)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    print(json.dumps({"workload": "batched overlap: 12 point sources on 16^3x32 + 8 lattices (8^4, 8^3x16, "
                                  "12^3x24, 16^4, 2x12^4, 2x8^3x24), KL order 12, mixed, tol 1e-10",
                      "applies_per_step": applies, "batch_s_per_step": tb, "sequential_s_per_step": ts,
                      "batch_applies_per_s": applies / tb, "speedup_vs_sequential": ts / tb}), flush=True)


def c2_solve(args):
    """FP64 massive overlap solves (complete form) with cascaded preconditioning on 16^3x32."""
    import torch

    import synthetic_fields as sf
    from paper_1701_00726_gb300 import PREC_F64, Lattice
    dims = (16, 16, 16, 32)
    u = sf.gauge_field(dims, GAUGE_SEED, 0.1, 3, device="cuda")
    b = torch.from_numpy(sf.gaussian_source(dims, 1, GAUGE_SEED + 1000)).cuda()
    lat = Lattice(dims)
    lat.build_links(torch.from_numpy(u).cuda(), C_SW)
    del u
    rows = []
    for kernel in ("bri", "wil"):
        lat.set_kernel(kernel)
        for am in (float(v) for v in args.c2_masses.split(",")):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = lat.overlap_solve(b, 16, 4, rho=RHO, am=am, complete=True, tol=args.c2_tol, prec=PREC_F64)
            torch.cuda.synchronize()
            rows.append({"kernel": kernel, "am": am, "seconds": round(time.perf_counter() - t0, 3),
                         "outer_iterations": st["iterations"], "inner_iterations": st["refinements"],
                         "kernel_matvecs": st["matvecs"], "true_residual": st["max_true_residual"],
                         "converged": st["converged"]})
            print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"workload": "FP64 16^3x32 massive overlap solve, complete form, KL order 16 with cascade "
                                  f"order 4, stout 3x0.1, c_SW=1, rho=1, outer tol {args.c2_tol:g}, FGMRES outer",
                      "results": rows}), flush=True)


def c5_grad(args):
    """Mixed-precision backward of L = Re<eta, D_ov psi> on 32^3x64 (KL order 12), next to its forward."""
    import torch

    import synthetic_fields as sf
    from paper_1701_00726_gb300 import PREC_F32, Lattice
    dims = (32, 32, 32, 64)
    u = sf.gauge_field(dims, 3, device="cuda")
    eta = torch.from_numpy(sf.gaussian_source(dims, 1, 1003, normalize=True)).cuda()
    psi = torch.from_numpy(sf.gaussian_source(dims, 1, 2003, normalize=True)).cuda()
    lat = Lattice(dims)
    lat.build_links(torch.from_numpy(u).cuda(), 0.0)
    del u
    lat.overlap_apply(psi, 12, rho=RHO, tol=TOL, prec=PREC_F32)  # warm-up (autotuner, pool)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, stf = lat.overlap_apply(psi, 12, rho=RHO, tol=TOL, prec=PREC_F32)
    torch.cuda.synchronize()
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, _, stb = lat.overlap_grad(eta, psi, 12, rho=RHO, tol=TOL, prec=PREC_F32)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    print(json.dumps({"workload": "gradient of Re<eta, D_ov psi> on 32^3x64, KL order 12, mixed precision, tol 1e-10, "
                                  "c_SW=0, w.r.t. psi and the thin links",
                      "forward_seconds": round(tf, 3), "backward_seconds": round(tb, 3),
                      "backward_over_forward": round(tb / tf, 3), "forward_iterations": stf["iterations"],
                      "backward_iterations": stb["iterations"], "backward_converged": stb["converged"],
                      "backward_phase_seconds": {"solves": round(stb["phase_seconds"][0], 3),
                                                 "dx_and_rationals": round(stb["phase_seconds"][1], 3),
                                                 "forces": round(stb["phase_seconds"][2], 3),
                                                 "link_backprop": round(stb["phase_seconds"][3], 3)},
                      "device_GB_in_use_after": round((lambda fr: (fr[1] - fr[0]) / 1e9)(torch.cuda.mem_get_info()), 2)}),
          flush=True)


def main():
    args = parse()
    if args.c2:
        c2_solve(args)
        return
    if args.c5_grad:
        c5_grad(args)
        return
    if args.batch_c4:
        batch_c4(args)
        return
    if args.stencil_probe:
        stencil_probe(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    import synthetic_fields as sf
    from paper_1701_00726_gb300 import PREC_F32, PREC_F32_BF16, PREC_F64, Lattice

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = PREC_F32_BF16 if args.links == "bf16" else PREC_F32
    nrhs = args.nrhs
    vol = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]

    u = sf.gauge_field(DIMS, GAUGE_SEED + rank, 0.1, 3, device="cuda")
    x_host = sf.gaussian_source(DIMS, nrhs, GAUGE_SEED + 1000 + rank)
    lat = Lattice(DIMS)
    lat.build_links(torch.from_numpy(u).cuda(), C_SW)
    del u
    x = torch.from_numpy(x_host).cuda()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    stats = []
    for _ in range(args.warmup):
        _, st = lat.overlap_apply(x, n=KL_ORDER, rho=RHO, tol=TOL, prec=prec, out=y)
    barrier()
    lat.profile(True)
    lat.profile_read(0, prec)
    launches0 = Lattice.kernel_launches()
    clocks = ClockSampler(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        _, st = lat.overlap_apply(x, n=KL_ORDER, rho=RHO, tol=TOL, prec=prec, out=y)
        stats.append(st)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = Lattice.kernel_launches() - launches0
    nlaunch, kms, units = lat.profile_read(0, prec)
    lat.profile(False)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    if world > 1:
        t = torch.tensor([elapsed], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed = float(t.item())
    applies = args.steps * nrhs * world
    value = applies / elapsed

    # roofline of the dominant kernel (the FP32 Brillouin stencil): the
    # attainable time of its launches is max(bytes / HBM peak, flops / FP32
    # FMA peak) with algorithmic bytes and flops; the larger term names the
    # bound.  Both peaks are measured on this GPU (copy bandwidth from
    # MEASURED_PEAKS.json, FMA rate by the library's probe kernel).
    from paper_1701_00726_gb300 import _lib
    peak, peak_src = measured_peak()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_scalar, _ = _lib.fma_probe(1, stream.cuda_stream)
    fp32_paired, _ = _lib.fma_probe(2, stream.cuda_stream)
    fp64_peak, _ = _lib.fma_probe(0, stream.cuda_stream)
    fp32_peak = max(fp32_scalar, fp32_paired)
    clock_mhz = (clk or {}).get("sm_mhz") or 2070.0
    alg_bytes = nlaunch * vol * (LINK_BYTES[prec] + CLOVER_BYTES) + units * SPINOR_BYTES
    alg_flops = units * FLOPS_PER_SITE
    ksec = kms / 1e3
    t_hbm = alg_bytes / (peak * 1e9)
    t_alu = alg_flops / (fp32_peak * 1e12)
    traffic = stencil_traffic()
    lt = "bf16x2" if prec == PREC_F32_BF16 else "float2"
    common = {"kernel": f"bri_kernel<float,{lt},1|2> | bri_kernel_c2<{lt}> | bri_kernel_c2x2<{lt}> (autotuned per rhs count)",
              "launches": nlaunch, "avg_launch_ms": round(kms / max(nlaunch, 1), 4),
              "avg_rhs_per_launch": round(units / max(nlaunch, 1) / vol, 3),
              "alg_bytes_per_launch": int(alg_bytes / max(nlaunch, 1)),
              "alg_flops_per_launch": int(alg_flops / max(nlaunch, 1)),
              "stencil_share_of_step": round(ksec / elapsed, 4) if world == 1 else None,
              "traffic": stencil_traffic_per_launch(traffic, vol, nlaunch, units, prec)}
    probe_src = (f"measured: bri_fma_probe on {sms} SMs (FP32 FMA {fp32_scalar:.1f}, paired FP32 FMA "
                 f"{fp32_paired:.1f} TFLOP/s; nominal {sms} x 128 lanes x 2 x {clock_mhz:.0f} MHz = "
                 f"{sms * 128 * 2 * clock_mhz / 1e6:.1f})")
    if t_alu >= t_hbm:
        achieved = alg_flops / ksec / 1e12 if ksec > 0 else 0.0
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak, 4), "peak_source": probe_src,
                "hbm_GBps_alg": round(alg_bytes / ksec / 1e9, 1) if ksec > 0 else 0.0}
    else:
        achieved = alg_bytes / ksec / 1e9 if ksec > 0 else 0.0
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "alu_TFLOPs_alg": round(alg_flops / ksec / 1e12, 2) if ksec > 0 else 0.0}
    roof.update(common)

    # end to end through the same C ABI call with host buffers (pinned), both
    # copies inside the timed region
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x_host).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        e_steps = max(1, min(args.steps, 5))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            xd = xh.to("cuda", non_blocking=True)
            yd, _ = lat.overlap_apply(xd, n=KL_ORDER, rho=RHO, tol=TOL, prec=prec)
            yh.copy_(yd, non_blocking=True)
            torch.cuda.synchronize()
        barrier()
        te = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([te], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            te = float(t.item())
        e2e = {"value": e_steps * nrhs * world / te, "unit": UNIT, "steps": e_steps,
               "h2d_bytes_per_step": int(xh.numel() * 16), "d2h_bytes_per_step": int(yh.numel() * 16)}

    extras = {}
    if rank == 0 and not args.no_extras:
        # (1) the timed step's accuracy: an untimed repeat with FP64 true residuals
        # of every shift; the solver is deterministic, so its output must equal the
        # timed output bit for bit, and the residuals are those of the timed step
        y_chk, st_chk = lat.overlap_apply(x, n=KL_ORDER, rho=RHO, tol=TOL, prec=prec, want_true_residual=True)
        extras["accuracy"] = {"max_true_residual": st_chk["max_true_residual"], "tol": TOL,
                              "shift_residual_max": max(st_chk["shift_residual"]),
                              "repeat_bitwise_equal_to_timed": bool(torch.equal(y_chk, y))}
        del y_chk
        # (2) the single-rhs stencil against its rooflines (CUDA events, 20 launches)
        x1 = x[:1].to(torch.complex64).contiguous()
        y1 = torch.empty_like(x1)

        def stencil_ms(xx, yy, bf16, dw=False):
            lat.bri_apply(xx, -RHO, bf16_links=bf16, out=yy, double_word=dw)
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ea.record(stream)
            for _ in range(20):
                lat.bri_apply(xx, -RHO, bf16_links=bf16, out=yy, double_word=dw)
            eb.record(stream)
            torch.cuda.synchronize()
            return ea.elapsed_time(eb) / 20

        one = {}
        for name, bf16, lb in (("fp32_links", False, LINK_BYTES[1]), ("bf16_links", True, LINK_BYTES[2])):
            ms = stencil_ms(x1, y1, bf16)
            byt = vol * (lb + CLOVER_BYTES + SPINOR_BYTES)
            one[name] = {"ms": round(ms, 4), "alg_bytes": byt, "alg_GBps": round(byt / ms / 1e6, 1),
                         "hbm_frac": round(byt / ms / 1e6 / peak, 4),
                         "alu_frac": round(vol * FLOPS_PER_SITE / ms / 1e9 / fp32_peak, 4)}
        one["hbm_peak_GBps"] = peak
        one["hbm_peak_source"] = peak_src
        x64 = x[:1].contiguous()
        y64 = torch.empty_like(x64)
        ms64 = stencil_ms(x64, y64, False)
        one["fp64"] = {"ms": round(ms64, 3), "alg_TFLOPs": round(vol * FLOPS_PER_SITE / ms64 / 1e9, 3),
                       "fp64_peak_TFLOPs": round(fp64_peak, 3),
                       "alu_frac": round(vol * FLOPS_PER_SITE / ms64 / 1e9 / fp64_peak, 4),
                       "alg_GBps": round(vol * (F64_LINK_CLOVER_BYTES + F64_SPINOR_BYTES) / ms64 / 1e6, 1)}
        # the double-word FP32 operator that serves the FP64-class residuals
        ydw = torch.empty_like(x64)
        msdw = stencil_ms(x64, ydw, False, dw=True)
        one["double_word"] = {"ms": round(msdw, 3), "speedup_vs_fp64": round(ms64 / msdw, 2),
                              "max_rel_diff_vs_fp64": float((ydw - y64).abs().max() / y64.abs().max()),
                              "note": "includes the FP64 -> double-word split and join of the vectors"}
        del ydw
        extras["bri_apply_1rhs"] = one
        extras["fma_peaks_TFLOPs"] = {"fp64": round(fp64_peak, 3), "fp32": round(fp32_scalar, 2),
                                      "fp32_paired": round(fp32_paired, 2), "sms": sms}
        del x1, y1, x64, y64
        # (3) the plain FP64 GPU solve (one rhs) and the mixed-over-FP64 ratio
        if not args.no_fp64:
            xs = x[:1].contiguous()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st64 = lat.overlap_apply(xs, n=KL_ORDER, rho=RHO, tol=TOL, prec=PREC_F64)
            torch.cuda.synchronize()
            t64 = time.perf_counter() - t0
            extras["fp64_gpu"] = {"applies_per_s": 1.0 / t64, "seconds_per_apply": round(t64, 3), "rhs": 1,
                                  "iterations": st64["iterations"], "converged": st64["converged"],
                                  "mixed_over_fp64": round(value / world / (1.0 / t64), 3)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_measure()

    if rank == 0:
        last = stats[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(nrhs, world, "fp32 spinors, " + ("bf16" if prec == PREC_F32_BF16 else "fp32") +
                                      " links, fp64 reductions, fp64 refinement"),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "solver": {"iterations": last["iterations"], "matvecs": last["matvecs"],
                       "matvecs_f64": last["matvecs_f64"], "refinements": last["refinements"],
                       "phase_seconds": [round(v, 4) for v in last["phase_seconds"]]},
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
