#!/usr/bin/env python
"""Benchmark of the LRI space-time RPA path on GB300.

One step = one RPA correlation energy of the graphene-slab workload (35 atoms:
a 4x4 graphene supercell plus a water-shaped molecule, N_aux = 2010, 4x4x1
k-mesh, 16 tau/omega points, FP64): G(R, tau) -> chi0(R, tau) -> chi0(q, i omega)
-> ln det -> E_c, every step through the library's C ABI.

Prints one JSON line.  ``value`` = RPA energies/s of the whole job with inputs
resident in HBM; ``e2e`` = the same with the inputs pushed from host buffers
through the C ABI and E_c read back inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gpu,reference}]

Under torchrun (N > 1) every rank computes its own energy (independent
requests, no collective on the data path): weak scaling, value = all ranks'
energies / the slowest rank's time.  ``--impl reference`` times the CPU oracle
(chi0 from the matrix form of Sec. 2 in plain C, OpenMP) on a bounded sample of the same
workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RPA energies/s"
UNIT = "energies/s"
WORKLOAD_CUBIC = "cubic cell: 2 atoms, 8 NAO / 24 ABF each, N_aux 48, 2x2x2 k-mesh, %d tau/omega points"
WORKLOAD = ("graphene 4x4 supercell + H2O-shaped molecule: 35 atoms, n_ao 431, N_aux 2010, "
            "4x4x1 k-mesh, 16 tau/omega points")

# nominal FP64/BF16 ratio of GB300 (1.25 TFLOP/s / 2250 TFLOP/s): the FP64 peak derived from the
# measured BF16 peak, reported next to the FP64 peaks this benchmark measures itself
NOMINAL_FP64_OVER_BF16 = 1.25 / 2250.0

# precision presets of the library (include/librpa_gpu.h): name -> (LIBRPA_* value, dtype label)
PRECISIONS = {"fp64": (0, "f64"), "fp64_tc": (1, "f64-accurate: bf16 digit planes (5) on tcgen05"),
              "split": (2, "mixed: chi0 GEMMs on 3 bf16 digit planes, ln det on 5"),
              "bf16": (3, "mixed: chi0 GEMMs in plain bf16 (fp32 accumulation), ln det on 5 digit planes"),
              "tf32": (4, "mixed: chi0 GEMMs in plain tf32 (fp32 accumulation), ln det on 5 digit planes"),
              "tf32x3": (5, "mixed: chi0 GEMMs as 3xtf32 split products (fp32 accumulation), ln det on 5 digit planes"),
              "split_fast": (6, "mixed: chi0 GEMMs on 3 bf16 digit planes, ln det on 4, transforms in fp32")}
MEV_PER_HA = 27211.386245988

# DRAM traffic per launch of the dominant kernels from one ncu capture (see profiles/), valid only
# while the kernel's source text is unchanged (sha256 of the text between the markers at capture time).
TRAFFIC = {
    # Gamma case of the graphene slab, one (R, tau) point per launch as at 4x4x1: N/X group 0.681 GB,
    # final contraction 1.225 GB, averaged (profiles/k_dgemm_nt_dram_graphene_gamma.md)
    "k_dgemm_nt": {"bytes_per_launch": 0.953e9, "src": "paper_2407_19930_gb300/csrc/k_chi0.cu",
                   "begin": "template <int WM, int WN>", "end": "// tile variants {WM, WN}", "src_sha": "431079ebc2084c1e"},
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _src_sha(path, begin=None, end=None):
    """sha256 (16 hex digits) of a source file, or of its text from `begin` up to `end`."""
    with open(os.path.join(ROOT, path), "rb") as f:
        b = f.read()
    if begin:
        i = b.index(begin.encode())
        b = b[i:b.index(end.encode(), i)]
    return hashlib.sha256(b).hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                if self.uuid and parts[0] != self.uuid:
                    continue
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ peaks measured in the run


def measure_fp64_peaks(device):
    """FP64 and TF32 peaks of this GPU, measured now: the DFMA pipe and the FP64 tensor path
    (mma.sync m8n8k4, the instruction of the FP64 chi0 GEMM) by the register-only probes of
    probe/peaks.cu, a cuBLAS DGEMM and a cuBLAS TF32 GEMM (8192^3, torch.matmul), each timed with
    CUDA events after a warm-up, with the SM clock sampled meanwhile."""
    import ctypes
    import torch
    from paper_2407_19930_gb300 import build as lbuild
    lib = ctypes.CDLL(lbuild.PROBE_LIB)
    lib.librpa_probe_fp64.restype = ctypes.c_int
    out = {}
    clocks = ClockSampler()
    clocks.start()
    for name, kind, iters in (("dfma", 0, 200000), ("dmma_m8n8k4", 1, 100000)):
        tf, ms = ctypes.c_double(), ctypes.c_double()
        rc = lib.librpa_probe_fp64(kind, iters, 8, ctypes.byref(tf), ctypes.byref(ms))
        out[name] = {"tflops": tf.value, "ms": ms.value} if rc == 0 else {"error": rc}
    n = 8192

    def gemm(dtype, tf32):
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        try:
            a = torch.randn(n, n, dtype=dtype, device=device)
            b = torch.randn(n, n, dtype=dtype, device=device)
            c = a @ b
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            reps = 3 if dtype == torch.float64 else 20
            e0.record()
            for _ in range(reps):
                c = a @ b
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            del a, b, c
            return {"tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12, "ms": ms}
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev

    out["cublas_dgemm"] = gemm(torch.float64, False)
    out["cublas_tf32"] = gemm(torch.float32, True)
    out["clocks"] = clocks.stop()
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ CPU oracle sample


def cpu_model():
    """nproc and the CPU model name of this host (lscpu, else /proc/cpuinfo)."""
    name = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().startswith("Model name:"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        name = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "model": name}



def cpu_sample(inp, grid, budget_s=25.0):
    """Time the oracle (chi0 by the matrix form in plain C with OpenMP, numpy LU) on a bounded
    sample of the workload and extrapolate to one RPA energy."""
    import numpy as np
    from oracle import energy, green
    from oracle.chi0_matrix import chi0_matrix_form
    st = inp.st
    ntau = len(grid["tau"])
    t0 = time.perf_counter()
    go, gv = green.green(st.kmesh, inp.kfrac, inp.eig, inp.occ, inp.wfc, inp.efermi, grid["tau"][:1])
    t_green = (time.perf_counter() - t0) * ntau
    pts = []
    t_pt = []
    deadline = time.perf_counter() + budget_s
    for p in [(0, 0), (5, 0), (10, 0)]:
        t0 = time.perf_counter()
        chi0_matrix_form(st, inp.lri, go, gv, [p])
        t_pt.append(time.perf_counter() - t0)
        pts.append(p)
        if time.perf_counter() > deadline:
            break
    n = st.naux
    rng = np.random.default_rng(0)
    x = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * 1e-3
    chi = -(x @ x.conj().T)
    t0 = time.perf_counter()
    energy.integrand_lu(chi, inp.vq[0])
    t_lu = time.perf_counter() - t0
    tp = statistics.median(t_pt)
    npts = ntau * st.nk
    t_energy = npts * tp + st.nk * ntau * t_lu + t_green
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"t_energy_s": t_energy, "t_point_s": tp, "t_lu_s": t_lu, "t_green_s": t_green, "cores": cores,
            "t_sample_s": sum(t_pt) + t_lu + t_green / ntau,
            "sample": "chi0(R,tau) by the oracle's matrix form on %d of %d (R,tau) points, ln det by LU on 1 of %d (q,omega), "
                      "G on 1 of %d tau; extrapolated to one energy" % (len(pts), npts, st.nk * ntau, ntau)}


def oracle_full_energy(inp, grid):
    """Seconds of one whole RPA energy by the oracle (G, chi0 at every (R, tau) point, the
    transforms, LU of every (q, omega)); returns (seconds, E_c)."""
    from oracle import pipeline
    t0 = time.perf_counter()
    out = pipeline.rpa_energy(inp, grid)
    return time.perf_counter() - t0, out["ec"]


# ------------------------------------------------------------------ arms


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (x itself on one rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world_size, t_max):
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return units_per_rank * world_size / t_max


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The oracle as the reference arm.  Each step is a bounded sample of one energy of the
    workload (chi0 at one (R, tau) point, one LU of a (q, omega) matrix, G at one tau);
    ms_per_step is the measured wall time of that sample, and value is one energy's time
    extrapolated from the sample (stated in the "extrapolated" key).  With --full NAME the whole
    energy of a workload runs instead, median of --steps runs plus one single-thread run."""
    ws, rank, local = dist_init()
    if rank != 0:
        return 0
    from paper_2407_19930_gb300 import synthetic as syn
    from oracle import build as obuild, grid as ogrid
    obuild.build()
    if args.full:
        return run_reference_full(args)
    inp = syn.config_graphene()
    grid = ogrid.make_grid(16, *inp.delta_range)
    per = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        s = cpu_sample(inp, grid, budget_s=0.0)
        s["wall_s"] = time.perf_counter() - t0
        if i >= args.warmup:
            per.append(s)
    t = statistics.median([s["t_energy_s"] for s in per])
    v = 1.0 / t
    ms_step = statistics.median([s["wall_s"] for s in per]) * 1e3
    cpu = cpu_model()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "extrapolated": {"value_from": "per-step sample times scaled to one energy: %d (R,tau) points x "
                                          "median point time + %d LUs x LU time + G" % (16 * 16, 16 * 16),
                             "s_per_energy": t, "ms_per_step_is": "measured wall time of one sample step",
                             "t_point_s": statistics.median([s["t_point_s"] for s in per]),
                             "t_lu_s": statistics.median([s["t_lu_s"] for s in per])},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": per[0]["cores"], "kind": "oracle",
                             "sample": per[0]["sample"], "nproc": cpu["nproc"], "cpu_model": cpu["model"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_full(args):
    """Whole energies by the oracle on the host cores: median of --steps runs with every core,
    and one run with a single OpenMP thread (a child process, the thread count being fixed when
    the OpenMP runtime starts)."""
    from paper_2407_19930_gb300 import synthetic as syn
    from oracle import grid as ogrid
    if args.full == "cubic":
        inp, ntau, name = syn.config_cubic(), 8, ("cubic cell: 2 atoms, 8 NAO / 24 ABF each, 2x2x2 k-mesh, "
                                                  "8 tau/omega points")
    else:
        inp, ntau, name = syn.config_graphene(), 16, WORKLOAD
    grid = ogrid.make_grid(ntau, *inp.delta_range)
    if args.single_thread_child:
        t, ec = oracle_full_energy(inp, grid)
        print(json.dumps({"t": t, "ec": ec}), flush=True)
        return 0
    times, ecs = [], []
    for _ in range(args.steps):
        t, ec = oracle_full_energy(inp, grid)
        times.append(t)
        ecs.append(ec)
    single = None
    if args.single_thread:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--impl", "reference", "--full", args.full,
                            "--single-thread-child"], capture_output=True, text=True, env=env)
        if r.returncode == 0:
            single = json.loads(r.stdout.strip().splitlines()[-1])
    t = statistics.median(times)
    cpu = cpu_model()
    line = {"impl": "reference", "metric": METRIC, "value": 1.0 / t, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": 0, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "none",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": name},
            "cpu_baseline": {"value": 1.0 / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "whole energies, median of %d runs" % len(times),
                             "nproc": cpu["nproc"], "cpu_model": cpu["model"], "runs_s": times,
                             "single_thread_s": single["t"] if single else None},
            "ec_ha": ecs[0]}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch
    ws, rank, local = dist_init()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(local)
    from paper_2407_19930_gb300 import build as lbuild
    from paper_2407_19930_gb300 import librpa_gpu as L
    from paper_2407_19930_gb300 import synthetic as syn
    if rank == 0:
        lbuild.build()
    if dist:
        dist.barrier()
    L.load(build_if_missing=False)
    inp = syn.config_cubic() if args.workload == "cubic" else syn.config_graphene(kmesh=args.kmesh)
    st = inp.st
    stream = torch.cuda.Stream(device=local)
    o = L.librpa_gpu_default_opts()
    o.device = local
    o.n_tau = args.ntau
    o.precision = PRECISIONS[args.precision][0]
    h = L.librpa_gpu_create(o, torch_stream=stream, torch_alloc=True)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    peaks_run = None
    if not args.no_peaks:
        peaks_run = measure_fp64_peaks(torch.device("cuda", local))
    try:
        L.set_inputs(h, inp)
        for _ in range(args.warmup):
            L.librpa_gpu_chi0(h)
            L.librpa_gpu_ec(h)
        # ---------------- device-resident timing
        uuid = None
        try:
            uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
        except Exception:
            pass
        clocks = ClockSampler(uuid)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        clocks.start()
        ev0.record(stream)
        for _ in range(args.steps):
            L.librpa_gpu_chi0(h)
            ec, _, _ = L.librpa_gpu_ec(h)
        ev1.record(stream)
        barrier()
        clk = clocks.stop()
        # counters of the last step (every step launches the same kernels), read after the timed region
        stats = [L.librpa_gpu_get_stats(h)]
        grid_used = L.librpa_gpu_get_grid(h)
        launches = stats[-1]["launches"] * args.steps
        t = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dist, "cuda")
        value = job_value(args.steps, ws, t)
        # ---------------- end to end through host buffers
        h2d = sum(C.nbytes for *_, C in inp.lri) + st.nk * (inp.wfc[0].real.nbytes * 2 + inp.eig[0].nbytes * 2) \
            + st.nk * inp.vq[0].real.nbytes * 2
        d2h = 8
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for I, K, R, C in inp.lri:
                L.librpa_gpu_set_lri_coeffs(h, I, K, R, C)
            for ik in range(st.nk):
                L.librpa_gpu_set_green(h, 0, ik, inp.eig[ik], inp.occ[ik], inp.wfc[ik], inp.efermi)
            for iq in range(st.nk):
                L.librpa_gpu_set_coulomb(h, iq, inp.vq[iq])
            L.librpa_gpu_chi0(h)
            ec_e2e, _, _ = L.librpa_gpu_ec(h)
        barrier()
        te = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e = job_value(args.e2e_steps, ws, te) if args.e2e_steps else 0.0
    finally:
        L.librpa_gpu_destroy(h)
    # ---------------- the other precision modes on the same workload (1 GPU only)
    modes = {}
    if ws == 1:
        for m in [x for x in args.modes.split(",") if x and x != args.precision]:
            modes[m] = time_mode(L, inp, stream, local, args.ntau, m, ec, torch)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    s = stats[-1]
    peaks, src = _peaks()
    fp64_derived = peaks["bf16_tflops"] * NOMINAL_FP64_OVER_BF16
    # the FP64 kernels' roofline: the FP64 tensor-path peak measured in this run (the same
    # mma.sync m8n8k4 instruction as k_dgemm_nt; the derived value when the probes were skipped)
    dmma = (peaks_run or {}).get("dmma_m8n8k4", {}).get("tflops")
    fp64_peak = dmma if dmma else fp64_derived
    fp64_src = ("measured in this run: DMMA m8n8k4 register probe (probe/peaks.cu), SM clock median %s MHz"
                % ((peaks_run.get("clocks") or {}).get("sm_mhz") if peaks_run else None)) if dmma else \
        "derived: %s BF16 dense burst x nominal FP64/BF16 (1.25/2250)" % src
    # dominant kernel by device time within the step
    kern = {"k_dgemm_nt": (s["ms_gemm_chi0"], s["flop_gemm_chi0"], s["n_gemm_chi0"], "paper_2407_19930_gb300/csrc/k_chi0.cu"),
            "k_zgemm": (s["ms_gemm_ec"], s["flop_gemm_ec"], s["n_gemm_ec"], "paper_2407_19930_gb300/csrc/k_zgemm.cu")}
    name = max(kern, key=lambda k: kern[k][0])
    ms, fl, nl, srcf = kern[name]
    achieved = fl / (ms * 1e-3) / 1e12 if ms > 0 else None
    tr = TRAFFIC.get(name)
    # the captured traffic is the graphene slab's (its per-launch work is the same at every k-mesh)
    traffic = tr["bytes_per_launch"] if (tr and args.workload == "graphene" and
                                         tr["src_sha"] == _src_sha(tr["src"], tr["begin"], tr["end"])) else None
    step_ms = t / args.steps * 1e3 * ws / ws
    chi0_tflops = s["flop_chi0"] / (s["ms_chi0"] * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": PRECISIONS[args.precision][1],
        "data": "synthetic (seeded tight-binding KS data, LRI coefficients and Coulomb matrices "
                "of the paper's graphene/H2O workload shape)",
        "config": {"workload": (WORKLOAD_CUBIC % args.ntau) if args.workload == "cubic" else
                   WORKLOAD if (args.kmesh, args.ntau) == ((4, 4, 1), 16) else
                   "profiling variant: graphene slab, %s k-mesh, %d tau" % ("x".join(map(str, st.kmesh)), args.ntau),
                   "atoms": st.natoms, "n_ao": st.nao, "n_aux": st.naux,
                   "kmesh": "x".join(map(str, st.kmesh)), "n_tau": args.ntau, "precision": args.precision,
                   "l2": "inputs larger than L2: chi0(R,tau) %.1f GB and G %.2f GB are streamed every step"
                         % (args.ntau * st.nk * st.naux ** 2 * 8 / 1e9, 2 * args.ntau * st.nk * st.nao ** 2 * 8 / 1e9)},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "chi0_tflops": chi0_tflops,
        "stage_ms": {"green": s["ms_green"], "chi0": s["ms_chi0"], "freq": s["ms_freq"], "ec": s["ms_ec"]},
        "ec_ha": ec,
        "roofline": {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak if achieved else None, "traffic": traffic,
                     "peak_note": "FP64 tensor path, %s; derived from the BF16 peak: %.3f" % (fp64_src, fp64_derived),
                     "launches": nl, "flop": fl},
        "clocks": clk,
    }
    if peaks_run:
        line["peaks_measured"] = peaks_run
    if args.precision != "fp64":
        line["roofline"] = tc_roofline(s, peaks, src)
    if modes:
        line["modes"] = modes
    if ws == 1 and args.serve_sample > 0:
        torch.cuda.empty_cache()   # the headline's blocks cached by torch go back to the device
        reqs = _serve_inputs(args.serve_sample)
        sweep = []
        for rate in [float(x) for x in args.serve_rates.split(",") if x]:
            m = serve_measure(L, reqs, rate, args.slots, args.ntau, local)
            sweep.append({"rate_req_per_s": rate, "value": m["value"], "unit": UNIT, "latency_ms": m["latency_ms"],
                          "completed": m["completed"], "failed": m["failed"], "peak_running": m["peak_running"],
                          "seconds": m["seconds"], "errors": m["errors"]})
        sizes = [inp.st.natoms for inp in reqs]
        line["serving"] = {"workload": "%d requests per arrival rate, Poisson arrivals, random cells of %d-%d atoms "
                                       "(5/9/13 NAO, 20/40/60 ABF), k-mesh 1x1x1..3x3x1, %d tau; precision per "
                                       "request alternating fp64_tc / split"
                                       % (len(reqs), min(sizes), max(sizes), args.ntau),
                           "slots": args.slots, "sweep": sweep}
    if ws == 1 and args.batch_sample > 0:
        torch.cuda.empty_cache()
        binp = _batch_inputs(args.batch_sample)
        bout, bclk = batch_measure(L, binp, args.ntau, 1, local, torch)
        line["batch"] = {"workload": _batch_workload(binp, args.ntau), "modes": bout, "clocks": bclk}
    if ws == 1 and not args.no_cpu and args.workload == "cubic":
        # the oracle's whole energy on the library's grid (a fraction of a second on the host cores)
        from oracle import build as obuild
        obuild.build()
        t_or, ec_or = oracle_full_energy(inp, grid_used)
        cpu = cpu_model()
        line["cpu_baseline"] = {"value": 1.0 / t_or, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": "the whole energy of the workload", "nproc": cpu["nproc"],
                                "cpu_model": cpu["model"], "ec_ha": ec_or,
                                "ec_gpu_minus_oracle_mev_per_atom": (ec - ec_or) * MEV_PER_HA / st.natoms}
        for m, v in modes.items():
            v["ec_diff_vs_oracle_mev_per_atom"] = abs(v["ec_ha"] - ec_or) * MEV_PER_HA / st.natoms
    elif ws == 1 and not args.no_cpu:
        from oracle import build as obuild, grid as ogrid
        obuild.build()
        cb = cpu_sample(inp, ogrid.make_grid(args.ntau, *inp.delta_range))
        cpu = cpu_model()
        line["cpu_baseline"] = {"value": 1.0 / cb["t_energy_s"], "unit": UNIT, "cores": cb["cores"],
                                "kind": "oracle", "sample": cb["sample"], "sample_s": cb["t_sample_s"],
                                "nproc": cpu["nproc"], "cpu_model": cpu["model"],
                                "chi0_tflops": s["flop_chi0"] / (args.ntau * st.nk) / cb["t_point_s"] / 1e12}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def tc_roofline(s, peaks, src):
    """Roofline of the dominant digit-plane GEMM (chi0 or ln det) against the BF16 tensor peak:
    achieved = MMA flops issued / device time of those launches (both from the library's stats)."""
    legs = {"k_ozgemm (chi0 GEMMs)": (s["ms_gemm_chi0"], s["flop_exec_gemm_chi0"], s["n_gemm_chi0"]),
            "k_ozgemm (ln det GEMMs)": (s["ms_gemm_ec"], s["flop_exec_gemm_ec"], s["n_gemm_ec"])}
    name = max(legs, key=lambda k: legs[k][0])
    ms, fl, nl = legs[name]
    if ms <= 0 or fl <= 0:
        return None
    peak = peaks["bf16_tflops"]
    achieved = fl / (ms * 1e-3) / 1e12
    return {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_note": "BF16 dense burst, %s; sustained %.1f; achieved counts the BF16 MMA flops issued "
                         "(all digit-plane products, tile padding included)" % (src, peaks.get("bf16_tflops_sustained", peak)),
            "launches": nl, "flop": fl}


def time_mode(L, inp, stream, device, ntau, mode, ec_ref, torch):
    """One warm-up and one timed step of `mode` on its own handle; E_c against the headline's.
    `mode` is a precision preset, optionally with a Green's-function screening threshold
    ("fp64@1e-3": the paper's production setting; its E_c difference is then the screening's)."""
    prec, _, thr = mode.partition("@")
    theta = float(thr) if thr else 0.0
    o = L.librpa_gpu_default_opts()
    o.device = device
    o.n_tau = ntau
    o.precision = PRECISIONS[prec][0]
    h = L.librpa_gpu_create(o, torch_stream=stream, torch_alloc=True)
    try:
        L.set_inputs(h, inp)
        if theta > 0:
            L.librpa_gpu_set_screening(h, theta)
        L.librpa_gpu_chi0(h)
        L.librpa_gpu_ec(h)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.librpa_gpu_chi0(h)
        ec, _, _ = L.librpa_gpu_ec(h)
        e1.record(stream)
        torch.cuda.synchronize()
        s = L.librpa_gpu_get_stats(h)
    finally:
        L.librpa_gpu_destroy(h)
    ms = e0.elapsed_time(e1)
    dmev = abs(ec - ec_ref) * MEV_PER_HA / inp.st.natoms
    peaks, src = _peaks()
    out = {"dtype": PRECISIONS[prec][1], "ms_per_step": ms, "value": 1e3 / ms, "unit": UNIT,
           "chi0_tflops_fp64_equiv": s["flop_chi0"] / (s["ms_chi0"] * 1e-3) / 1e12,
           "stage_ms": {"green": s["ms_green"], "chi0": s["ms_chi0"], "freq": s["ms_freq"], "ec": s["ms_ec"]},
           "ec_ha": ec, "ec_diff_vs_fp64_mev_per_atom": dmev, "within_0.1_mev_per_atom": dmev <= 0.1,
           "steps": 1, "warmup": 1}
    if prec != "fp64":
        out["roofline"] = tc_roofline(s, peaks, src)
    if theta > 0:
        out["screening"] = {"threshold": theta, "points_contracted": s["n_points_chi0"],
                            "points_skipped": s["n_points_skipped"],
                            "g_blocks_kept_frac": s["n_blocks_kept"] / max(1, s["n_blocks_total"]),
                            "chi0_flop_alg": s["flop_chi0"]}
    return out


def _serve_inputs(n):
    """The serving workload's requests, drawn in parallel (spawned workers)."""
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor
    from paper_2407_19930_gb300 import synthetic as syn
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                             mp_context=multiprocessing.get_context("spawn")) as ex:
        return list(ex.map(syn.config_request, range(n)))


def serve_measure(L, reqs_in, rate, slots, ntau, device):
    """Poisson arrivals of the requests into the library's serving loop; precision per request
    alternates between the FP64-accurate tensor-core mode and the mixed mode."""
    import numpy as np
    modes = ["fp64_tc", "split"]
    n = len(reqs_in)
    arrivals = np.cumsum(np.random.default_rng(4004).exponential(1.0 / rate, size=n))
    s = L.librpa_gpu_server_create(device=device, slots=slots)
    handles = []
    try:
        for i, inp in enumerate(reqs_in):
            o = L.librpa_gpu_default_opts()
            o.n_tau = ntau
            o.precision = PRECISIONS[modes[i % 2]][0]
            r = L.librpa_gpu_server_request(s, o)
            handles.append(r)
            L.set_inputs(r, inp)
        clocks = ClockSampler()
        clocks.start()
        t0 = time.perf_counter()
        tickets = []
        for i, r in enumerate(handles):
            d = arrivals[i] - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            tickets.append(L.librpa_gpu_server_submit(s, r))
        res = [L.librpa_gpu_server_wait(s, t, 1800.0) for t in tickets]
        t_all = time.perf_counter() - t0
        clk = clocks.stop()
        st = L.librpa_gpu_server_get_stats(s)
        errors = [{"request": i, "status": r["status"] if r else None,
                   "message": L.librpa_gpu_last_error(handles[i])}
                  for i, r in enumerate(res) if not r or r["status"] != 0]
    finally:
        L.librpa_gpu_server_destroy(s)
        for r in handles:
            L.librpa_gpu_destroy(r)
    sizes = [inp.st.natoms for inp in reqs_in]
    return {
        "value": st["energies_per_s"], "unit": UNIT, "seconds": t_all,
        "workload": "serving: %d requests, Poisson arrivals at %.1f req/s, random cells of %d-%d atoms "
                    "(5/9/13 NAO, 20/40/60 ABF), k-mesh 1x1x1..3x3x1, %d tau; precision per request alternating "
                    "fp64_tc / split" % (n, rate, min(sizes), max(sizes), ntau),
        "slots": slots, "hbm_budget_bytes": st["hbm_budget"],
        "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"], "mean_queue": st["mean_queue_ms"]},
        "completed": st["completed"], "failed": st["failed"], "peak_running": st["peak_running"],
        "peak_reserved_bytes": st["peak_reserved"], "errors": errors,
        "requests": [{"atoms": inp.st.natoms, "kmesh": "x".join(map(str, inp.st.kmesh)), "n_aux": inp.st.naux,
                      "mode": modes[i % 2], "status": r["status"] if r else None, "ec_ha": r["ec"] if r else None,
                      "ms_queue": r["ms_queue"] if r else None, "ms_run": r["ms_run"] if r else None,
                      "ms_total": r["ms_total"] if r else None, "slot": r["slot"] if r else None}
                     for i, (inp, r) in enumerate(zip(reqs_in, res))],
        "clocks": clk,
    }


def run_serve(args):
    """Serving workload: a Poisson stream of RPA energy requests (random cells of 2-64 atoms,
    mixed species, 1x1x1 to 3x3x1 k) into the library's serving loop."""
    ws, rank, local = dist_init()
    if ws > 1:
        print(json.dumps({"metric": METRIC, "unavailable": "the serving run is one process on one GPU"}))
        return 0
    reqs_in = _serve_inputs(args.serve_requests)
    import torch
    from paper_2407_19930_gb300 import build as lbuild
    from paper_2407_19930_gb300 import librpa_gpu as L
    torch.cuda.set_device(local)
    lbuild.build()
    L.load(build_if_missing=False)
    m = serve_measure(L, reqs_in, args.rate, args.slots, args.ntau, local)
    n = len(reqs_in)
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": 1, "steps": n, "warmup": 0,
        "ms_per_step": 1e3 * m["seconds"] / max(1, m["completed"]), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "per request: " + PRECISIONS["fp64_tc"][1] + "; " + PRECISIONS["split"][1],
        "data": "synthetic (seeded random cells, tight-binding KS data, LRI coefficients, Coulomb matrices)",
        "config": {"workload": m["workload"], "slots": m["slots"], "hbm_budget_bytes": m["hbm_budget_bytes"]},
        "latency_ms": m["latency_ms"], "completed": m["completed"], "failed": m["failed"],
        "peak_running": m["peak_running"], "peak_reserved_bytes": m["peak_reserved_bytes"],
        "requests": m["requests"], "clocks": m["clocks"],
    }
    print(json.dumps(line), flush=True)
    return 0 if m["completed"] == n else 1


def _batch_inputs(n):
    """The batched workload's structures, drawn in parallel (spawned workers, before any GPU use)."""
    import functools
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor
    from paper_2407_19930_gb300 import synthetic as syn
    f = functools.partial(syn.config_request, natoms_range=(2, 40), seed_base=3000)
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                             mp_context=multiprocessing.get_context("spawn")) as ex:
        return list(ex.map(f, range(n)))


def run_batch(args):
    """Batched workload: n independent structures (2-40 atoms, mixed species, 1x1x1 to 3x3x1 k) in
    one librpa_gpu_batch_run (merged chi0 launches, graph replay for FP64), against the same
    structures one by one through librpa_gpu_chi0 + librpa_gpu_ec."""
    ws, rank, local = dist_init()
    if ws > 1:
        print(json.dumps({"metric": METRIC, "unavailable": "the batched run is one process on one GPU"}))
        return 0
    inputs = _batch_inputs(args.batch_n)
    import torch
    from paper_2407_19930_gb300 import build as lbuild
    from paper_2407_19930_gb300 import librpa_gpu as L
    torch.cuda.set_device(local)
    lbuild.build()
    L.load(build_if_missing=False)
    out, clk = batch_measure(L, inputs, args.ntau, args.steps, local, torch)
    sizes = [inp.st.natoms for inp in inputs]
    line = {
        "metric": METRIC, "value": out["fp64"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": 1, "ms_per_step": out["fp64"]["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded random cells, tight-binding KS data, LRI coefficients, Coulomb matrices)",
        "config": {"workload": _batch_workload(inputs, args.ntau)},
        "modes": out, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def _batch_workload(inputs, ntau):
    sizes = [inp.st.natoms for inp in inputs]
    return ("batched: %d structures of %d-%d atoms (5/9/13 NAO, 20/40/60 ABF), k-mesh 1x1x1..3x3x1, %d tau, "
            "one batch run per step" % (len(inputs), min(sizes), max(sizes), ntau))


def batch_measure(L, inputs, ntau, steps, local, torch):
    """The structures in one librpa_gpu_batch_run per step (FP64 and the mixed mode; one run first to
    tune and capture) against the same structures one by one; returns (per-mode results, clocks)."""

    def opts(mode):
        o = L.librpa_gpu_default_opts()
        o.device = local
        o.n_tau = ntau
        o.precision = PRECISIONS[mode][0]
        return o

    out = {}
    clocks = ClockSampler()
    clocks.start()
    for mode in ("fp64", "split"):
        hs, b = [], None
        try:
            for inp in inputs:
                h = L.librpa_gpu_create(opts(mode))
                L.set_inputs(h, inp)
                hs.append(h)
            b = L.librpa_gpu_batch_create(hs)
            ec0 = L.librpa_gpu_batch_run(b)             # tunes the tiles, captures the graph
            t0 = time.perf_counter()
            for _ in range(steps):
                ec = L.librpa_gpu_batch_run(b)
            t_batch = (time.perf_counter() - t0) / steps
            st = L.librpa_gpu_batch_get_stats(b)
        finally:
            L.librpa_gpu_batch_destroy(b)
            for h in hs:
                L.librpa_gpu_destroy(h)
        # one by one: each structure warm (its own tuning), then one timed chi0 + ec
        t_one, ec_one = 0.0, []
        for inp in inputs:
            h = L.librpa_gpu_create(opts(mode))
            try:
                L.set_inputs(h, inp)
                L.librpa_gpu_chi0(h)
                L.librpa_gpu_ec(h)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                L.librpa_gpu_chi0(h)
                ec_one.append(L.librpa_gpu_ec(h)[0])
                t_one += time.perf_counter() - t0
            finally:
                L.librpa_gpu_destroy(h)
        dmax = max(abs(a - c) / abs(c) for a, c in zip(ec, ec_one))
        out[mode] = {"value": len(inputs) / t_batch, "ms_per_batch": 1e3 * t_batch,
                     "one_by_one": len(inputs) / t_one, "speedup": t_one / t_batch,
                     "max_rel_diff_vs_one_by_one": dmax, "repeat_identical": bool((ec0 == ec).all()),
                     "n_merged": st["n_merged"], "n_merged_tc": st["n_merged_tc"], "graph": st["graph"],
                     "tile_variants": [st["var_nx"], st["var_fin"]],
                     "launches_per_batch": st["launches"],
                     "stage_ms": {"green": st["ms_green"], "chi0": st["ms_chi0"], "freq": st["ms_freq"],
                                  "ec": st["ms_ec"]}}
    clk = clocks.stop()
    return out, clk


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--full", choices=["cubic", "graphene"], default=None,
                    help="reference arm: whole oracle energies of this workload instead of the sample")
    ap.add_argument("--single-thread", action="store_true", help="with --full: also one single-thread run")
    ap.add_argument("--single-thread-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-peaks", action="store_true", help="skip the FP64/TF32 peak probes")
    # smaller variants of the same workload, for profiler captures only (not bench lines)
    ap.add_argument("--workload", choices=["graphene", "cubic"], default="graphene",
                    help="graphene: the slab of the headline; cubic: the 2-atom cubic cell (2x2x2 k)")
    ap.add_argument("--kmesh", default="4,4,1", help="k-mesh of the graphene slab (profiling variants)")
    ap.add_argument("--ntau", type=int, default=16)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp64")
    ap.add_argument("--serve", action="store_true", help="serving workload instead of the headline")
    ap.add_argument("--batch", action="store_true", help="batched workload instead of the headline")
    ap.add_argument("--batch-n", type=int, default=64)
    ap.add_argument("--batch-sample", type=int, default=8,
                    help="structures of the batched sample added to the headline line (0: none)")
    ap.add_argument("--serve-requests", type=int, default=16)
    ap.add_argument("--serve-sample", type=int, default=12,
                    help="requests per arrival rate of the serving sweep added to the headline line (0: none)")
    ap.add_argument("--serve-rates", default="5,20,50,200",
                    help="arrival rates (req/s) of the serving sweep in the headline line")
    ap.add_argument("--rate", type=float, default=20.0, help="request arrival rate (Poisson), per second")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--modes", default="fp64_tc,split,split_fast,tf32x3,tf32,bf16,fp64@1e-3,fp64_tc@1e-3",
                    help="other precision modes timed after the headline, 'mode@theta' with G screening "
                         "(1 GPU; '' for none)")
    args = ap.parse_args()
    args.kmesh = tuple(int(x) for x in args.kmesh.split(","))
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.batch:
        return run_batch(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
