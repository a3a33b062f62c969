#!/usr/bin/env python3
"""Benchmark of the LLG forward + adjoint hot path on one node.

A step is one level-set iteration of the batched demultiplexer workload
(`batch64`): 8 candidates x 4 grid shapes (128x64, 256x64, 256x128, 512x128)
x 2 drive frequencies = 64 instances, 1,966,080 nodes, each integrated for
10,000 RK4 steps (forward), swept back by the checkpointed discrete adjoint
(dJ/dPhi) and updated by the level-set step.  Metric: node-steps per second
of forward + adjoint, node-steps = sum over instances of nodes x RK4 steps.
FP32 state with the adjoint's demag transpose in double-float (the
configuration whose gradient meets the FP64 oracle's 1e-4); the line also
carries forward-only throughput, the plain FP32 adjoint spectrum, the FP64
store-all path, and the nanoparticle, single-demultiplexer and thick-film
workloads.

Multi-GPU: every rank runs its own copy of the workload (independent
instances, no collective on the data path); value = all ranks' node-steps /
the slowest rank's time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "LLG fwd+adjoint node-steps/s, FP32 batched vs FP64 plain on GB300; % HBM roofline"
UNIT = "node-steps/s"

# The workloads a timed step can run: instances for N RK4 steps, the adjoint
# spectrum that meets the gradient bar on them (double-float on the
# demultiplexer shapes; the nanoparticle meets it in FP32; 3D grids have no
# double-float spectrum), and a description.
WORKLOADS = {
    "batch64": (lambda n: W.batch64(nsteps=n), "dfloat",
                "batch64: 8 candidates x {128x64,256x64,256x128,512x128} x 2 frequencies (3.0/3.4 GHz), "
                "YIG demultiplexer, 5 nm cells"),
    "particle64": (lambda n: [W.particle64(nsteps=n)], "working", "particle64: 64x64 Permalloy nanoparticle, 2 nm"),
    "demux256": (lambda n: [W.demux256(0, nsteps=n), W.demux256(1, nsteps=n)], "dfloat",
                 "demux256: 256x64 YIG demultiplexer at 3.0 and 3.4 GHz, 5 nm"),
    "thick512": (lambda n: [W.thick512(nsteps=n)], "working", "thick512: 512x512x4 YIG film, 3D demag"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--nsteps", type=int, default=10000, help="RK4 steps per instance")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, FP64 and CPU legs")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="batch64",
                    help="the timed level-set iteration's workload (batch64: the benchmark; the others for "
                         "profiling and comparison runs)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources the FP32 stage, column and adjoint kernels are compiled from
KERNEL_SOURCES = ("common.cuh", "dfloat.cuh", "kernels.cuh", "kernels_impl.cuh", "regfft.cuh", "tma.cuh", "cols16.cuh",
                  "k_stage_f32.cu", "k_cols_f32.cu", "k_cols16_f32.cu", "k_adj_f32.cu", "k_adj_df.cu", "k_cols_df.cu")


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2411_19109_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(family, spec):
    """DRAM bytes per whole-batch launch of a kernel family in the given
    adjoint-spectrum configuration, from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("source_hash") != kernel_source_hash():
            return None
        e = d["families"].get(f"{spec}:{family}")
        return None if e is None else float(e["dram_bytes_per_full_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank gets it): an all-reduce MAX of one
    float64 on `device` ("cuda" under NCCL, "cpu" under gloo)."""
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(node_steps_per_rank, world, ms_max):
    """Whole-job node-steps/s: every rank integrates its own replica of the
    workload, so the job does world x node_steps in the slowest rank's time."""
    return node_steps_per_rank * world / (ms_max / 1e3)


def fft_flops(insts, family):
    """FP64 path: FFT flops of one launch of a kernel family over the batch,
    5 N log2 N per complex transform of length N (pointwise arithmetic not
    counted).  Row kernels (0 stage, 2 adjoint): per grid row, 3 components
    x (inverse + forward) transforms of length Px/2 (the real rows ride as
    half-length complex sequences); column kernel (1): per column kx < Px/2,
    3 components x (forward + inverse) transforms of length Py."""
    tot = 0.0
    for i in insts:
        p = i.problem
        Px = max(16, 1 << (2 * p.nx - 1).bit_length())
        Py = max(1, 1 << (2 * p.ny - 1).bit_length()) if p.ny > 1 else 1
        Lx = Px // 2
        if family == 1:
            tot += Lx * 6 * 5 * Py * np.log2(Py)
        else:
            tot += p.ny * p.nz * 6 * 5 * Lx * np.log2(Lx)
    return tot


def fp64_roofline(insts, ka, kb):
    """Arithmetic roofline of the FP64 path: the kernel family with the most
    time, its FFT flops per launch over its average launch time, against the
    measured FP64 FMA throughput of the device."""
    from paper_2411_19109_gb300 import llg_fp64_fma_rate
    peak, _ = llg_fp64_fma_rate()
    fam = {f: (kb[f][0] - ka[f][0], kb[f][1] - ka[f][1]) for f in (0, 1, 2)}
    top = max(fam, key=lambda f: fam[f][1])
    n, ms = fam[top]
    if n <= 0 or ms <= 0:
        return None
    avg_s = ms / 1e3 / n
    ach = fft_flops(insts, top) / avg_s / 1e12
    names = {0: "rows_kernel<double,ROW_STAGE>", 1: "cols_kernel<double>", 2: "adj_kernel<double>"}
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "kernel": names[top], "avg_us": avg_s * 1e6,
            "shares": {names[f]: fam[f][1] / max(1e-30, sum(v[1] for v in fam.values())) for f in fam},
            "flops": "FFT flops only, 5 N log2 N per complex transform",
            "peak_source": "llg_fp64_fma_rate: FMA-chain kernel on this GPU (measured)"}


# --------------------------------------------------------------------------
# oracle leg (host cores): the CPU baseline and the reference arm
# --------------------------------------------------------------------------

def oracle_sample(nsteps=120):
    """Forward + adjoint of one 128x64 demultiplexer instance for `nsteps`
    RK4 steps with the FP64 oracle.  Returns (node-steps/s, seconds, sample)."""
    from oracle import llg as ollg
    inst = W.batch64(nsteps=nsteps, candidates=1)[0]
    t0 = time.perf_counter()
    model = ollg.Model(inst.problem, inst.phi)
    J, _, traj = model.forward(inst.m0, keep=True)
    model.adjoint(inst.m0, traj)
    dt = time.perf_counter() - t0
    ns = inst.problem.nx * inst.problem.ny * nsteps
    return ns / dt, dt, f"1 instance 128x64 of batch64, {nsteps} RK4 steps forward + store-all adjoint (FP64 numpy)"


def _oracle_worker(job):
    """One 128x64 instance of batch64 (index k < 16) through the oracle's
    forward + store-all adjoint; returns seconds."""
    k, nsteps = job
    from oracle import llg as ollg
    inst = W.batch64(nsteps=nsteps)[k]
    t0 = time.perf_counter()
    model = ollg.Model(inst.problem, inst.phi)
    _, _, traj = model.forward(inst.m0, keep=True)
    model.adjoint(inst.m0, traj)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The oracle on all host cores: one single-threaded process per core
    (spawned, so no process inherits a CUDA context), each integrating its
    own 128x64 instance of batch64; up to 16 instances (the 128x64 ones)."""

    def __init__(self):
        import multiprocessing as mp
        self.n = max(1, min(16, host_cores()))
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        self.pool = mp.get_context("spawn").Pool(self.n)

    def sample(self, nsteps=120):
        """(node-steps/s, wall seconds, sample) over self.n instances at once."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker, [(k, nsteps) for k in range(self.n)])
        wall = time.perf_counter() - t0
        ns = self.n * 128 * 64 * nsteps
        return ns / wall, wall, (f"{self.n} instances 128x64 of batch64 at once, one process per core, {nsteps} RK4 "
                                 "steps forward + store-all adjoint each (FP64 numpy)")

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    nst = 120
    pool = OraclePool()
    pool.sample(10)                       # starts the workers
    for _ in range(max(0, args.warmup)):
        pool.sample(20)
    vals, secs = [], []
    for _ in range(max(1, args.steps)):
        v, s, sample = pool.sample(nst)
        vals.append(v)
        secs.append(s)
    pool.close()
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "batch64 (sampled: the 128x64 instances, one per host core, per step)",
                       "nsteps": nst},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.n, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

# FP32 operations of the double-float (compensated) arithmetic, as the kernels
# implement it: a complex add 16, a complex product 32, a real product 5.
def _df_fft_ops(L, half_in=False):
    """FP32 operations of one double-float register FFT of length L
    (8-element lanes: a first pass of radix R0 without twiddles, then radix-8
    passes with 7 twiddle products per butterfly).  half_in: the forward
    transform of zero-padded data, whose first pass leaves out the zero upper
    half of every butterfly's inputs (radix 2: a copy; radix 4: 4 complex sums
    of 8; radix 8: 16 of 24)."""
    m = int(np.log2(L))
    r0 = 2 if m % 3 == 1 else (4 if m % 3 == 2 else 8)
    npass = m // 3 if m % 3 == 0 else m // 3 + 1
    dft = {2: 0, 4: 64, 8: 308} if half_in else {2: 32, 4: 128, 8: 436}
    return (L // r0) * dft[r0] + (npass - 1) * (L // 8) * (436 + 7 * 32)


def df_ops_per_launch(insts, family):
    """FP32 operations of one whole-batch launch of a double-float kernel:
    family 2 (fused adjoint stage: inverse and forward row FFTs of length
    Px/2 per row and component, with the packed-real unpack (80 per point)
    and pack (90)), family 4 (one row transform of the split adjoint stage,
    inverse or forward: half of that), family 3 (column pass: forward and
    inverse FFT of length Py per column kx < Px/2 and component, and the
    tensor product, about 27 per point).  The forward transforms take
    zero-padded inputs (half-input first pass).  Node-phase arithmetic is
    not counted."""
    tot = 0.0
    for i in insts:
        p = i.problem
        Px = max(16, 1 << (2 * p.nx - 1).bit_length())
        Py = max(8, 1 << (2 * p.ny - 1).bit_length())
        Lx = Px // 2
        if family == 2:
            tot += p.ny * p.nz * 3 * (_df_fft_ops(Lx) + _df_fft_ops(Lx, True) + Lx * (80 + 90))
        elif family == 4:
            tot += p.ny * p.nz * 3 * ((_df_fft_ops(Lx) + _df_fft_ops(Lx, True)) / 2 + Lx * 85)
        else:
            tot += Lx * 3 * (_df_fft_ops(Py) + _df_fft_ops(Py, True) + Py * 27)
    return tot


# Algorithmic bytes per node per launch, the data each kernel must move at
# least once: FP32 stage (spectrum 24+24, Y 12, psi 4, m 12, accumulator 9+9,
# outputs 12, recorded field 6); FP32 column pass (24 read + 24 written);
# adjoint stage (spectrum read and written, the stage's Y, Bbar, psi, adjoint
# state, gradient sums and next-stage records: 137 + the spectrum 48 in FP32,
# 96 in double-float); double-float column pass (48 read + 48 written); the
# split adjoint stage's FP32 node phase (137 + the demag transpose 12) and
# one of its double-float row transforms (spectrum 48 + nodes 12).
BYTES_PER_NODE = {0: 112.0, 1: 48.0, 2: 233.0, 3: 96.0, 4: 60.0}
BYTES_PER_NODE_FP32_ADJ = 185.0
BYTES_PER_NODE_SPLIT_ADJ = 149.0
FAMILY = {0: "rows_kernel<float,ROW_STAGE> (inverse row FFT + field + RK4 stage + forward row FFT)",
          1: "cols16_kernel<float> (column FFT with 16-element lanes, tensor product, inverse column FFT)",
          2: "adj_kernel<float,dfloat> (adjoint stage: double-float row FFTs, demag/exchange transposes, dJ/dpsi)",
          3: "cols_kernel<dfloat> (column pass of the adjoint's double-float frequency domain)",
          4: "spec_rows_kernel<float,dfloat> (double-float row transforms of the split adjoint stage)"}
SPLIT_ADJ_NAME = "adj_split_kernel<float> (split adjoint stage: FP32 node phase, demag/exchange transposes, dJ/dpsi)"
FP32_LANES_PER_SM, SMS = 128, 152


def family_kind(f, spec, split):
    """How a timing family is measured: ("df", bytes/node) for double-float
    kernels (FP32-arithmetic roofline), ("hbm", bytes/node) otherwise."""
    if f == 2:
        if spec != "dfloat":
            return "hbm", BYTES_PER_NODE_FP32_ADJ, "adj_kernel<float> (adjoint stage)"
        if split:
            return "hbm", BYTES_PER_NODE_SPLIT_ADJ, SPLIT_ADJ_NAME
        return "df", BYTES_PER_NODE[2], FAMILY[2]
    if f in (3, 4):
        return "df", BYTES_PER_NODE[f], FAMILY[f]
    return "hbm", BYTES_PER_NODE[f], FAMILY[f]


def kernel_families(sk, step_fn, insts, nodes, spec, split):
    """Per-family launches and average device time over one step of a
    context that brackets every stage-kernel launch with CUDA events."""
    fams = (0, 1, 2, 3, 4)
    f0 = {f: sk.kernel_time(f) for f in fams}
    step_fn(sk)
    import torch
    torch.cuda.synchronize()
    f1 = {f: sk.kernel_time(f) for f in fams}
    kern = {}
    for f in fams:
        n = f1[f][0] - f0[f][0]
        t = f1[f][1] - f0[f][1]
        if n <= 0:
            continue
        avg_ms = t / n
        kind, bpn, name = family_kind(f, spec, split)
        bytes_launch = bpn * nodes
        kern[f] = {"kernel": name, "kind": kind, "bytes_per_node": bpn, "launches": n, "total_ms": t,
                   "avg_us": 1e3 * avg_ms, "bytes_per_launch": bytes_launch,
                   "achieved_gbs": bytes_launch / (avg_ms / 1e3) / 1e9}
        if kind == "df":
            ops = df_ops_per_launch(insts, f)
            kern[f]["fp32_ops_per_launch"] = ops
            kern[f]["achieved_tops"] = ops / (avg_ms / 1e3) / 1e12
    tot = sum(v["total_ms"] for v in kern.values()) or 1.0
    for v in kern.values():
        v["share"] = v["total_ms"] / tot
    return kern


def name_column_family(kern, insts, cfg):
    """Name the FP32 column kernel that family 1 ran on these grids."""
    if 1 in kern:
        kern[1]["kernel"] = ("cols3_kernel<float> (3D column pass)" if any(i.problem.nz > 1 for i in insts) else
                             "cols16_kernel<float> (16-element lanes)" if cfg.get("col_lanes") == 16 else
                             "cols_kernel<float> (8-element lanes)")


def roofline_of(kern, spec, hbm, peak_kind, sm_mhz, nodes, timing_note, with_traffic=True):
    """Roofline of the kernel with the largest total time.  `traffic` is the
    ncu DRAM capture of that kernel on the benchmarked batch; other workloads
    (with_traffic=False) report null, as no capture covers them."""
    dom = max(kern, key=lambda f: kern[f]["total_ms"])
    k = kern[dom]
    name = k["kernel"]
    traffic = ncu_traffic(dom, spec) if with_traffic else None
    if k["kind"] == "df":
        # double-float kernels: bound by FP32 arithmetic (the compensated
        # operations), against the FP32 lanes x clock of the device
        peak = SMS * FP32_LANES_PER_SM * (sm_mhz or 2070.0) * 1e6 / 1e12
        return {"bound": "alu", "achieved": k["achieved_tops"], "peak": peak, "unit": "TFLOP/s",
                "frac": k["achieved_tops"] / peak, "traffic": traffic, "kernel": name,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x the median SM clock under load, one FP32 "
                               "add/multiply/FMA per lane per clock (FP32 operations, an FMA counted once)",
                "ops_per_launch": k["fp32_ops_per_launch"],
                "ops": "FP32 operations of the double-float FFTs (and pack/unpack, tensor product) per launch",
                "hbm_model": {"bytes_per_node": k["bytes_per_node"], "achieved_gbs": k["achieved_gbs"],
                              "frac": k["achieved_gbs"] / hbm},
                "kernel_timing": timing_note}
    bpn = k["bytes_per_node"]
    return {"bound": "hbm", "achieved": k["achieved_gbs"], "peak": hbm, "unit": "GB/s",
            "frac": k["achieved_gbs"] / hbm, "traffic": traffic,
            "kernel": name, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
            "bytes_per_node": bpn, "nodes_per_launch": nodes, "kernel_timing": timing_note}


def time_workload(insts, nsteps, precision="fp32", ckpt="periodic", spec="working", reps=1, stream=None,
                  kinsts=None):
    """Forward and forward+adjoint node-steps/s of one workload (CUDA graphs,
    measured launch configuration), its device memory, and, given `kinsts`
    (the same instances at fewer RK4 steps), the dominant kernel's roofline
    from a pass with CUDA events around every launch."""
    import torch
    from paper_2411_19109_gb300 import Solver
    nodes = sum(i.problem.nx * i.problem.ny * i.problem.nz for i in insts)
    s = Solver([i.problem for i in insts], precision=precision, ckpt=ckpt, use_graph=True, stream=stream,
               adj_spectral=spec, tune="measure" if precision == "fp32" else "default")
    try:
        phi = s.pack_scalar([i.phi for i in insts])
        m0 = s.pack_vector([i.m0 for i in insts])
        s.forward(phi, m0)
        s.adjoint()                                       # warm-up: graph captures
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        tf = ta = 0.0
        for _ in range(reps):
            e[0].record(s.stream)
            s.forward(phi, m0)
            e[1].record(s.stream)
            s.adjoint()
            e[2].record(s.stream)
            torch.cuda.synchronize()
            tf += e[0].elapsed_time(e[1])
            ta += e[1].elapsed_time(e[2])
        ns = nodes * nsteps * reps
        cfg = s.launch_config()[0]
        out = {"forward": ns / (tf / 1e3), "forward_adjoint": ns / ((tf + ta) / 1e3), "unit": UNIT,
               "ms_forward": tf / reps, "ms_adjoint": ta / reps, "device_bytes": int(s.query()[0]),
               "launch": cfg, "nodes": nodes, "rk4_steps": nsteps, "instances": len(insts)}
    finally:
        s.close()
    if kinsts is not None:
        sk = Solver([i.problem for i in kinsts], precision=precision, ckpt=ckpt, use_graph=False, stream=stream,
                    adj_spectral=spec, tune="given", launch=cfg, time_kernels=True)
        try:
            def one(sv):
                sv.forward(phi, m0)
                sv.adjoint()
            one(sk)
            kern = kernel_families(sk, one, kinsts, nodes, spec, bool(cfg.get("adj_split")))
        finally:
            sk.close()
        name_column_family(kern, insts, cfg)
        hbm, peak_kind = measured_peaks()
        out["roofline"] = roofline_of(kern, spec, hbm, peak_kind, None, nodes, with_traffic=False, timing_note=
                                      f"CUDA events around every launch, a forward + adjoint of "
                                      f"{kinsts[0].problem.nsteps} RK4 steps without graphs")
        out["kernels"] = {v["kernel"].split(" ")[0]: {kk: vv for kk, vv in v.items() if kk != "kernel"}
                          for v in kern.values()}
    return out


def run_ours(args):
    import torch
    from paper_2411_19109_gb300 import Solver

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    else:
        dist = None

    def barrier():
        if dist is not None:
            dist.barrier()

    make, SPEC, wdesc = WORKLOADS[args.workload]
    insts = make(args.nsteps)
    nodes = sum(i.problem.nx * i.problem.ny * i.problem.nz for i in insts)
    node_steps = nodes * args.nsteps
    stream = torch.cuda.current_stream()
    s = Solver([i.problem for i in insts], precision="fp32", ckpt="periodic", use_graph=True, stream=stream,
               adj_spectral=SPEC, tune="measure")
    launch, tune_ms = s.launch_config()
    phi0 = s.pack_scalar([i.phi for i in insts])
    m0 = s.pack_vector([i.m0 for i in insts])
    mask = torch.cat([torch.as_tensor(i.mask.reshape(-1)) for i in insts]).cuda()
    phi = phi0.clone()
    ev_fwd = []

    # Every step repeats the same level-set iteration (forward, adjoint,
    # update) from phi0: the exact gradient of this workload over 10,000
    # steps is dominated by the chaotic motion of m at air nodes (it grows
    # e-fold every ~4 ps of simulated time and leaves the FP32 range on the
    # 512x128 grids), so iterating the update would feed overflowed values
    # back into phi.  Throughput does not depend on the values.
    def step(lr, solver=None, mark=False):
        sv = solver or s
        if mark:
            a = torch.cuda.Event(enable_timing=True)
            a.record(stream)
        J, _ = sv.forward(phi, m0)
        if mark:
            b = torch.cuda.Event(enable_timing=True)
            b.record(stream)
            ev_fwd.append((a, b))
        g, _ = sv.adjoint()
        sv.levelset_step(phi, g, mask, lr)
        phi.copy_(phi0)
        return J, g

    def finite_absmax(g):
        a = g.abs()
        a = a[torch.isfinite(a)]
        return float(a.max().item()) if a.numel() else 0.0

    # warm-up; the learning rate is fixed from the first gradient
    lr = 0.0
    for w in range(max(3, args.warmup)):
        J, g = step(lr)
        if w == 0:
            gmax = finite_absmax(g)
            lr = 0.02 / gmax if gmax > 0 else 0.0
    torch.cuda.synchronize()

    l0 = s.launch_count()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        J, g = step(lr, mark=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_fwd = sum(a.elapsed_time(b) for a, b in ev_fwd) / len(ev_fwd)
    launches = s.launch_count() - l0
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(node_steps, world, ms_max)
    csum = clocks.summary()

    # per-launch kernel durations: one more step through a second context of
    # the same launch configuration that brackets every stage-kernel launch
    # with CUDA events on the solver stream (graph replays hide per-launch
    # times, so the timed region above runs graphs and this pass does not)
    sk = Solver([i.problem for i in insts], precision="fp32", ckpt="periodic", time_kernels=True,
                use_graph=False, stream=stream, adj_spectral=SPEC, tune="given", launch=launch)
    kern = kernel_families(sk, lambda sv: step(lr, sv), insts, nodes, SPEC, bool(launch.get("adj_split")))
    sk.close()
    if args.workload != "batch64":
        name_column_family(kern, insts, launch)
    hbm, peak_kind = measured_peaks()
    roofline = roofline_of(kern, SPEC, hbm, peak_kind, csum.get("sm_mhz"), nodes,
                           "CUDA events around every launch on the solver stream, over one more step of the "
                           "same workload and launch configuration without graphs",
                           with_traffic=args.workload == "batch64")

    mem_bytes, _ = s.query()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wdesc,
                       "instances": len(insts), "nodes": nodes, "rk4_steps": args.nsteps,
                       "checkpoint": "periodic, K = ceil(sqrt(N))", "precision": "fp32",
                       "adjoint_spectrum": ("double-float (hi + lo FP32 pairs) for the adjoint's demag transpose; "
                                            "node arrays FP32") if SPEC == "dfloat" else "FP32",
                       "parity": ("dJ/dPhi within 1e-4 of the FP64 oracle on all four shapes (measured <= 2.7e-6 "
                                  "at 100 steps, tests/test_gpu_fullsize.py)") if args.workload == "batch64" else
                                 "see tests/test_gpu_fullsize.py for this workload's parity",
                       "launch": launch, "launch_tuning_ms": tune_ms,
                       "step": "forward + checkpointed adjoint + level-set update, each timed step "
                               "repeated from the same phi (CUDA-graph replays of every segment)",
                       "l2": "inputs larger than L2 (working set %.1f GB per GPU)" % (mem_bytes / 1e9),
                       "parallelism": f"replicas x{world}"},
            "forward_only": {"value": node_steps / (ms_fwd / 1e3), "unit": UNIT, "ms_per_forward": ms_fwd,
                             "note": "the forward pass of each timed step (periodic checkpoints, objective)"},
            "roofline": roofline, "gpu_launches": launches,
            "clocks": csum,
            "kernels": {v["kernel"].split(" ")[0]: {kk: vv for kk, vv in v.items() if kk != "kernel"}
                        for v in kern.values()},
            "peak_mem_bytes": int(mem_bytes)}

    if rank == 0 and not args.no_extras and args.workload == "batch64":
        # e2e: the same step through the public API with host buffers
        phi_h = phi0.cpu().pin_memory()
        m0_h = m0.cpu().pin_memory()
        g_h = torch.empty(s.total, dtype=torch.float32).pin_memory()
        phi_d = torch.empty_like(phi0)
        m0_d = torch.empty_like(m0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        phi_d.copy_(phi_h, non_blocking=True)
        m0_d.copy_(m0_h, non_blocking=True)
        Jh, _ = s.forward(phi_d, m0_d)
        gd, _ = s.adjoint()
        s.levelset_step(phi_d, gd, mask, lr)
        g_h.copy_(gd, non_blocking=True)
        a1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        e2e_ms = max(a0.elapsed_time(a1), 1e3 * wall)
        h2d = (phi0.numel() + m0.numel()) * 4
        d2h = s.total * 4 + 8 * len(insts)
        line["e2e"] = {"value": node_steps / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "steps": 1}
        s.close()
        # the same step with the plain FP32 adjoint spectrum (faster; its
        # gradient misses 1e-4 on these shapes: 1e-3 on the 256x64
        # demultiplexer at 100 steps)
        sw = Solver([i.problem for i in insts], precision="fp32", ckpt="periodic", use_graph=True, stream=stream,
                    adj_spectral="working", tune="measure")
        step(lr, sw)
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        step(lr, sw)
        b1.record(stream)
        torch.cuda.synchronize()
        line["fp32_adjoint_spectrum"] = {"value": node_steps / (b0.elapsed_time(b1) / 1e3), "unit": UNIT,
                                         "steps": 1, "launch": sw.launch_config()[0],
                                         "parity": "dJ/dPhi misses 1e-4 on the demultiplexer shapes (1.0e-3 on "
                                                   "256x64 at 100 steps); m and J meet their bars"}
        sw.close()
        # plain FP64 store-all path on the same instances, sampled steps
        nst64 = 200
        insts64 = W.batch64(nsteps=nst64)
        s64 = Solver([i.problem for i in insts64], precision="fp64", ckpt="store_all", time_kernels=True)
        p64 = s64.pack_scalar([i.phi for i in insts64])
        q64 = s64.pack_vector([i.m0 for i in insts64])
        s64.forward(p64, q64)
        s64.adjoint()
        torch.cuda.synchronize()
        k64a = {f: s64.kernel_time(f) for f in (0, 1, 2)}
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        s64.forward(p64, q64)
        s64.adjoint()
        b1.record(stream)
        torch.cuda.synchronize()
        ms64 = b0.elapsed_time(b1)
        mem64, _ = s64.query()
        per_step = mem64 / nst64
        k64b = {f: s64.kernel_time(f) for f in (0, 1, 2)}
        line["fp64_store_all"] = {"value": nodes * nst64 / (ms64 / 1e3), "unit": UNIT,
                                  "sample": f"all 64 instances, {nst64} RK4 steps",
                                  "device_bytes_sample": int(mem64),
                                  "device_bytes_projected_full": int(per_step * args.nsteps),
                                  "roofline": fp64_roofline(insts64, k64a, k64b),
                                  "launches": "direct, with CUDA events around each launch (per-kernel times)"}
        s64.close()
        del p64, q64
        line["workloads"] = other_workloads(stream)
        line["record_modes"] = record_modes(stream)
        # CPU baseline: the oracle on this host's cores (all cores, and one)
        pool = OraclePool()
        pool.sample(10)                   # starts the workers
        v, secs, sample = pool.sample(300)      # about 10 s on 16 cores
        pool.close()
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": pool.n, "kind": "oracle", "sample": sample,
                                "seconds": secs}
        v1, secs1, sample1 = oracle_sample(300)    # about 10 s on one core
        line["cpu_baseline_1core"] = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample1,
                                      "seconds": secs1}
    else:
        if rank == 0:
            line["e2e"] = None
        s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def record_modes(stream):
    """Memory against time of the two segment records: every stage (the
    default) or only m per step with each reverse step recomputing its
    stages.  Device bytes at the full configurations (contexts created,
    not run) and forward+adjoint throughput on batch64 at 1000 RK4 steps."""
    from paper_2411_19109_gb300 import Solver
    out = {}
    for rec in ("stages", "states"):
        r = {}
        sv = Solver([i.problem for i in W.batch64(nsteps=10000)], precision="fp32", ckpt="periodic",
                    adj_spectral="dfloat", record=rec, stream=stream)
        r["batch64_10000_device_bytes"] = int(sv.query()[0])
        sv.close()
        sv = Solver([W.thick512(nsteps=50000).problem], precision="fp32", ckpt="periodic", record=rec, stream=stream)
        r["thick512_50000_device_bytes"] = int(sv.query()[0])
        sv.close()
        insts = W.batch64(nsteps=1000)
        t = time_workload_rec(insts, 1000, rec, stream)
        r["batch64_1000_forward_adjoint"] = t
        out[rec] = r
    out["unit"] = UNIT
    return out


def time_workload_rec(insts, nsteps, rec, stream):
    import torch
    from paper_2411_19109_gb300 import Solver
    nodes = sum(i.problem.nx * i.problem.ny * i.problem.nz for i in insts)
    s = Solver([i.problem for i in insts], precision="fp32", ckpt="periodic", use_graph=True, stream=stream,
               adj_spectral="dfloat", tune="measure", record=rec)
    try:
        phi = s.pack_scalar([i.phi for i in insts])
        m0 = s.pack_vector([i.m0 for i in insts])
        s.forward(phi, m0)
        s.adjoint()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.forward(phi, m0)
        s.adjoint()
        e1.record(s.stream)
        torch.cuda.synchronize()
        return nodes * nsteps / (e0.elapsed_time(e1) / 1e3)
    finally:
        s.close()


def other_workloads(stream):
    """The nanoparticle (config 2), the single 256 x 64 demultiplexer at
    both drive frequencies (config 3) and the 512 x 512 x 4 thick film
    (config 5): forward and forward+adjoint node-steps/s, device memory, and
    the plain FP64 store-all path (measured, sampled or projected)."""
    out = {}
    # config 2: 64 x 64 nanoparticle, 5000 steps, energy + area objective
    # (its FP32 gradient meets 1e-4 with the FP32 adjoint spectrum)
    c2 = [W.particle64(nsteps=5000)]
    r = time_workload(c2, 5000, spec="working", stream=stream, kinsts=[W.particle64(nsteps=200)])
    r64 = time_workload(c2, 5000, precision="fp64", ckpt="store_all", stream=stream)
    r["fp64_store_all"] = {"forward_adjoint": r64["forward_adjoint"], "device_bytes": r64["device_bytes"],
                           "steps": 5000}
    r["note"] = "4096 nodes per launch: latency-bound (launch and barrier latency, not bandwidth)"
    out["particle64_5000"] = r
    # config 3: 256 x 64 demultiplexer, 3.0 and 3.4 GHz runs of one design,
    # 20,000 steps, double-float adjoint spectrum (its gradient parity case)
    c3 = [W.demux256(0, nsteps=20000), W.demux256(1, nsteps=20000)]
    r = time_workload(c3, 20000, spec="dfloat", stream=stream,
                      kinsts=[W.demux256(0, nsteps=200), W.demux256(1, nsteps=200)])
    n64 = 2000
    c3s = [W.demux256(0, nsteps=n64), W.demux256(1, nsteps=n64)]
    r64 = time_workload(c3s, n64, precision="fp64", ckpt="store_all", stream=stream)
    r["fp64_store_all"] = {"forward_adjoint": r64["forward_adjoint"], "steps": n64,
                           "device_bytes_sample": r64["device_bytes"],
                           "device_bytes_projected_20000": int(r64["device_bytes"] * 20000 / n64)}
    r["note"] = "32768 nodes per launch over both runs: latency-bound"
    out["demux256_20000"] = r
    # config 5: 512 x 512 x 4 thick film (full 3D demag, padded 1024 x 1024 x 8)
    # at a stated step count; the FP32 periodic path at 50,000 steps is
    # projected from its per-step rate, the FP64 store-all path's footprint
    # (50,001 states of 3 x 1,048,576 doubles) does not fit the device
    n5 = 1000
    c5 = [W.thick512(nsteps=n5)]
    r = time_workload(c5, n5, spec="working", stream=stream, kinsts=[W.thick512(nsteps=50)])
    nn = 512 * 512 * 4
    r["projected_50000"] = {"seconds_forward_adjoint": nn * 50000 / r["forward_adjoint"],
                            "fp64_store_all_bytes": int(50001 * 3 * nn * 8)}
    r["note"] = (f"{n5} RK4 steps (of the configuration's 50,000); the 3D column pass keeps whole padded "
                 "columns of all layers in shared memory; FP64 cannot run this grid (nz * Py = 4096 > 2048)")
    out["thick512"] = r
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
