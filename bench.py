#!/usr/bin/env python3
"""Training throughput of gradient-optimised NEP on one GB300.

One step = the whole hot path over one batch: descriptors, network, energies,
forces, virials, loss, the exact gradient w.r.t. every parameter, and an Adam
update with the Eq. 17 learning rate, captured once as a CUDA graph and
replayed.  The headline runs the FP32 form (FP32 network; the sweep
contractions as split-TF32 tensor-core products with FP32-level error, held
to the FP32 tolerances against the FP64 oracle); the BF16 and TF32 network
modes are timed beside it with their force difference from it.  The workload
is 256 synthetic Sb/Te structures of 32-400 atoms (perturbed rocksalt,
liquid-like and strained cells in equal thirds), n_max 8/8, basis 12/12,
l_max 4 with the 4-body term, 50 hidden neurons, labels from a random teacher
model of the same shape.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--repeats R]
                    [--impl gnep|reference] [--precision fp32|tf32|bf16]

Prints one JSON line (rank 0).  The neighbour build is done once before the
timed region (structures are fixed during training) and is reported apart.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "training atoms/sec per loss+grad step (E+F+V) at stated force error; % of roofline"
UNIT = "atoms/s"
WORKLOAD = dict(workload="sbte_256_structures_32-400_atoms_nmax8_basis12_lmax4_4body_h50",
                n_struct=256, size_range=[32, 400], phases="rocksalt/liquid/strained thirds",
                n_max=[8, 8], basis=[12, 12], l_max=4, four_body=True, hidden=50,
                rc=[7.0, 4.0], batch="full (one step = all 256 structures)")
MODEL_KW = dict(n_max=(8, 8), basis=(12, 12), hidden=50, four_body=True)
LAMBDAS = dict(lambda_e=1.0, lambda_f=1.0, lambda_v=0.1)
L2_BYTES = 129 * 1024 * 1024


# ----------------------------------------------------------------- FLOP model

def work_model_flops(nqr=9, kr=13, nqa=9, ka=13, ns=2, H=50, fb=True, N=1, PR=1, PA=1, L=24, lmax=4):
    """Algorithmic FP32 FLOPs per launch of each kernel, on the fixed work
    model of the method (FMA = 2 FLOP), counted per unit as the formulation
    needs it, whatever the kernels do:
      sweep 1 (descriptors)  radial pair 15 + 4K + 2 N_q^R K;
                             angular pair 15 + 4K + 2 N_q^A K + 50 + 2 N_q^A L;
                             atom 2 N_q^A L (q_nl) + 60 N_q^A (4-body)
      sweep 2 (forces)       radial pair 4K + 2 N_q^R K + 20;
                             angular pair 4 N_q^A K + 150 + 8 N_q^A L
      sweep 3 (tangent)      radial pair as sweep 2;
                             angular pair 4 N_q^A K + 270 + 4 N_q^A L; atom 2 N_q^A L
      sweep 4 (c-gradient)   radial pair 8K + 4 N_q^R K;
                             angular pair 8K + 120 + 6 N_q^A L + 6 N_q^A K
      network                atom 4 N_des H (forward), 8 N_des H (backward)
    with K the basis functions, N_q the channels and L = 24 (l, m) components
    (l_max 4; lmax sets the angular descriptor columns, L is passed with it,
    and the per-pair constants stay those of l_max 4).
    Each sweep's radial part is charged to the kernel that does it (the radial
    force is fused into the force gather, the radial c-gradient works on
    per-atom basis sums but is charged per pair here)."""
    D = nqr + lmax * nqa + (nqa if fb else 0)
    q4 = 60 * nqa if fb else 0
    f = {}
    f["desc_radial"] = PR * (15 + 4 * kr + 2 * nqr * kr)
    f["desc_angular"] = PA * (15 + 4 * ka + 2 * nqa * ka + 50 + 2 * nqa * L) + N * (2 * nqa * L + q4)
    f["mlp_fwd"] = N * 4 * D * H
    f["force_angular"] = PA * (4 * nqa * ka + 150 + 8 * nqa * L)
    f["force_atoms"] = PR * (4 * kr + 2 * nqr * kr + 20)
    f["tangent_radial"] = PR * (4 * kr + 2 * nqr * kr + 20)
    f["tangent_angular"] = PA * (4 * nqa * ka + 270 + 4 * nqa * L) + N * 2 * nqa * L
    f["mlp_bwd"] = N * 8 * D * H
    f["cgrad_radial"] = PR * (8 * kr + 4 * nqr * kr)
    f["cgrad"] = PA * (8 * ka + 120 + 6 * nqa * L + 6 * nqa * ka)
    return f


def algo_bytes(nqr=9, kr=13, nqa=9, ka=13, ns=2, H=50, fb=True, N=1, PR=1, PA=1, HP=64):
    """Compulsory DRAM bytes per launch of each kernel: every input the
    kernel needs read once and every output written once (FP32 arrays, int32
    indices, float4 pair vectors), nothing re-read."""
    D = nqr + 4 * nqa + (nqa if fb else 0)
    A = nqa * 24                   # S_nlm per atom
    FRn = ns * kr
    ang_cols = 4 * nqa + (nqa if fb else 0)
    b = {}
    b["desc_radial"] = 4 * (PR * 4 + 2 * N + N * FRn + N * nqr)
    b["desc_angular"] = 4 * (PA * 4 + 2 * N + N * A + N * ang_cols)
    b["mlp_fwd"] = 4 * N * (D + D + 1 + HP + FRn)
    b["force_angular"] = 4 * (PA * 5 + N * A + N * D + PA * 4)
    b["force_atoms"] = 4 * (PR * 5 + N * FRn + N + PA * 9 + 9 * N)
    b["tangent_radial"] = 4 * (PR * 5 + 4 * N + N * FRn + N * nqr)
    b["tangent_angular"] = 4 * (PA * 6 + 4 * N + N * A + N * A + N * ang_cols + PA * 4)
    b["mlp_bwd"] = 4 * N * (2 * D + HP + D + 2)
    b["cgrad"] = 4 * (N * (2 * A + 2 * (ang_cols + nqr)) + PA * 8 + N)
    b["cgrad_radial"] = 4 * N * (2 * nqr + 2 * FRn + 1)
    return b


# ----------------------------------------------------------------- helpers

def csrc_sha() -> str:
    """Hash of the kernel sources without their comments and with white space
    collapsed, so that a profile stays matched to the code it measured across
    edits of comments only."""
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2507_00528_gb300", "csrc", "*"))):
        txt = open(p, encoding="utf-8", errors="replace").read()
        txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", " ", txt)
        h.update(" ".join(txt.split()).encode())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    for p in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        txt = open(p).read()
        m1 = re.search(r"^kernel:\s*(\S+)", txt, re.M)
        m2 = re.search(r"^source_sha:\s*(\S+)", txt, re.M)
        m3 = re.search(r"^dram_bytes_per_launch_full_workload:\s*([0-9.eE+]+)", txt, re.M)
        if m1 and m2 and m3 and m1.group(1) == kernel and m2.group(1) == csrc_sha():
            return float(m3.group(1))
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, ident: str, interval_ms: int = 50):
        self.ident = ident
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []
        self.out = ""

    def _reader(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line))

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.ident}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._reader, daemon=True)
        self.thread.start()
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 5.0:  # sampler running before timing starts
            time.sleep(0.01)
        self.t_start = time.perf_counter()
        return self

    def __exit__(self, *a):
        if self.proc:
            t_end = time.perf_counter()
            time.sleep(2.5 * self.interval_ms / 1000)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)
            lo, hi = self.t_start, t_end + 1.5 * self.interval_ms / 1000
            self.out = "".join(l for t, l in self.lines if lo <= t <= hi)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------- oracle leg

def oracle_sample_step(batch, seconds: float, steps: int = 1):
    """Time the FP64 oracle (loss + explicit gradient + Adam) on a bounded
    sample of the workload: the smallest structures whose estimated cost fits
    in `seconds` per step."""
    import oracle as O
    from paper_2507_00528_gb300 import synth
    cfg = O.Cfg(nq_r=9, nq_a=9, k_r=13, k_a=13, hidden=50, four_body=True)
    sizes = batch.sizes()
    per_atom = 0.07  # s/atom, measured order of magnitude for this shape
    budget = max(1, int(seconds / per_atom))
    idx, tot = [], 0
    for s in np.argsort(sizes):  # smallest first keeps the sample bounded
        if tot + sizes[s] > budget and idx:
            break
        idx.append(int(s))
        tot += int(sizes[s])
    sb = batch.subset(sorted(idx))
    T = synth.uniform_params(cfg.n_params, 12).astype(np.float64)
    P = synth.uniform_params(cfg.n_params, 11).astype(np.float64)
    s = O.descriptor_scale(cfg, T, sb)
    y = O.teacher_labels(cfg, T, s, sb, **LAMBDAS)
    m = np.zeros_like(P); v = np.zeros_like(P)
    times = []
    for k in range(steps):
        t0 = time.perf_counter()
        _, g = O.loss_grad(cfg, P, s, sb, y)
        O.adam(P, m, v, g, k + 1, 1e-3)
        times.append(time.perf_counter() - t0)
    return sb.n_atoms, len(idx), times


def _oracle_structure_step(sb):
    """Worker: one oracle loss + gradient on the one-structure batch sb;
    returns (atoms, seconds of the gradient evaluation)."""
    import oracle as O
    from paper_2507_00528_gb300 import synth
    cfg = O.Cfg(nq_r=9, nq_a=9, k_r=13, k_a=13, hidden=50, four_body=True)
    T = synth.uniform_params(cfg.n_params, 12).astype(np.float64)
    P = synth.uniform_params(cfg.n_params, 11).astype(np.float64)
    sc = O.descriptor_scale(cfg, T, sb)
    y = O.teacher_labels(cfg, T, sc, sb, **LAMBDAS)
    t0 = time.perf_counter()
    O.loss_grad(cfg, P, sc, sb, y)
    return sb.n_atoms, time.perf_counter() - t0


def oracle_all_cores(batch):
    """The oracle on every host core at once (a spawn pool, one structure per
    process: the smallest structures, one per core).  The evaluations run
    concurrently, so the sample's wall time is the slowest one; atoms/s is the
    sample's atoms over that time."""
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    subs = [batch.subset([int(s)]) for s in np.argsort(batch.sizes())[:ncores]]
    with mp.get_context("spawn").Pool(ncores) as pool:
        res = pool.map(_oracle_structure_step, subs, chunksize=1)
    atoms = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": atoms / wall, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": f"{len(subs)} smallest structures ({atoms} atoms), one per process, loss + explicit-route "
                      f"gradient, {wall:.1f} s for the slowest"}


def run_reference(args):
    from paper_2507_00528_gb300 import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    batch = synth.make_config(2)
    # The oracle needs ~2 s for even the smallest structure of this workload, so
    # the arm keeps to a wall-clock budget: one structure-sample per step, at
    # most three warm-up steps, and as many of the requested steps as fit.
    budget_s, per_step = 150.0, 2.5
    warm = min(args.warmup, 3)
    timed = max(1, min(args.steps, int(budget_s / per_step) - warm))
    n_atoms, n_s, times = oracle_sample_step(batch, per_step, warm + timed)
    times = times[warm:]
    total = sum(times)
    value = n_atoms * timed / total
    sample = (f"{n_s} smallest structure(s) of the workload ({n_atoms} atoms) per step, FP64 explicit-route "
              f"oracle (loss + gradient + Adam), {timed} timed steps")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": timed, "steps_requested": args.steps, "warmup": warm, "ms_per_step": 1e3 * total / timed,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "cpu_all_cores": oracle_all_cores(batch),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU leg

def run_gnep(args):
    import torch
    import torch.distributed as dist

    from paper_2507_00528_gb300 import build as gbuild
    gbuild.build()
    from paper_2507_00528_gb300 import gnep, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # per-rank workload: the same shape, independent structures (weak scaling)
    batch = synth.make_config(2, seed=None if rank == 0 else 20250702 + 1000 * rank)
    n_atoms = batch.n_atoms

    teacher = gnep.GNEP(**MODEL_KW, seed=12)
    dbatch = gnep.DeviceBatch.from_host(batch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nl = teacher.neighbors(dbatch)
    torch.cuda.synchronize()
    nbuild_ms = 1e3 * (time.perf_counter() - t0)
    PR, PA = nl.info()
    teacher.compute_scale(nl)
    scale = teacher.get_scale()
    sizes = batch.sizes()
    y = teacher.teacher_labels(nl, sizes, **LAMBDAS)
    student = gnep.GNEP(**MODEL_KW, seed=11, precision=args.precision)
    student.set_scale(scale)

    n_total = args.warmup + args.steps * args.repeats + 10
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    if world == 1:
        # one captured graph per step: loss + gradient + scheduled Adam
        graph = gnep.TrainGraph(student, nl, y, 1e-3, 1e-5, 2, n_total)
        stream = graph.stream
        run_step = lambda: graph.launch(stream)
    else:
        # data-parallel step: each rank its own 256 structures, the FP64 gradient
        # summed over ranks (NCCL all-reduce) before the identical Adam update
        from paper_2507_00528_gb300 import data_parallel as dp
        cnt = torch.tensor([batch.n_struct, n_atoms], dtype=torch.float64, device="cuda")
        dist.all_reduce(cnt)
        dstep = dp.DataParallelStep(student, nl, y, dp.Counts(batch.n_struct, n_atoms),
                                    dp.Counts(int(cnt[0].item()), int(cnt[1].item())))
        stream = torch.cuda.current_stream()
        run_step = lambda: dstep.step(1e-3, 1e-5, 2, n_total, want_loss=False)
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            run_step()
    torch.cuda.synchronize()
    loss0 = student.loss(nl, y).cpu().numpy().copy()

    # The K timed steps are run `repeats` times, each repeat bracketed by a
    # barrier and a synchronisation, so that the clock sampler sees the load
    # for a few seconds; the line reports the median repeat.
    props = torch.cuda.get_device_properties(local)
    reps_ms = []
    with ClockSampler(_gpu_ident(torch, local)) as clk:
        for _ in range(args.repeats):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            for k in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.zero_()  # evict L2 between steps (outside the timed events)
                    ev[k][0].record(stream)
                    run_step()
                    ev[k][1].record(stream)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            reps_ms.append(sum(a.elapsed_time(b) for a, b in ev))
    if world > 1:
        t = torch.tensor(reps_ms, dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        reps_ms = t.cpu().tolist()
        a = torch.tensor([n_atoms], dtype=torch.float64, device="cuda")
        dist.all_reduce(a)
        atoms_all = a.item()
    else:
        atoms_all = n_atoms
    total_ms = statistics.median(reps_ms)
    value = atoms_all * args.steps / (total_ms / 1e3)
    loss_end = student.loss(nl, y).cpu().numpy().copy()
    student.sync_status()
    clocks = clk.summary()

    # per-kernel durations (CUDA events between launches, eager step)
    stage_ms = {}
    reps = 5
    for _ in range(reps):
        for name, ms in student_profile(student, nl, y, gnep):
            stage_ms[name] = stage_ms.get(name, 0.0) + ms / reps
    roofline = roofline_line(stage_ms, n_atoms, PR, PA, props, clocks, total_ms / args.steps)

    # end to end through the C ABI with host buffers: H2D of the structures and
    # labels from pinned memory, neighbour rebuild, loss + gradient, Adam, D2H loss
    e2e = run_e2e(student, nl, batch, y, args, gnep, torch)

    # the narrower network modes beside the headline: their step time and the
    # force difference from the FP32 form at identical parameters
    other_modes = {}
    if world == 1:
        for mode in [m for m in ("bf16", "tf32") if m != args.precision]:
            other_modes[mode] = time_mode(mode, nl, y, scale, args, flush, torch, gnep, total_ms / args.steps,
                                          args.precision)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        n_s_atoms, n_s, times = oracle_sample_step(batch, args.cpu_seconds, 1)
        cpu = {"value": n_s_atoms / times[0], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n_s} smallest structures of the workload ({n_s_atoms} atoms), one full step "
                         f"(FP64 loss + explicit-route gradient + Adam), {times[0]:.1f} s",
               "all_cores": oracle_all_cores(batch)}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": dict(WORKLOAD, atoms_per_step_per_gpu=n_atoms, radial_pairs=PR, angular_pairs=PA,
                       graph=world == 1, precision=args.precision, l2="flushed between steps (256 MB write)",
                       parallelism=f"dp{world}" + (" (FP64 gradient all-reduce per step)" if world > 1 else ""),
                       neighbor_build_ms=round(nbuild_ms, 3)),
        "repeats": {"count": args.repeats, "ms_per_step": [round(r / args.steps, 5) for r in reps_ms],
                    "reported": "median repeat"},
        "roofline": roofline,
        "kernel_ms": {k: round(v, 5) for k, v in stage_ms.items()},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "other_modes": other_modes,
        # kernels of the captured step (its gradient reduction and Adam are one
        # kernel), or of the eager data-parallel step
        "gpu_launches": args.steps * (graph.kernel_count() if world == 1 else
                                      sum(1 for k in stage_ms if not k.startswith("memset"))),
        "clocks": clocks,
        "loss": {"after_warmup": loss0.tolist(), "end": loss_end.tolist()},
        "source_sha": csrc_sha(),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


DTYPES = {
    "fp32": "f32 (FP32 geometry and network; descriptor, force, tangent and c-gradient contractions as "
            "split-TF32 tensor-core products with FP32-level error; FP64 cross-atom sums)",
    "tf32": "tf32 network (tcgen05, FP32 accumulation); otherwise as the f32 form",
    "bf16": "bf16 network (tcgen05, FP32 accumulation); otherwise as the f32 form",
}


def roofline_line(stage_ms, n_atoms, PR, PA, props, clocks, step_ms):
    """Roofline of the dominant kernel (the longest launch) on the FP32-ALU
    bound: the work model's FLOPs per launch over the launch's measured time,
    against the FP32 peak SMs x 128 lanes x 2 FLOP x clock (no FP32 figure is
    measured), at the maximum clock and at the median clock of the run.  The
    kernel's compulsory bytes against the measured copy bandwidth, and the
    whole step's FLOPs and compulsory bytes per atom, stand beside it."""
    fl = work_model_flops(N=n_atoms, PR=PR, PA=PA)
    by = algo_bytes(N=n_atoms, PR=PR, PA=PA)
    kernels = {k: v for k, v in stage_ms.items() if k in fl}
    dom = max(kernels, key=kernels.get)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sm_run = clocks.get("sm_mhz") or sm_max
    fp32 = lambda mhz: props.multi_processor_count * 128 * 2 * mhz * 1e6 / 1e12  # TFLOP/s
    hbm = peaks.get("hbm_gbs")
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if hbm else "fallback 6.8 TB/s (of fallback)"
    hbm = float(hbm or 6800.0)
    sec = stage_ms[dom] / 1e3
    achieved = fl[dom] / sec / 1e12
    step_flops = sum(fl.values())
    step_bytes = sum(by.values())
    return {
        "bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp32(sm_max), "unit": "TFLOP/s",
        "frac": achieved / fp32(sm_max), "traffic": committed_traffic(dom),
        "peak_source": (f"FP32 peak derived as {props.multi_processor_count} SMs x 128 lanes x 2 FLOP x "
                        f"{sm_max:.0f} MHz (maximum SM clock); no FP32 figure is measured"),
        "peak_at_run_clock": {"sm_mhz": sm_run, "peak": fp32(sm_run), "frac": achieved / fp32(sm_run)},
        "kernel_ms": stage_ms[dom], "kernel_algo_flops": fl[dom],
        "hbm": {"kernel_compulsory_bytes": by[dom], "achieved_gbs": by[dom] / sec / 1e9, "peak_gbs": hbm,
                "frac": by[dom] / sec / 1e9 / hbm, "peak_source": hbm_src},
        "step": {"algo_gflop": step_flops / 1e9, "achieved_tflops": step_flops / (step_ms / 1e3) / 1e12,
                 "frac": step_flops / (step_ms / 1e3) / 1e12 / fp32(sm_max),
                 "compulsory_bytes_per_atom": step_bytes / n_atoms,
                 "compulsory_bytes_per_atom_over_2kb": step_bytes / n_atoms / 2048.0},
        "per_kernel": {k: {"ms": round(stage_ms[k], 5), "tflops": round(fl[k] / (stage_ms[k] / 1e3) / 1e12, 3),
                           "frac": round(fl[k] / (stage_ms[k] / 1e3) / 1e12 / fp32(sm_max), 4)}
                       for k in kernels},
    }


def time_mode(mode, nl, y, scale, args, flush, torch, gnep, head_ms, head_mode):
    """Step time of another network mode (graph replays, L2 flushed between
    steps) and its forces' relative RMS difference from the headline form's."""
    m = gnep.GNEP(**MODEL_KW, seed=11, precision=mode)
    m.set_scale(scale)
    gr = gnep.TrainGraph(m, nl, y, 1e-3, 1e-5, 2, 10 ** 6)
    k = min(args.steps, 100)
    for _ in range(args.warmup):
        gr.launch(gr.stream)
    reps = []
    for _ in range(3):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        torch.cuda.synchronize()
        for q in range(k):
            with torch.cuda.stream(gr.stream):
                flush.zero_()
                ev[q][0].record(gr.stream)
                gr.launch(gr.stream)
                ev[q][1].record(gr.stream)
        torch.cuda.synchronize()
        reps.append(sum(a.elapsed_time(b) for a, b in ev) / k)
    ms = statistics.median(reps)
    probe = gnep.GNEP(**MODEL_KW, seed=11, precision=mode)
    probe.set_scale(scale)
    F_mode = probe.forward(nl)[2].double().cpu().numpy()
    probe.set_precision(head_mode)
    F_ref = probe.forward(nl)[2].double().cpu().numpy()
    m.sync_status()
    return {"value": nl.n_atoms / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": k, "repeats": 3,
            "speedup_over_headline": head_ms / ms, "dtype": DTYPES[mode],
            f"force_rel_rms_vs_{head_mode}_form": float(np.linalg.norm(F_mode - F_ref) / np.linalg.norm(F_ref))}


def student_profile(student, nl, y, gnep):
    import ctypes as C
    L = gnep._lib.load()
    ms = (C.c_float * 64)()
    n = C.c_int32()
    yc = y.c()
    gnep.check(L.gnep_profile_step(student.h, nl.h, C.byref(yc), ms, 64, C.byref(n), gnep._stream()))
    return [(L.gnep_profile_stage_name(i).decode(), ms[i]) for i in range(n.value)]


def run_e2e(student, nl, batch, y, args, gnep, torch):
    """End to end through the C ABI with host buffers, pipelined as a training
    loop with a data loader would run it: step k's loss + gradient + Adam run on
    one stream while step k+1's structures go to the device and its neighbour
    lists are rebuilt on a second stream, into the other of two neighbour lists
    (a list is rebuilt only after the step that read it has finished).  Every
    step's H2D of structures and labels, rebuild, loss + gradient, Adam and D2H
    of the loss lie inside the timed region."""
    import ctypes as C
    L = gnep._lib.load()
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_off = pin(batch.struct_off.astype(np.int32))
    h_pos = pin(batch.pos.astype(np.float64))
    h_typ = pin(batch.types.astype(np.int32))
    h_cell = pin(batch.cell.astype(np.float64))
    h_e = y.energy.cpu().pin_memory()
    h_f = y.force.cpu().pin_memory()
    h_v = y.virial.cpu().pin_memory()
    h_loss = torch.zeros(4, dtype=torch.float64).pin_memory()
    d_loss = torch.zeros(4, dtype=torch.float64, device="cuda")
    cb = gnep._lib.Batch(batch.n_struct, batch.n_atoms, h_off.data_ptr(), h_pos.data_ptr(), h_typ.data_ptr(),
                         h_cell.data_ptr())
    yc = gnep._lib.Labels(h_e.data_ptr(), h_f.data_ptr(), h_v.data_ptr(), y.lambda_e, y.lambda_f, y.lambda_v,
                          y.lambda_l2, y.loss_form)
    nls = [nl, student.neighbors(gnep.DeviceBatch.from_host(batch))]
    s_train, s_load = torch.cuda.Stream(), torch.cuda.Stream()
    st, sl = C.c_void_p(s_train.cuda_stream), C.c_void_p(s_load.cuda_stream)
    done = [torch.cuda.Event(), torch.cuda.Event()]  # step that last read list 0 / 1 has finished
    steps = max(3, min(args.steps, 100))

    def load(k):  # structures of step k to the device, lists rebuilt into nls[k % 2]
        s_load.wait_event(done[k % 2])
        gnep.check(L.gnep_rebuild_neighbors(student.h, C.byref(cb), nls[k % 2].h, sl))

    def train(k):  # loss + gradient + Adam of step k on nls[k % 2], loss back to the host
        gnep.check(L.gnep_loss_grad(student.h, nls[k % 2].h, C.byref(yc), C.c_void_p(d_loss.data_ptr()), None, st))
        gnep.check(L.gnep_adam_step(student.h, 1e-4, 0.9, 0.999, 1e-8, 0.0, st))
        with torch.cuda.stream(s_train):
            h_loss.copy_(d_loss, non_blocking=True)
            done[k % 2].record(s_train)

    for e in done:
        e.record(s_train)
    load(0)
    train(0)
    load(1)
    torch.cuda.synchronize()
    reps = []
    k = 1
    for _ in range(3):  # three timed loops of `steps` steps; the median is reported
        t0 = time.perf_counter()
        for _ in range(steps):
            train(k)      # runs on the device while the host rebuilds the next list
            load(k + 1)
            done[(k - 1) % 2].synchronize()  # step k-1's loss is on the host
            k += 1
        s_train.synchronize()
        reps.append((time.perf_counter() - t0) / steps)
    dt = statistics.median(reps)
    assert np.isfinite(h_loss.numpy()).all()
    h2d = sum(t.numel() * t.element_size() for t in (h_off, h_pos, h_typ, h_cell, h_e, h_f, h_v))
    return {"value": batch.n_atoms / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(h_loss.numel() * 8), "ms_per_step": 1e3 * dt, "steps": steps,
            "repeats_ms_per_step": [round(1e3 * r, 4) for r in reps], "reported": "median of 3 timed loops",
            "includes": "H2D structures+labels (pinned), neighbour rebuild, loss+gradient, Adam, D2H loss; "
                        "the next step's H2D + rebuild overlap the current step on a second stream"}


# ----------------------------------------------------------- workload reports
#
# Two further measurements, outside the headline line:
#   --report precision  the 4,000-structure workload (100-300 atoms, n_max 8/8,
#                       basis 12/12, 3-body, 100 hidden neurons): E/F/V and
#                       gradient errors of each network mode against the FP64
#                       oracle on sampled structures, and training throughput
#                       of each mode over one pass of 256-structure batches.
#   --report epoch      the 10,000-structure workload (64-512 atoms, 4-body,
#                       100 hidden): graph-captured epochs of 256-structure
#                       batches in FP32 and BF16, with the force and energy
#                       RMSE on a held-out batch after each epoch.

CFG4_KW = dict(n_max=(8, 8), basis=(12, 12), hidden=100, four_body=False)
CFG5_KW = dict(n_max=(8, 8), basis=(12, 12), hidden=100, four_body=True)


def _chunks_parallel(cfg_id, idx):
    """Workload chunks from a spawn pool (started before any CUDA use)."""
    import multiprocessing as mp
    from paper_2507_00528_gb300 import synth
    idx = list(idx)
    workers = max(1, min(len(idx), (os.cpu_count() or 2) - 1, 32))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.starmap(synth.config_chunk, [(cfg_id, c) for c in idx])


def _gpu_ident(torch, dev=0):
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "") or "")
    return ("GPU-" + uuid) if uuid and not uuid.startswith("GPU-") else (uuid or str(dev))


def report_precision(args):
    from paper_2507_00528_gb300 import synth
    t_gen = time.perf_counter()
    chunks = _chunks_parallel(4, range(synth.n_chunks(4)))
    t_gen = time.perf_counter() - t_gen
    import torch
    import oracle as O
    from paper_2507_00528_gb300 import build as gbuild
    gbuild.build()
    from paper_2507_00528_gb300 import gnep
    cfg = O.Cfg(nq_r=9, nq_a=9, k_r=13, k_a=13, hidden=100, four_body=False)
    T = synth.uniform_params(cfg.n_params, 12)
    P = synth.uniform_params(cfg.n_params, 11)
    teacher = gnep.GNEP(**CFG4_KW, seed=12)
    teacher.set_params(torch.from_numpy(T))
    nls = [teacher.neighbors(gnep.DeviceBatch.from_host(b)) for b in chunks]
    teacher.compute_scale(nls[0])
    scale = teacher.get_scale().cpu().numpy()
    s64, T64, P64 = scale.astype(np.float64), T.astype(np.float64), P.astype(np.float64)
    # oracle sample: forward on 4 structures, gradient on 2
    sample_f = chunks[0].subset([0, 1, 2, 3])
    sample_g = chunks[0].subset([0, 1])
    t0 = time.perf_counter()
    ref_f = O.forward(cfg, P64, s64, sample_f)
    y_g = O.teacher_labels(cfg, T64, s64, sample_g, **LAMBDAS)
    y_g.force = y_g.force.astype(np.float32).astype(np.float64)
    _, ref_g = O.loss_grad(cfg, P64, s64, sample_g, y_g)
    t_oracle = time.perf_counter() - t0
    student = gnep.GNEP(**CFG4_KW, seed=11)
    student.set_params(torch.from_numpy(P))
    student.set_scale(torch.from_numpy(scale))
    nl_f = student.neighbors(gnep.DeviceBatch.from_host(sample_f))
    nl_g = student.neighbors(gnep.DeviceBatch.from_host(sample_g))
    yg = gnep.Labels(torch.tensor(y_g.energy, device="cuda"),
                     torch.tensor(y_g.force, dtype=torch.float32, device="cuda").contiguous(),
                     torch.tensor(y_g.virial, device="cuda").contiguous(), **LAMBDAS)
    rel = lambda a, b: float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))
    errors = {}
    for mode in ("fp32", "tf32", "bf16"):
        student.set_precision(mode)
        Ea, Es, F, W = (t.double().cpu().numpy() for t in student.forward(nl_f))
        _, g = student.loss_grad(nl_g, yg)
        g = g.double().cpu().numpy()
        errors[mode] = {"energy_per_atom_rel_l2": rel(Ea, ref_f[0]), "force_rel_rms": rel(F, ref_f[2]),
                        "virial_rel_rms": rel(W, ref_f[3]), "gradient_rel_l2": rel(g, ref_g),
                        "gradient_max_abs_over_max": float(np.abs(g - ref_g).max() / np.abs(ref_g).max())}
    # throughput: one pass over all 256-structure batches per mode, labels from the teacher
    ys = [teacher.teacher_labels(nl, b.sizes(), **LAMBDAS) for nl, b in zip(nls, chunks)]
    n_atoms = sum(b.n_atoms for b in chunks)
    thr, pass_ms = {}, {}
    clk_all = {}
    for mode in ("fp32", "tf32", "bf16"):
        student.set_precision(mode)
        student.set_params(torch.from_numpy(P))
        graphs = [gnep.TrainGraph(student, nl, y, 1e-3, 1e-5, len(nls), 4 * len(nls)) for nl, y in zip(nls, ys)]
        for gr in graphs:  # warm-up pass
            gr.launch()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(_gpu_ident(torch)) as clk:
            e0.record()
            for _ in range(3):
                for gr in graphs:
                    gr.launch()
            e1.record()
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        pass_ms[mode] = ms
        thr[mode] = n_atoms / (ms / 1e3)
        clk_all[mode] = clk.summary()
        student.sync_status()
        del graphs
    line = {"report": "precision", "workload": "sbte_4000_structures_100-300_atoms_nmax8_basis12_lmax4_h100",
            "n_struct": sum(b.n_struct for b in chunks), "n_atoms": n_atoms, "batches": len(chunks),
            "errors_vs_fp64_oracle": errors,
            "oracle_sample": {"forward": f"4 structures ({sample_f.n_atoms} atoms)",
                              "gradient": f"2 structures ({sample_g.n_atoms} atoms)", "seconds": round(t_oracle, 1)},
            "train_pass_ms": pass_ms, "atoms_per_s": thr, "clocks": clk_all,
            "generation_s": round(t_gen, 1), "source_sha": csrc_sha()}
    print(json.dumps(line), flush=True)


def report_epoch(args):
    from paper_2507_00528_gb300 import synth
    t_gen = time.perf_counter()
    chunks = _chunks_parallel(5, range(synth.n_chunks(5)))
    t_gen = time.perf_counter() - t_gen
    import torch
    from paper_2507_00528_gb300 import build as gbuild
    gbuild.build()
    from paper_2507_00528_gb300 import gnep
    teacher = gnep.GNEP(**CFG5_KW, seed=12)
    t0 = time.perf_counter()
    nls = [teacher.neighbors(gnep.DeviceBatch.from_host(b)) for b in chunks]
    torch.cuda.synchronize()
    t_nl = time.perf_counter() - t0
    teacher.compute_scale(nls[0])
    scale = teacher.get_scale()
    ys = [teacher.teacher_labels(nl, b.sizes(), **LAMBDAS) for nl, b in zip(nls, chunks)]
    train = list(range(len(chunks) - 1))  # the last batch is held out
    test = len(chunks) - 1
    n_train_atoms = sum(chunks[c].n_atoms for c in train)
    epochs = args.epochs
    F_test = ys[test].force.double().cpu().numpy()
    E_test = ys[test].energy.cpu().numpy()
    sizes_test = chunks[test].sizes()
    out = {}
    for mode in ("fp32", "bf16"):
        student = gnep.GNEP(**CFG5_KW, seed=11, precision=mode)
        student.set_scale(scale)
        graphs = [gnep.TrainGraph(student, nls[c], ys[c], 2e-3, 2e-5, len(train), epochs * len(train))
                  for c in train]
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(epochs)]
        frmse, ermse = [], []
        torch.cuda.synchronize()
        with ClockSampler(_gpu_ident(torch)) as clk:
            for k in range(epochs):
                ev[k][0].record()
                for gr in graphs:
                    gr.launch()
                ev[k][1].record()
                _, Es, F, _ = student.forward(nls[test])
                frmse.append(float(np.sqrt(np.mean((F.double().cpu().numpy() - F_test) ** 2))))
                ermse.append(float(np.sqrt(np.mean((Es.cpu().numpy() / sizes_test - E_test) ** 2))))
            torch.cuda.synchronize()
        student.sync_status()
        ms = [a.elapsed_time(b) for a, b in ev]
        med = statistics.median(ms)
        out[mode] = {"epoch_ms": [round(x, 3) for x in ms], "epoch_ms_median": med,
                     "atoms_per_s": n_train_atoms / (med / 1e3),
                     "force_rmse_test_per_epoch": frmse, "energy_rmse_test_per_epoch": ermse,
                     "clocks": clk.summary()}
        del graphs
    line = {"report": "epoch", "workload": "sbte_10000_structures_64-512_atoms_nmax8_basis12_lmax4_4body_h100",
            "n_struct": sum(b.n_struct for b in chunks), "n_atoms": sum(b.n_atoms for b in chunks),
            "batches": len(chunks), "train_batches": len(train), "train_atoms_per_epoch": n_train_atoms,
            "held_out": f"batch {test} ({chunks[test].n_struct} structures, {chunks[test].n_atoms} atoms)",
            "epochs": epochs, "lr": "Eq. 17, 2e-3 -> 2e-5, warm-up one epoch", "modes": out,
            "neighbor_build_s": round(t_nl, 2), "generation_s": round(t_gen, 1), "source_sha": csrc_sha()}
    print(json.dumps(line), flush=True)


def report_batch_size(args):
    """Batch-size / epoch-budget study (the paper's experimental axis, on
    synthetic data): the same student trained for a fixed number of epochs over
    the 256-structure workload split into batches of B structures, with the
    Eq. 17 schedule over the whole run; final training loss, held-out force and
    energy RMSE, and wall time per B, with the steps of an epoch captured as
    one graph and, for comparison, as one graph per step (the same training
    bit for bit, checked)."""
    from paper_2507_00528_gb300 import synth
    import torch
    from paper_2507_00528_gb300 import build as gbuild
    gbuild.build()
    from paper_2507_00528_gb300 import gnep
    train = synth.make_config(2)
    test = synth.make_config(2, seed=20250702 + 7, n_struct=32)
    teacher = gnep.GNEP(**MODEL_KW, seed=12)
    nl_all = teacher.neighbors(gnep.DeviceBatch.from_host(train))
    teacher.compute_scale(nl_all)
    scale = teacher.get_scale()
    nl_te = teacher.neighbors(gnep.DeviceBatch.from_host(test))
    y_te = teacher.teacher_labels(nl_te, test.sizes(), **LAMBDAS)
    F_te = y_te.force.double().cpu().numpy()
    E_te = y_te.energy.cpu().numpy()
    order = np.random.default_rng(5).permutation(train.n_struct)  # fixed batch composition
    epochs = args.epochs
    out = {}
    for B in [int(b) for b in args.study_batches.split(",")]:
        groups = [order[k:k + B] for k in range(0, train.n_struct, B)]
        subs = [train.subset(sorted(g)) for g in groups]
        nls = [teacher.neighbors(gnep.DeviceBatch.from_host(b)) for b in subs]
        if args.radial_beside:
            for nl in nls:
                nl.set_tuning({"radial_beside": args.radial_beside})
        ys = [teacher.teacher_labels(nl, b.sizes(), **LAMBDAS) for nl, b in zip(nls, subs)]
        n_steps = epochs * len(nls)

        def run_training(epoch_graph):
            # one graph per epoch (all its steps), or one graph per step
            student = gnep.GNEP(**MODEL_KW, seed=11, precision=args.precision)
            student.set_scale(scale)
            if epoch_graph:
                graphs = [gnep.TrainGraph(student, nls, ys, 2e-3, 2e-5, len(nls), n_steps)]
            else:
                graphs = [gnep.TrainGraph(student, nl, y, 2e-3, 2e-5, len(nls), n_steps) for nl, y in zip(nls, ys)]
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(epochs):
                for gr in graphs:
                    gr.launch()
            e1.record()
            torch.cuda.synchronize()
            student.sync_status()
            for gr in graphs:
                gr.close()
            return student, e0.elapsed_time(e1)

        per_step, ms_step = run_training(False)
        student, ms = run_training(True)
        assert torch.equal(per_step.get_params(), student.get_params())  # the same training, bit for bit
        full = student.loss(nl_all, teacher.teacher_labels(nl_all, train.sizes(), **LAMBDAS)).cpu().numpy()
        _, Es, F, _ = student.forward(nl_te)
        out[str(B)] = {"steps": n_steps, "train_ms": round(ms, 2), "ms_per_step": round(ms / n_steps, 4),
                       "ms_per_step_graph_per_step": round(ms_step / n_steps, 4),
                       "train_loss_full_batch": float(full[0]),
                       "test_force_rmse": float(np.sqrt(np.mean((F.double().cpu().numpy() - F_te) ** 2))),
                       "test_energy_rmse": float(np.sqrt(np.mean((Es.cpu().numpy() / test.sizes() - E_te) ** 2)))}
        del nls, ys
    line = {"report": "batch-size", "workload": WORKLOAD["workload"], "epochs": epochs,
            "graphs": "one per epoch (ms_per_step); one per step (ms_per_step_graph_per_step)",
            "precision": args.precision, "lr": "Eq. 17, 2e-3 -> 2e-5, warm-up one epoch",
            "held_out": f"{test.n_struct} structures ({test.n_atoms} atoms) from another seed",
            "radial_beside": args.radial_beside or "default",
            "by_batch_structures": out, "source_sha": csrc_sha()}
    print(json.dumps(line), flush=True)


def report_small_batch(args):
    """Latency of one training step at small batches (the paper trains one
    structure per step by default): for B structures (`--batches`, default 1,
    4, 16 and 64) of the 256-structure workload, the graph-replayed step time (`--steps` replays
    after `--warmup`) and each kernel's time from the library's per-stage
    events, with their sum beside the step; then the step time with each
    radial lane count and each network tile size forced (the others at their
    defaults), to check the default launch-shape rule."""
    import torch
    from paper_2507_00528_gb300 import build as gbuild
    gbuild.build()
    from paper_2507_00528_gb300 import gnep, synth
    train = synth.make_config(2)
    teacher = gnep.GNEP(**MODEL_KW, seed=12)
    nl_all = teacher.neighbors(gnep.DeviceBatch.from_host(train))
    teacher.compute_scale(nl_all)
    scale = teacher.get_scale()
    order = np.random.default_rng(5).permutation(train.n_struct)
    out = {}
    for B in [int(b) for b in args.batches.split(",")]:
        sub = train.subset(sorted(order[:B]))
        nl = teacher.neighbors(gnep.DeviceBatch.from_host(sub))
        y = teacher.teacher_labels(nl, sub.sizes(), **LAMBDAS)
        student = gnep.GNEP(**MODEL_KW, seed=11, precision=args.precision)
        student.set_scale(scale)

        def graph_ms():
            gr = gnep.TrainGraph(student, nl, y, 1e-3, 1e-5, 10, args.steps + args.warmup)
            for _ in range(args.warmup):
                gr.launch()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                gr.launch()
            e1.record()
            torch.cuda.synchronize()
            gr.close()
            return e0.elapsed_time(e1) / args.steps

        default = nl.tuning()
        variants = {}
        for key, vals in (("radial_lanes", (4, 8, 16)), ("net_tile_atoms", (32, 128)), ("radial_beside", (1, 2))):
            for v in vals:
                nl.set_tuning({key: v})
                variants[f"{key}={v}"] = round(graph_ms(), 4)
        nl.set_tuning(None)
        step_ms = graph_ms()
        prof = {}
        for _ in range(5):
            for k, v in student_profile(student, nl, y, gnep):
                prof[k] = prof.get(k, 0.0) + v / 5
        student.sync_status()
        out[str(B)] = {"atoms": int(sub.n_atoms), "ms_per_step": round(step_ms, 4),
                       "default_shapes": {k: default[k] for k in ("radial_lanes", "net_tile_atoms", "radial_beside")},
                       "forced_shapes_ms_per_step": variants,
                       "stage_ms": {k: round(v, 4) for k, v in prof.items()},
                       "stage_sum_ms": round(sum(prof.values()), 4)}
    print(json.dumps({"report": "small-batch", "workload": WORKLOAD["workload"], "precision": args.precision,
                      "steps": args.steps, "by_batch_structures": out, "source_sha": csrc_sha()}), flush=True)


def report_lmax(args):
    """Angular degrees above 4 (App. B, B5-B8): the training step on the
    256-structure workload with n_max 4/4, basis 8/8 and 30 hidden neurons at
    l_max 4 (3-body), 6 (3-body) and 8 (4-body), the compiled shapes of the
    higher degrees, in the FP32 form: the graph-replayed step time (`--steps`
    replays after `--warmup`; the step's data exceed L2), atoms/s, each
    kernel's time from the library's per-stage events, and the work model's
    FLOPs of the step against the FP32 peak."""
    import torch
    from paper_2507_00528_gb300 import build as gbuild
    gbuild.build()
    from paper_2507_00528_gb300 import gnep, synth
    batch = synth.make_config(2)
    props = torch.cuda.get_device_properties(0)
    sm_max = float(measured_peaks().get("sm_max_mhz", 2070.0))
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    out = {}
    for lmax, fb in ((4, False), (6, False), (8, True)):
        kw = dict(n_max=(4, 4), basis=(8, 8), l_max=lmax, four_body=fb, hidden=30)
        teacher = gnep.GNEP(**kw, seed=12)
        nl = teacher.neighbors(gnep.DeviceBatch.from_host(batch))
        PR, PA = nl.info()
        teacher.compute_scale(nl)
        y = teacher.teacher_labels(nl, batch.sizes(), **LAMBDAS)
        student = gnep.GNEP(**kw, seed=11)
        student.set_scale(teacher.get_scale())
        gr = gnep.TrainGraph(student, nl, y, 1e-3, 1e-5, 10, args.steps + args.warmup + 10)
        for _ in range(args.warmup):
            gr.launch()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            gr.launch()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        kernels = gr.kernel_count()
        gr.close()
        prof = {}
        for _ in range(5):
            for k, v in student_profile(student, nl, y, gnep):
                prof[k] = prof.get(k, 0.0) + v / 5
        student.sync_status()
        fl = work_model_flops(nqr=5, kr=9, nqa=5, ka=9, H=30, fb=fb, N=batch.n_atoms, PR=PR, PA=PA,
                              L=lmax * (lmax + 2), lmax=lmax)
        step_fl = sum(fl.values())
        out[str(lmax)] = {"four_body": fb, "n_desc": student.n_des, "n_params": student.n_params,
                          "ms_per_step": round(ms, 4), "atoms_per_s": batch.n_atoms / (ms / 1e3),
                          "kernels_per_step": kernels, "stage_ms": {k: round(v, 4) for k, v in prof.items()},
                          "work_model_gflop": round(step_fl / 1e9, 3),
                          "work_model_tflops": round(step_fl / (ms / 1e3) / 1e12, 2),
                          "fp32_frac": round(step_fl / (ms / 1e3) / 1e12 / peak, 3)}
        del gr, nl, teacher, student
    print(json.dumps({"report": "lmax", "workload": "sbte_256_structures_32-400_atoms_nmax4_basis8_h30",
                      "precision": "fp32", "steps": args.steps, "n_atoms": batch.n_atoms,
                      "fp32_peak_tflops": round(peak, 2), "by_lmax": out, "source_sha": csrc_sha()}), flush=True)


def report_step(args):
    """A driver for profiler captures: the benchmark model and batch, then
    `--steps` loss + gradient evaluations in `--precision` (no timing, no
    graph), so that a capture sees the step's kernels in order."""
    import torch
    from paper_2507_00528_gb300 import build as gbuild
    gbuild.build()
    from paper_2507_00528_gb300 import gnep, synth
    batch = synth.make_config(2)
    teacher = gnep.GNEP(**MODEL_KW, seed=12)
    nl = teacher.neighbors(gnep.DeviceBatch.from_host(batch))
    teacher.compute_scale(nl)
    y = teacher.teacher_labels(nl, batch.sizes(), **LAMBDAS)
    m = gnep.GNEP(**MODEL_KW, seed=11, precision=args.precision)
    m.set_scale(teacher.get_scale())
    for _ in range(args.steps):
        m.loss_grad(nl, y)
    torch.cuda.synchronize()
    m.sync_status()
    print(json.dumps({"report": "step", "precision": args.precision, "evaluations": args.steps,
                      "n_atoms": batch.n_atoms, "source_sha": csrc_sha()}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gnep", choices=["gnep", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tf32", "bf16"],
                    help="network contractions: the FP32 form (default), or bf16 / tf32 on tensor cores")
    ap.add_argument("--repeats", type=int, default=10,
                    help="times the K timed steps are repeated (the median repeat is reported)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--report", choices=["precision", "epoch", "batch-size", "small-batch", "step", "lmax"],
                    default=None,
                    help="a workload report instead of the headline line")
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batches", default="1,4,16,64",
                    help="small-batch report: batch sizes in structures, comma separated")
    ap.add_argument("--study-batches", default="1,4,16,64,256",
                    help="batch-size report: batch sizes in structures, comma separated")
    ap.add_argument("--radial-beside", type=int, default=0, choices=[0, 1, 2],
                    help="batch-size report: radial sweeps in turn (1) or beside the angular ones (2); 0 = default")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.report == "precision":
        report_precision(args)
    elif args.report == "epoch":
        report_epoch(args)
    elif args.report == "batch-size":
        report_batch_size(args)
    elif args.report == "small-batch":
        report_small_batch(args)
    elif args.report == "step":
        report_step(args)
    elif args.report == "lmax":
        report_lmax(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gnep(args)


if __name__ == "__main__":
    main()
