#!/usr/bin/env python
"""Benchmark of the random-batch MD step on B300 (arXiv 2407.09315 workload).

Default workload: the N = 1,000,000 2:1 electrolyte (333,333 cations +2,
666,666 anions -1, one neutral atom; 4 LJ types, sigma ~ U[0.8, 1.2],
epsilon ~ U[0.5, 1.5]; density 0.2; L = 170.998), alpha = 0.62, P = 200,
r_core = 2.0, r_cut = 3.5, p = 10, dt = 0.001, Berendsen T0 = 1.  One step is
a full velocity-Verlet step: half kick + drift, RBE (mode sampling, structure
factors, force), RBL (cell sort, core list + shell batch pair forces, momentum
correction), half kick + thermostat.

Before timing, the context's tile shapes (cell division, structure-factor tiles,
pair look-up table) are autotuned on the initial state (rbmd_autotune; the chosen
shape is reported under "tiles"; --no-autotune keeps the defaults).

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the context's stream; the L2 cache (126 MB, larger than the 1M-atom working
set) is flushed by writing a 256 MB buffer before every timed step, outside
the timed region.  The FP64 path is timed the same way on the same system.
Per-stage times (and the roofline of the dominant kernel) come from a second
pass of K steps whose step graph records CUDA events between the stages; that
pass runs the stages one after another on one stream, so it is a little slower
than the timed steps, where the RBE structure factors overlap the RBL kernels.
`e2e` times the force step through the C ABI with host buffers
(rbmd_forces_host): positions copied in from pinned host memory, forces copied
back, every step, host wall clock per call.  `fwd_bwd` times the forward energy
and the backward gradients (positions, charges, eps, sigma) of one state, with
the adjoint kernels' stage times and the dominant one's roofline.  The timed
steps include the rebuilds of the step's neighbour candidate lists as they come
(`candidate_rebuilds`).

`cpu_baseline` is the FP64 CPU oracle (the checker, as it stands) on a bounded
sample of the workload, on every host core and on one; --impl reference times it
on every host core, per step, on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms/step and atom-steps/s at 1M atoms (RBE+RBL), FP32 path vs plain FP64 path"
UNIT = "atom-steps/s"
PARAMS = dict(alpha=0.62, r_core=2.0, r_cut=3.5, rbl_p=10, rbe_P=200, coulomb_k=1.0,
              dt=0.001, temperature=1.0, tau_T=0.1, thermostat=1)
L2_FLUSH_BYTES = 256 << 20
WORKLOAD = ["c3"]

# Algorithmic FP32-pipe lane operations per unit of work (each elementary
# function counted as one operation; FMA as one); the roofline's peak is one such
# operation per lane per clock: SMs (read from the device) x 128 lanes x 2032 MHz.
OPS_RHO_PER_ATOM_MODE = 8      # 3 phase IMAD, 1 convert, sin, cos, 2 FMA
OPS_FORCE_PER_ATOM_MODE = 11   # 3 phase IMAD, 1 convert, sin, cos, 2 (g), 3 FMA
OPS_CLASSIFY_PER_NEIGHBOUR = 7  # 3 sub, 3 IMAD, 1 compare
OPS_PHILOX = 80                # 10 rounds x (2 mul.hi + 2 mul.lo + 4 xor/add)
OPS_PAIR = 22                  # r^2, rsqrt, erfc, exp, Coulomb, LJ, accumulate
OPS_RBE_ADJ_PER_ATOM_MODE = 13  # 3 phase IMAD, convert, sin, cos, 2 (g), 3 FMA (force), 2 (potential)
OPS_RBL_ADJ_PER_PAIR = 40       # pair energy and force, eps and sigma derivatives, both atoms
SM_COUNT = [148]                # replaced by the device's count when a GPU is present


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-fwd-bwd", action="store_true")
    ap.add_argument("--fwd-bwd-steps", type=int, default=10)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default tile shapes (the run autotunes them otherwise)")
    ap.add_argument("--pair-table", action="store_true",
                    help="erfc-Coulomb pair terms from the look-up table (RBMD_PAIR_TABLE)")
    ap.add_argument("--cpu-sample", type=int, default=400_000)
    ap.add_argument("--ref-sample", type=int, default=100_000)
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.n is None:
        args.n = w["n"]
    if args.n is None and w.get("replicas"):
        from paper_2407_09315_b300 import synth
        args.n = int(sum(synth.replica_sizes(w["replicas"], w["n_lo"], w["n_hi"], seed=4)))
    PARAMS.update(w["params"])
    if args.pair_table:
        PARAMS["flags"] = PARAMS.get("flags", 0) | 16
    return args


# Workloads: "c3" (default) is the headline 1M-ion 2:1 electrolyte; the others
# are reported with --workload: "c2" 100k 1:1 ions at P = 200, "c4" 10M 1:1 ions
# at P = 500, "c5" a batch of 64 independent 1:1 replicas with N_r log-uniform in
# [2000, 200000] at P = 100 (one context, every kernel covers all replicas),
# "lj001" an LJ fluid at density 0.01 with r_core = 2.5, r_cut = 5, p = 30, RBL
# only (the paper's Sec. 4.2 LJ efficiency runs), "el001" a 1:1 primitive
# electrolyte at density 0.01, r_core = 6, r_cut = 12, coulomb_k = 3.5,
# alpha = 0.362, P = 100 (Sec. 4.2).
WORKLOADS = {
    "c3": dict(n=1_000_000, charges="2:1", n_types=4, density=0.2, params={}),
    "c2": dict(n=100_000, charges="1:1", n_types=1, density=0.2, params={}),
    "c4": dict(n=10_000_000, charges="1:1", n_types=1, density=0.2, params=dict(rbe_P=500)),
    "c5": dict(n=None, replicas=64, n_lo=2000, n_hi=200_000, charges="1:1", n_types=1,
               density=0.2, params=dict(rbe_P=100)),
    "lj001": dict(n=1_000_000, charges="none", n_types=1, density=0.01,
                  params=dict(r_core=2.5, r_cut=5.0, rbl_p=30, flags=4)),
    "el001": dict(n=100_000, charges="1:1", n_types=1, density=0.01,
                  params=dict(r_core=6.0, r_cut=12.0, rbl_p=30, rbe_P=100, alpha=0.362,
                              coulomb_k=3.5)),
}


class Batch:
    """The systems of one context (one, or the replicas of a batched workload)."""

    def __init__(self, systems):
        import numpy as np
        self.systems = systems
        self.R = len(systems)
        self.n = int(sum(s.n for s in systems))
        self.sizes = [s.n for s in systems]
        self.L = [s.L for s in systems] if self.R > 1 else systems[0].L
        cat = lambda k: np.concatenate([getattr(s, k) for s in systems])
        self.u, self.q, self.types, self.v = cat("u"), cat("q"), cat("types"), cat("v")
        self.x = np.concatenate([s.x for s in systems])
        self.eps, self.sig = systems[0].eps, systems[0].sig
        # number density of every replica (all are made at the workload's density)
        self.density = systems[0].n / systems[0].L ** 3


def make_system(n, seed, workload="c3", max_replicas=None):
    from paper_2407_09315_b300 import synth
    w = WORKLOADS[workload]
    if w.get("replicas"):
        sizes = synth.replica_sizes(w["replicas"], w["n_lo"], w["n_hi"], seed=4)
        if max_replicas is not None:
            sizes = sizes[:max_replicas]  # replica r depends on r alone
        return Batch(synth.replicas(sizes, seed=seed, density=w["density"],
                                    charges=w["charges"], n_types=w["n_types"]))
    if w["charges"] == "none":
        s = synth.electrolyte(n, seed=seed, charges="1:1", n_types=w["n_types"],
                              density=w["density"])
        s.q = s.q * 0.0
        return Batch([s])
    return Batch([synth.electrolyte(n, seed=seed, charges=w["charges"], n_types=w["n_types"],
                                    density=w["density"])])


def workload_config(args, world, system=None):
    w = WORKLOADS[args.workload]
    kind = {"2:1": "2:1 electrolyte", "1:1": "1:1 electrolyte", "none": "LJ fluid"}[w["charges"]]
    if w.get("replicas"):
        size = ("%d independent replicas, N_r log-uniform in [%d, %d] (%d atoms in all) per GPU"
                % (w["replicas"], w["n_lo"], w["n_hi"], system.n if system else args.n))
    else:
        size = "N=%d per GPU" % args.n
    return {"workload": "%s, %s, density %g, %d LJ type(s), P=%d, p=%d, r_core=%.1f, "
                        "r_cut=%.1f, alpha=%.3f, coulomb_k=%.1f, Berendsen NVT%s"
                        % (kind, size, w["density"], w["n_types"], PARAMS["rbe_P"],
                           PARAMS["rbl_p"], PARAMS["r_core"], PARAMS["r_cut"], PARAMS["alpha"],
                           PARAMS["coulomb_k"], ", RBL only" if PARAMS.get("flags", 0) & 4 else ""),
            "preset": args.workload,
            "n_atoms_per_gpu": system.n if system else args.n,
            "global_atoms": (system.n if system else args.n) * world,
            "replicas_per_gpu": system.R if system else (w.get("replicas") or 1),
            "parallelism": "independent replicas" if world > 1 else "single GPU",
            "l2": "flushed (256 MB write) before every timed step"}


# --------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names[1:], f[5:9]):
                if val.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- ranks
def max_over_ranks(x, dist, device):
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms_per_step):
    """Whole-job throughput of `world` ranks that each process units_per_rank per step,
    timed by the slowest rank."""
    return units_per_rank * world / (ms_per_step * 1e-3)


# --------------------------------------------------------------------------- ours
def make_ctx(system, precision, device):
    import torch
    import paper_2407_09315_b300 as rb

    dt = torch.float64 if precision == rb.FP64 else torch.float32
    extra = {}
    if system.R > 1:
        extra = dict(n_atoms=system.sizes, seed=[2 + r for r in range(system.R)],
                     replica=list(range(system.R)))
    else:
        extra = dict(seed=2)
    ctx = rb.RBMD(torch.from_numpy(system.x).to(device, dt), torch.from_numpy(system.q).to(device, dt),
                  system.eps, system.sig, box_length=system.L, precision=precision,
                  vel=torch.from_numpy(system.v).to(device, dt),
                  types=torch.from_numpy(system.types).to(device), **extra, **PARAMS)
    ctx.set_state_u(system.u, vel=system.v, step=0)
    return ctx


def time_steps(ctx, K, W, flush, profile, timed_rebuilds=None):
    """W warm-up and K timed steps; per-step CUDA-event times and (profile) the
    stage times.  timed_rebuilds (a list): the candidate-list rebuilds of the K
    timed steps are appended to it (counted outside the timed region)."""
    import torch

    stream = torch.cuda.current_stream()
    if profile:
        ctx.profile(True)
    for _ in range(W):
        flush.fill_(1)
        ctx.step(1)
    torch.cuda.synchronize()
    if profile:
        ctx.profile_read(reset=True)
    reb0 = ctx.candidate_rebuilds() if timed_rebuilds is not None else 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    for k in range(K):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        ctx.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    stages = ctx.profile_read(reset=True)[0] if profile else None
    if timed_rebuilds is not None:
        timed_rebuilds.append(ctx.candidate_rebuilds() - reb0)
    return ms, stages


def mean_lists(system):
    """Mean core and shell neighbour counts of a uniform fluid at this density."""
    import math
    n = system.density
    core = n * 4.0 / 3.0 * math.pi * PARAMS["r_core"] ** 3
    shell = n * 4.0 / 3.0 * math.pi * (PARAMS["r_cut"] ** 3 - PARAMS["r_core"] ** 3)
    return core, shell


def captured_traffic(n_atoms):
    """DRAM bytes per launch of the hot kernels, from the committed ncu summary of
    a 200k-atom capture of this workload's recipe, scaled to n_atoms (every
    kernel's traffic grows with the atoms it processes), per stage; {} when a
    kernel source changed since the capture (the counters no longer apply)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "hot_kernels_200k.md")
    try:
        m = re.search(r"```json\n(.*?)\n```", open(path).read(), re.S)
        d = json.loads(m.group(1))
        for name, sha in d["sources_sha256"].items():
            src = os.path.join(ROOT, "paper_2407_09315_b300", "csrc", name)
            if hashlib.sha256(open(src, "rb").read()).hexdigest() != sha:
                return {}
        f = n_atoms / d["atoms"]
        return {k: int(round(v * f)) for k, v in d["traffic_bytes_per_launch"].items()}
    except Exception:
        return {}


def step_stage_names(stages, candidates):
    """Stage times under the names of the kernels that run.  With the step's
    neighbour candidate lists (rbmd_step's default), the cell-sort stage holds the
    gather of the positions into the lists' order and the conditional rebuild, and
    one kernel (k_rbl_vsel) classifies the candidates and draws the batch, so the
    selection stage is empty; without them the cell walk scans (k_rbl_scan) and a
    second kernel selects (k_rbl_select)."""
    if not candidates:
        return dict(stages)
    out = {}
    for k, v in stages.items():
        if k == "rbl_select":
            continue
        out[{"cell_sort": "cand_gather_rebuild", "rbl_scan": "rbl_classify_select"}.get(k, k)] = v
    return out


def roofline(stages_ms_per_step, system, peaks_clock_mhz):
    """Roofline object for the stage with the largest share of the step."""
    N, P, p = system.n, PARAMS["rbe_P"], PARAMS["rbl_p"]
    core, shell = mean_lists(system)
    ops = {
        "rho_partial": N * P * OPS_RHO_PER_ATOM_MODE,
        "rbe_force": N * P * OPS_FORCE_PER_ATOM_MODE,
        "rbl_scan": N * OPS_CLASSIFY_PER_NEIGHBOUR * (core + shell),
        "rbl_select": N * OPS_PHILOX * shell,
        # classification of the in-range neighbours and a priority per shell member
        "rbl_classify_select": N * (OPS_CLASSIFY_PER_NEIGHBOUR * (core + shell) + OPS_PHILOX * shell),
        "rbl_force": N * OPS_PAIR * (core + min(shell, p)),
    }
    ops = {k: v for k, v in ops.items() if stages_ms_per_step.get(k, 0.0) > 0}
    top = max(ops, key=lambda k: stages_ms_per_step.get(k, 0.0))
    t = stages_ms_per_step[top] * 1e-3
    clock = 2032.0 if not peaks_clock_mhz else peaks_clock_mhz
    peak = SM_COUNT[0] * 128 * clock * 1e6 / 1e12  # Top/s, one FP32 lane-op per lane per clock
    achieved = ops[top] / t / 1e12
    cap = captured_traffic(N) if (WORKLOAD[0] == "c3" and system.R == 1) else {}
    traffic = cap.get(top)
    every = {}
    for k, n_ops in ops.items():
        ms = stages_ms_per_step.get(k, 0.0)
        if ms > 0:
            a = n_ops / (ms * 1e-3) / 1e12
            every[k] = {"achieved": round(a, 3), "frac": round(a / peak, 4),
                        "ms_per_launch": round(ms, 4), "traffic": cap.get(k)}
    return {"bound": "alu", "kernel": top, "achieved": round(achieved, 3), "peak": round(peak, 3),
            "unit": "Top/s (FP32-pipe lane ops)", "frac": round(achieved / peak, 4),
            "peak_source": "derived: %d SMs (device) x 128 FP32 lanes x %.0f MHz" % (SM_COUNT[0], clock),
            "traffic": traffic, "ms_per_launch": round(stages_ms_per_step[top], 4),
            "algorithmic_ops_per_launch": ops[top], "every_kernel": every}


def fwd_bwd(ctx, system, K, W, flush, step, clock_mhz):
    """Forward energy (rbmd_energy: RBE + RBL energies and virials, FP64 sums) plus
    backward gradients (rbmd_energy_backward: dE/dr, dE/dq, dE/d eps, dE/d sigma)
    of one state, timed with CUDA events around the two calls (each synchronises),
    then a second pass with stage events for the per-kernel times."""
    import torch

    stream = torch.cuda.current_stream()
    for _ in range(W):
        ctx.energy(step)
        ctx.energy_backward(step)
    torch.cuda.synchronize()
    f_ms, b_ms = [], []
    for k in range(K):
        flush.fill_(k & 0xFF)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ctx.energy(step)
        e1.record(stream)
        ctx.energy_backward(step)
        e2.record(stream)
        torch.cuda.synchronize()
        f_ms.append(e0.elapsed_time(e1))
        b_ms.append(e1.elapsed_time(e2))
    ctx.profile(True)
    ctx.profile_read_grad(reset=True)
    for k in range(K):
        flush.fill_(k & 0xFF)
        ctx.energy(step)
        ctx.energy_backward(step)
    fwd, bwd, calls = ctx.profile_read_grad(reset=True)
    ctx.profile(False)
    fwd = {k: round(v / max(calls[0], 1), 4) for k, v in fwd.items()}
    bwd = {k: round(v / max(calls[1], 1), 4) for k, v in bwd.items()}
    N, P, p = system.n, PARAMS["rbe_P"], PARAMS["rbl_p"]
    core, shell = mean_lists(system)
    ops = {"rbe_adjoint": N * P * OPS_RBE_ADJ_PER_ATOM_MODE,
           "rbl_adjoint": N * OPS_RBL_ADJ_PER_PAIR * (core + min(shell, p))}
    top = max(ops, key=lambda k: bwd.get(k, 0.0))
    peak = SM_COUNT[0] * 128 * clock_mhz * 1e6 / 1e12
    ach = ops[top] / (bwd[top] * 1e-3) / 1e12 if bwd.get(top) else None
    fm, bm = sum(f_ms) / K, sum(b_ms) / K
    return {"ms": round(fm + bm, 4), "forward_ms": round(fm, 4), "backward_ms": round(bm, 4),
            "atom_steps_per_s": N / ((fm + bm) * 1e-3),
            "what": "rbmd_energy + rbmd_energy_backward of one state (gradients w.r.t. "
                    "positions, charges, eps and sigma), CUDA events around each call, L2 "
                    "flushed before each pair",
            "forward_stage_ms": fwd, "backward_stage_ms": bwd,
            "roofline": {"bound": "alu", "kernel": top,
                         "achieved": None if ach is None else round(ach, 3),
                         "peak": round(peak, 3), "unit": "Top/s (FP32-pipe lane ops)",
                         "frac": None if ach is None else round(ach / peak, 4),
                         "algorithmic_ops_per_launch": ops[top],
                         "ms_per_launch": bwd.get(top)}}


def e2e_force_step(ctx, system, K, W, device):
    """Force step through the C ABI with host buffers: positions in, forces out
    (rbmd_forces_host, which overlaps the copies with the kernels)."""
    import torch

    dt = ctx.dtype
    host_pos = torch.from_numpy(system.x).to(dt).pin_memory()
    host_f = torch.empty((system.n, 3), dtype=dt).pin_memory()
    for k in range(W):
        ctx.forces_host(host_pos, out=host_f, step=k)
    torch.cuda.synchronize()
    wall = []
    for k in range(K):
        t0 = time.perf_counter()
        ctx.forces_host(host_pos, out=host_f, step=k)  # returns with the forces on the host
        wall.append(time.perf_counter() - t0)
    ms = 1e3 * sum(wall) / K
    nbytes = 3 * system.n * (8 if dt == torch.float64 else 4)
    return {"value": system.n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "what": "rbmd_forces_host: host pinned positions in (they become the state), "
                    "forces of the step out to pinned host memory; host wall clock per call"}


def oracle_sample(n_sample, seed, workload):
    """The systems the oracle times: a workload system of n_sample atoms, or the
    first replicas of a batched workload up to n_sample atoms."""
    w = WORKLOADS[workload]
    if not w.get("replicas"):
        b = make_system(n_sample, seed, workload)
        return b.systems, b.n
    from paper_2407_09315_b300 import synth
    sizes = synth.replica_sizes(w["replicas"], w["n_lo"], w["n_hi"], seed=4)
    k = 1
    while k < len(sizes) and sizes[:k + 1].sum() <= n_sample:
        k += 1
    b = make_system(n_sample, seed, workload, max_replicas=k)
    return b.systems, b.n


def oracle_forces(systems, step):
    import oracle
    for r, s in enumerate(systems):
        oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, PARAMS["alpha"], PARAMS["coulomb_k"],
                      PARAMS["r_core"], PARAMS["r_cut"], PARAMS["rbl_p"], PARAMS["rbe_P"], 2 + r,
                      step, replica=r if len(systems) > 1 else 0)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(n_sample, seed, workload="c3"):
    """The oracle's force evaluation on a sample of the workload, on every host core
    (its per-atom and per-mode loops in OpenMP threads), and on one core."""
    import oracle
    systems, n = oracle_sample(n_sample, seed, workload)
    cores = host_cores()
    rates = {}
    for th in sorted({cores, 1}, reverse=True):
        oracle.set_threads(th)
        t0 = time.perf_counter()
        oracle_forces(systems, 0)
        rates[th] = (n / (time.perf_counter() - t0), time.perf_counter() - t0)
    oracle.set_threads(1)
    what = ("a %d-atom system" % n if not WORKLOADS[workload].get("replicas") else
            "the first %d replica(s) (%d atoms)" % (len(systems), n))
    return {"value": rates[cores][0], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "one FP64 force evaluation (RBE + RBL + F_corr) of %s of the same "
                      "recipe on %d host threads, %.1f s" % (what, cores, rates[cores][1]),
            "single_core": {"value": rates[1][0], "unit": UNIT, "cores": 1,
                            "seconds": round(rates[1][1], 2)}}


def run_ours(args):
    import torch
    import paper_2407_09315_b300 as rb

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)

    WORKLOAD[0] = args.workload
    SM_COUNT[0] = torch.cuda.get_device_properties(device).multi_processor_count
    system = make_system(args.n, 2 + rank, args.workload)
    args.n = system.n
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(device)[0]
    ctx = make_ctx(system, rb.FP32, device)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()  # the input tensors' blocks: the context keeps its own copies
    footprint = free0 - torch.cuda.mem_get_info(device)[0]
    tiles = {"shape": ctx.tiles(), "autotuned": False}
    if not args.no_autotune:
        t0 = time.perf_counter()
        tiles = {"shape": ctx.autotune(step=0), "autotuned": True,
                 "tuning_s": round(time.perf_counter() - t0, 3)}
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    reb0 = ctx.candidate_rebuilds()
    timed_reb = []
    ms, _ = time_steps(ctx, args.steps, args.warmup, flush, profile=False, timed_rebuilds=timed_reb)
    clk = clocks.stop()
    # rebuilds of the step's neighbour candidate lists inside the warm-up and timed
    # steps (the timed mean includes them as they come)
    rebuilds = ctx.candidate_rebuilds() - reb0
    kernels_per_step = ctx.step_kernel_count()
    # the rebuild kernels of the step graph's conditional node run on rebuild steps only
    rebuild_kernels = ctx.rebuild_kernel_count()
    total_ms = max_over_ranks(sum(ms), dist, device)
    if dist:
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = job_rate(args.n, world, ms_per_step)
    # per-stage times: a second pass of K steps whose graph records CUDA events
    # between the stages (the stages then run one after another on one stream)
    ms_prof, stages = time_steps(ctx, args.steps, 2, flush, profile=True)
    ctx.profile(False)
    stage_ms = step_stage_names({k: v / args.steps for k, v in stages.items()}, rebuilds > 0)

    fb = None
    if not args.skip_fwd_bwd and system.R == 1:
        fb = fwd_bwd(ctx, system, args.fwd_bwd_steps, 2, flush, 0,
                     2032.0 if not clk else clk["sm_max_mhz"])

    e2e = None
    if not args.skip_e2e:
        e2e = e2e_force_step(ctx, system, args.e2e_steps, 2, device)
        if dist:
            e2e["ms_per_step"] = max_over_ranks(e2e["ms_per_step"], dist, device)
            e2e["value"] = job_rate(system.n, world, e2e["ms_per_step"])
    ctx.close()

    fp64 = None
    if not args.skip_fp64:
        c64 = make_ctx(system, rb.FP64, device)
        if args.no_autotune:
            c64.set_tiles(*tiles["shape"][:3])
            c64.set_pair_table(tiles["shape"][3])
            shape64 = tiles["shape"]
        else:
            shape64 = c64.autotune(step=0)  # the FP64 kernels have their own best shape
        ms64, _ = time_steps(c64, args.fp64_steps, 2, flush, profile=False)
        _, st64 = time_steps(c64, args.fp64_steps, 1, flush, profile=True)
        st64 = step_stage_names(st64, c64.candidate_rebuilds() > 0)
        c64.close()
        m64 = sum(ms64) / len(ms64)
        fp64 = {"ms_per_step": round(m64, 4), "atom_steps_per_s": args.n / (m64 * 1e-3),
                "tiles": list(shape64),
                "stage_ms": {k: round(v / args.fp64_steps, 4) for k, v in st64.items()}}

    if rank != 0:
        return
    peak_clock = clk["sm_max_mhz"] if clk else None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "ms_per_step_median": round(statistics.median(ms), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded %s, paper-shaped recipe in synth.py)" % WORKLOADS[args.workload]["charges"].replace("none", "LJ fluid"),
        "config": workload_config(args, world, system),
        "stage_ms_per_step": {k: round(v, 4) for k, v in stage_ms.items()},
        "stage_pass": {"ms_per_step": round(sum(ms_prof) / len(ms_prof), 4),
                       "what": "second pass of K steps with CUDA events between the stages, "
                               "stages serialised on one stream"},
        "roofline": roofline(stage_ms, system, 2032.0),
        "sm_count": SM_COUNT[0],
        "gpu_launches": kernels_per_step * args.steps + rebuild_kernels * timed_reb[0],
        "device_memory_bytes": int(footprint),
        "kernels_per_step": kernels_per_step,
        "rebuild_kernels": {"per_rebuild": rebuild_kernels, "rebuilds_in_timed_steps": timed_reb[0]},
        "candidate_rebuilds": {"in_warmup_and_timed_steps": rebuilds,
                               "steps": args.steps + args.warmup},
        "tiles": dict(tiles, names=["cell_div", "rho_tile", "rho_mode_tile", "pair_table"]),
    }
    if fp64:
        out["fp64"] = fp64
        out["speedup_fp32_over_fp64"] = round(fp64["ms_per_step"] / ms_per_step, 2)
    if e2e:
        out["e2e"] = e2e
    if fb:
        out["fwd_bwd"] = fb
    if clk:
        out["clocks"] = clk
    out["paper_context"] = ("8.20 ms/step nonbonded at N=1e6 (SPC/E water, A100 + 1 CPU core); "
                            "different workload and hardware, not a target")
    if not args.skip_cpu and world == 1:
        out["cpu_baseline"] = cpu_baseline(min(args.cpu_sample, args.n), 2, args.workload)
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    import oracle

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    n_sample = min(args.ref_sample, args.n) if args.n else args.ref_sample
    systems, n = oracle_sample(n_sample, 2, args.workload)
    cores = host_cores()
    oracle.set_threads(cores)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle_forces(systems, k)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    sec = sum(times) / len(times)
    value = n / sec
    what = ("a %d-atom system" % n if not WORKLOADS[args.workload].get("replicas") else
            "the first %d replica(s) (%d atoms)" % (len(systems), n))
    sample = ("one FP64 force evaluation (RBE + RBL + F_corr) per step of %s of the "
              "same recipe on %d host threads" % (what, cores))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded %s, paper-shaped recipe in synth.py)" % WORKLOADS[args.workload]["charges"].replace("none", "LJ fluid"),
           "config": workload_config(args, world),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
