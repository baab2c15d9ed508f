"""Benchmark: atom-steps/s of velocity-Verlet MD with the Tersoff potential, fp64 path and
mixed-precision path, on one GB300 (the paper's speed metric, Sec. 3: N x steps / time).

Workload (default): Tersoff-1989 carbon honeycomb sheet, 500 x 500 rectangular cells =
1,000,000 atoms, bond 1.42 A, periodic in-plane, 20 A periodic length along z, jitter
+-0.02 A, Maxwell-Boltzmann 300 K, NVE, dt = 0.5 fs.  A "step" is one full velocity-Verlet
step: kick/drift, conditional neighbour rebuild, pair pass, gather (F, W, J), half-kick
and the per-step fp64 totals (U, K, J).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line.  Timing: W untimed warm-up steps, then K steps between CUDA events
on the library's stream, bracketed by a barrier and a device synchronise; the per-step
working set (~0.5 GB) exceeds the 129 MB L2, so no flush is needed between steps.
Multi-GPU (torchrun): every rank runs its own independent replica of the workload
("replicas only" -- one MD system does not shard without a halo exchange), the job
value is the sum over ranks divided by the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1610_03343_gb300 import inputs as I  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP64 peak of a GB300 from its unit counts and clock (152 SMs x 2 DFMA/clk/SM x 2 flop x
# 2.07 GHz): context for the measured peak (md_peak_flops), which the roofline uses.
FP64_PEAK_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# iterations per FMA chain of the peak kernels: about 40 ms (fp64) and 30 ms (fp32) a launch
PEAK_ITERS = {"fp64": 20_000, "fp32": 1_000_000}

# Algorithmic flops of the pair pass, counted from the final expressions of the method
# (Eqs. 2-6 and dU_i/dr_ij = 1/2 [(f_C f_R)' - b (f_C f_A)'] u_j - 1/2 f_C f_A b'_j dzeta_ij/dr_ij
#  - 1/2 sum_k f_C f_A b'_k dzeta_ik/dr_ij), not from the kernel: an addition, subtraction or
# multiplication is 1 flop; a division, reciprocal or reciprocal square root 8 (a seed and
# Newton steps); exp, log and a sine-cosine pair 16 each (reduction and a polynomial).  Bonds
# below R (f_C = 1, f_C' = 0: every bond of the crystal and sheet workloads at 300 K).
# Each entry: (what, flops).
EL, DIV = 16, 8
TERSOFF_ALG_PER_BOND = [
    ("r_ij = r_j - r_i", 3), ("|r|^2", 5), ("1/r", DIV), ("r = r^2 (1/r)", 1), ("u_j = r_ij / r", 3),
    ("f_R = A exp(-lambda r)", 2 + EL), ("f_A = B exp(-mu r)", 2 + EL),
    ("(beta zeta)^n = exp(n log(beta zeta))", 2 + 2 * EL), ("b = exp(-log(1 + x) / 2n)", 2 + 2 * EL),
    ("b' = -b x / (2 zeta (1 + x))", 4 + DIV), ("U_i += (f_R - b f_A) / 2", 4),
    ("radial (f_R' - b f_A') / 2", 5), ("P_j = -f_A b'_j / 2", 2), ("dU_i/dr_ij = A_j u_j + V_j", 6),
]
TERSOFF_ALG_PER_UNORDERED_PAIR = [
    ("cos theta = u_j . u_k", 5), ("g = 1 + c^2/d^2 - c^2/(d^2 + (h - cos)^2)", 5 + DIV),
    ("g' = -2 c^2 (h - cos) / (d^2 + (h - cos)^2)^2", 3 + DIV), ("Q = (P_j + P_k) g'", 2),
]
TERSOFF_ALG_PER_ORDERED_PAIR = [
    ("zeta_ij += f_C(r_ik) g", 1), ("dcos/dr_ij = (u_k - cos u_j) / r_ij", 9), ("d_ij += Q dcos/dr_ij", 6),
]
SW_ALG_PER_BOND = [
    ("r_ij, |r|^2, 1/r, r, u_j", 3 + 5 + DIV + 1 + 3), ("1/(r - a sigma)", 1 + DIV),
    ("exp(sigma/(r - a sigma))", 1 + EL), ("E = exp(gamma sigma/(r - a sigma))", 1 + EL), ("dE/dr", 3),
    ("(sigma/r)^p, (sigma/r)^q", 3), ("B (sigma/r)^p - (sigma/r)^q and its r-derivative", 2 + 5),
    ("phi2 / 2", 3), ("dphi2/dr", 6), ("two-body part of dU_i/dr_ij", 4), ("U_i += phi2 / 2", 1),
]
SW_ALG_PER_UNORDERED_PAIR = [
    ("cos, t = cos + 1/3, E_j E_k, U_i += lambda eps t^2 E_j E_k", 10),
    ("2 lambda eps t E_j E_k, lambda eps t^2 (E_j' E_k, E_j E_k')", 7), ("q_j, q_k", 2),
    ("d_j += q_j (u_k - cos u_j) + c_j u_j, and d_k", 36),
]


def pair_flops_algorithmic(kind: int, bonds: float, bond_pairs: float) -> float:
    """Algorithmic flops per atom of the pair pass (the tables above) for a mean of `bonds`
    in-cutoff neighbours and `bond_pairs` ordered bond pairs per atom."""
    if kind == I.MD_TERSOFF:
        per_bond = sum(f for _, f in TERSOFF_ALG_PER_BOND)
        per_pair = sum(f for _, f in TERSOFF_ALG_PER_ORDERED_PAIR) + \
            0.5 * sum(f for _, f in TERSOFF_ALG_PER_UNORDERED_PAIR)
    else:
        per_bond = sum(f for _, f in SW_ALG_PER_BOND)
        per_pair = 0.5 * sum(f for _, f in SW_ALG_PER_UNORDERED_PAIR)
    return per_bond * bonds + per_pair * bond_pairs


def gather_bytes_algorithmic(bonds: float, fused: bool = True, elem: int = 4) -> float:
    """Algorithmic DRAM bytes per atom of one step's gather (the mixed path's largest kernel):
    what it must read and write once each -- its list mask (4), the in-cutoff list entries (4 M)
    and reverse slots (M), the bonds' derivatives dU_i/dr_ij (3 M elem; the partner's dU_j/dr_ji
    is another atom's own row, read once overall), the bond vectors (3 M elem), U_i (8), the
    element (4), the velocity (24 read, 24 written), the force (24 written), and with the next
    step's drift fused in: the position (24 read, 24 written) and the build position (24 read)."""
    b = 4 + 5 * bonds + 6 * elem * bonds + 8 + 4 + 48 + 24
    return b + (72 if fused else 0)

# Instruction model of the fp64 pair pass, from ncu's instruction counters of the current
# kernels (profiles/pair_tersoff_fp64_c_graphene_1M.md, profiles/pair_sw_fp64_si_512k.md):
# per in-cutoff bond and per ordered pair of bonds (j, k != j) of one atom, solved from two
# states each -- Tersoff: the C sheet (3 bonds, 6 ordered pairs; the 3-bond staging the
# autotuner picks there) and Si diamond (4, 12; the 4-bond staging);
# SW: the Si lattice (4, 12) and the crystal after 100 fs at 300 K (5.1028, 21.8819; the
# common-case and full-capacity launches together, at the block of 32 the autotuner picks).
# The SW slot coefficients interpolate the two states: they are not costs of a bond and a
# pair (the per-bond ones come out negative), since the thermal state's warps also mix atoms
# of different bond counts, which the lattice's do not.
#   FLOP: DADD + DMUL + 2 DFMA thread instructions (the fp64 arithmetic that is left: the
#         bond geometry, the radial functions and the fp64 steps of exp, log, 1/r);
#   FP64: fp64-pipe issue slots (smsp__inst_executed_pipe_fp64 x 32);
#   ISSUE: issue slots of all instructions (smsp__inst_executed x 32), most of them the
#         float-pair arithmetic on the fp32 pipe.
TERSOFF_FLOP_PER_BOND, TERSOFF_FLOP_PER_BOND_PAIR = 41.4287, 3.12099
TERSOFF_FP64_PER_BOND, TERSOFF_FP64_PER_BOND_PAIR = 32.1030, 2.52050
TERSOFF_ISSUE_PER_BOND, TERSOFF_ISSUE_PER_BOND_PAIR = 1348.332, 288.810
SW_FLOP_PER_BOND, SW_FLOP_PER_BOND_PAIR = 47.5489, 0.504533
SW_FP64_PER_BOND, SW_FP64_PER_BOND_PAIR = -0.621724, 14.185241
SW_ISSUE_PER_BOND, SW_ISSUE_PER_BOND_PAIR = -2076.496, 1343.6406
# DRAM bytes (read + write) per launch of the current kernels at full size (ncu, one pass):
# the fp64 pair pass (common-case launch) and the step gathers, eager launches (no fused drift)
PAIR_TRAFFIC_BYTES = {"tersoff_c_graphene_1M": 175.08e6}
GATHER_TRAFFIC_BYTES = {"tersoff_c_graphene_1M": 167.58e6}
GATHER_TRAFFIC_NOTE = "ncu, full size, eager step launch (no fused drift: 72 B/atom fewer than the model)"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


def workload(name: str, scale: int = 1):
    if name == "tersoff_c_graphene_1M":
        return I.c_graphene_tersoff(nx=500 // scale, ny=500 // scale), 0.5
    if name == "sw_si_512k":
        return I.si_diamond_sw(n=40 // scale), 1.0
    if name == "tersoff_si_1728":
        return I.si_diamond_tersoff(n=6), 1.0
    if name == "tersoff_si_216k":
        return I.si_diamond_tersoff(n=30 // scale), 1.0
    raise ValueError(name)


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _loop(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([c.strip() for c in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._loop, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 5 + k and r[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def reduce_max_over_ranks(values, world, device):
    """Each value's maximum over the ranks (the slowest rank sets a replica run's time);
    the values themselves for one rank.  device: where the collective's tensor lives (cuda
    for NCCL, cpu for gloo)."""
    if world == 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_value(world, n_atoms, steps, ms):
    """Whole-job atom-steps/s of `world` replicas of n_atoms atoms run for `steps` steps,
    timed by the slowest rank (ms)."""
    return world * n_atoms * steps / (ms / 1e3)


def pair_flops(kind: int, bonds: float, bond_pairs: float) -> float:
    """Counted FP64 flops (DADD + DMUL + 2 DFMA) per atom of the fp64 pair pass for a mean of
    `bonds` in-cutoff neighbours and `bond_pairs` ordered bond pairs (the mean of M (M - 1))."""
    if kind == I.MD_TERSOFF:
        return TERSOFF_FLOP_PER_BOND * bonds + TERSOFF_FLOP_PER_BOND_PAIR * bond_pairs
    return SW_FLOP_PER_BOND * bonds + SW_FLOP_PER_BOND_PAIR * bond_pairs


def pair_slots(kind: int, bonds: float, bond_pairs: float):
    """(fp64-pipe issue slots, all issue slots) per atom of the fp64 pair pass."""
    if kind == I.MD_TERSOFF:
        return (TERSOFF_FP64_PER_BOND * bonds + TERSOFF_FP64_PER_BOND_PAIR * bond_pairs,
                TERSOFF_ISSUE_PER_BOND * bonds + TERSOFF_ISSUE_PER_BOND_PAIR * bond_pairs)
    return (SW_FP64_PER_BOND * bonds + SW_FP64_PER_BOND_PAIR * bond_pairs,
            SW_ISSUE_PER_BOND * bonds + SW_ISSUE_PER_BOND_PAIR * bond_pairs)


def pipe_model(kind: int, bonds: float, bond_pairs: float, n: int, peaks: dict) -> dict:
    """Lower bound on one fp64 pair launch's time from its instruction mix and the measured
    rates of this GPU: the FP64 pipe retires fp64_tflops/2 thread instructions a second (the
    FMA-chain peak, 2 flop per FMA), and the schedulers issue fp32_tflops/64 warp
    instructions a second (the fp32 FMA-chain peak: 32 lanes x 2 flop per issued FMA).  The
    launch cannot be faster than the larger of the two times."""
    s64, sall = pair_slots(kind, bonds, bond_pairs)
    t64 = s64 * n / (peaks["fp64_tflops"] * 1e12 / 2.0)
    tis = sall * n / 32.0 / (peaks["fp32_tflops"] * 1e12 / 64.0)
    return {"fp64_slots_per_atom": round(s64, 3), "issue_slots_per_atom": round(sall, 2),
            "t_fp64_pipe_us": t64 * 1e6, "t_issue_us": tis * 1e6,
            "bound_pipe": "fp64" if t64 >= tis else "issue", "t_model_us": max(t64, tis) * 1e6}


def bond_statistics(pos, box, pbc, rc):
    """Mean number M of neighbours within the cutoff rc per atom and the mean of M (M - 1),
    by minimum image along the periodic axes (a k-d tree over the wrapped positions)."""
    from scipy.spatial import cKDTree
    pos = np.asarray(pos, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    per = np.asarray(pbc) != 0
    x = pos.copy()
    x[:, per] = np.mod(x[:, per], box[per])
    x[:, per] = np.where(x[:, per] >= box[per], 0.0, x[:, per])   # mod can round up to L
    lo = x.min(axis=0)
    size = box.copy()
    # an open axis gets a period long enough that no pair wraps across it
    size[~per] = (x.max(axis=0) - lo)[~per] + 4.0 * rc + 1.0
    x[:, ~per] -= lo[~per]
    pairs = cKDTree(x, boxsize=size).query_pairs(rc, output_type="ndarray")
    m = np.bincount(pairs.ravel(), minlength=x.shape[0]).astype(np.float64)
    return float(m.mean()), float((m * (m - 1.0)).mean())


def kernel_window(md, g, steps, warmup, dt, stream):
    """Per-kernel times of `steps` more steps, right after the timed region, with a CUDA
    event pair around every kernel class of every step (md_set_profiling).  The events are
    nodes of the step graphs and cost time of their own (about 25 us a step on the 1M
    sheet), so the timed region runs without them and this window supplies the kernel
    durations.  Returns md_kernel_times and the window's ms."""
    import torch
    md.md_set_profiling(g.ctx, True)
    g.run(max(1, min(warmup, 8)), dt, record=True)   # captures the graphs with the events
    md.md_set_profiling(g.ctx, True)                 # zero the accumulators (graphs kept)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.run(steps, dt, record=True)
    e1.record(stream)
    torch.cuda.synchronize()
    kt = md.md_kernel_times(g.ctx)
    md.md_set_profiling(g.ctx, False)
    return kt, e0.elapsed_time(e1)


def run_ours(args, rank, world):
    import torch
    from paper_1610_03343_gb300 import md

    torch.cuda.set_device(0 if world == 1 else int(os.environ.get("LOCAL_RANK", rank)))
    sysm, dt = workload(args.workload, args.scale)
    n = sysm.n
    stream = torch.cuda.Stream()
    res = {}
    precs = [(md.MD_FP64, "fp64"), (md.MD_MIXED, "mixed")]
    if args.precision != "both":
        precs = [p for p in precs if p[1] == args.precision]
    for prec, tag in precs:
        g = md.System(sysm.box, sysm.pbc, n, sysm.kind, sysm.params, sysm.mass, precision=prec,
                      stream=stream.cuda_stream)
        g.set_positions(sysm.pos)
        g.set_velocities(sysm.vel)
        if args.eager:
            md.md_set_graph_mode(g.ctx, False)
        f0 = g.compute(want=("f",))["F"].copy()
        # untimed equilibration from the lattice start, so that the tuner and the timed
        # window see the thermal state that dominates a long run (SW silicon gains about
        # one bond per atom in the first ~100 fs)
        if args.equilibrate:
            g.run(args.equilibrate, dt, record=False)
        tuning = None
        if args.pair_block:
            pb = dict(zip(("fp64", "mixed"), (int(v) for v in args.pair_block.split(","))))[tag]
            md.md_set_tuning(g.ctx, pair_block=pb, pair_cap=args.pair_cap)
            tuning = {"pair_block": pb, "pair_cap": md.md_get_tuning(g.ctx).pair_cap, "imposed": True}
        elif not args.no_tune:
            tuning = md.tuning_dict(md.md_autotune(g.ctx, 10))
        # the warm-up captures the step graphs (the timed region replays them)
        g.run(args.warmup, dt, record=True)
        pos_first = g.state()[0] if tag == precs[0][1] else None
        st0 = g.stats()
        rebuilds0, kernels0 = st0.n_rebuilds, st0.kernels_launched
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(torch.cuda.current_device())
        with clocks:
            e0.record(stream)
            ser = g.run(args.steps, dt, record=True)
            e1.record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms = e0.elapsed_time(e1)
        st = g.stats()
        pos_last = g.state()[0] if tag == precs[0][1] else None
        kt, ms_ev = kernel_window(md, g, args.steps, args.warmup, dt, stream)
        res[tag] = dict(ms=ms, kt=kt, f0=f0, clocks=clocks.summary(), stats=st, sys=g, tuning=tuning, series=ser,
                        pos_window=(pos_first, pos_last),
                        ms_events=ms_ev, rebuilds=int(st.n_rebuilds - rebuilds0),
                        launches=int(st.kernels_launched - kernels0)
                        + int(st.kernel_launches_per_rebuild) * int(st.n_rebuilds - rebuilds0))
    # end-to-end through the public API with host buffers (pinned), copies inside the
    # timed region: upload x, v; run K steps; read back the series and the final state
    import torch as _t
    first = next(iter(res))
    if args.no_e2e:
        for tag in res:
            res[tag]["sys"].close()
        return n, dt, res, None, 0, 0, None
    g = res[first]["sys"]
    xs = _t.tensor(np.ascontiguousarray(sysm.pos.T), dtype=_t.float64).pin_memory()
    vs = _t.tensor(np.ascontiguousarray(sysm.vel.T), dtype=_t.float64).pin_memory()
    ser = _t.zeros((args.steps, 5), dtype=_t.float64).pin_memory()
    xo = _t.zeros(3 * n, dtype=_t.float64).pin_memory()
    vo = _t.zeros(3 * n, dtype=_t.float64).pin_memory()
    g.run(args.warmup, dt, record=False)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    md.md_set_positions(g.ctx, xs[0], xs[1], xs[2])
    md.md_set_velocities(g.ctx, vs[0], vs[1], vs[2])
    md.md_run(g.ctx, args.steps, dt, ser)
    md.md_get_state(g.ctx, xo, vo)
    t_e2e = time.perf_counter() - t0
    h2d = 6 * 8 * n
    d2h = 6 * 8 * n + 5 * 8 * args.steps
    mixed_err = None
    if "mixed" in res and "fp64" in res:
        mixed_err = float(np.abs(res["mixed"]["f0"] - res["fp64"]["f0"]).max() / np.abs(res["fp64"]["f0"]).max())
    for tag in res:
        res[tag]["sys"].close()
    return n, dt, res, t_e2e, h2d, d2h, mixed_err


# ---------------------------------------------------------------- NPT leg
def run_npt_leg(args, steps, warmup):
    """The same workload in the paper's benchmark ensemble (Sec. 3: NPT, 300 K, 0 Pa):
    Berendsen thermostat and barostat on the device inside the graph-replayed steps
    (periodic in-plane axes coupled for the sheet, every periodic axis for a crystal).
    Reports atom-steps/s for fp64 and mixed, and where the box and temperature went."""
    import torch
    from paper_1610_03343_gb300 import md

    sysm, dt = workload(args.workload)
    n = sysm.n
    couple = (1, 1, 0) if "graphene" in args.workload else (1, 1, 1)
    cpl = dict(T0=300.0, P0=0.0, tau_T=100.0, tau_P=1000.0, beta=0.01, couple=couple)
    stream = torch.cuda.Stream()
    out = {"coupling": {k: (list(v) if isinstance(v, tuple) else v) for k, v in cpl.items()},
           "steps": steps, "dt_fs": dt}
    for prec, tag in ((md.MD_FP64, "fp64"), (md.MD_MIXED, "mixed")):
        g = md.System(sysm.box, sysm.pbc, n, sysm.kind, sysm.params, sysm.mass, precision=prec,
                      stream=stream.cuda_stream)
        g.set_positions(sysm.pos)
        g.set_velocities(sysm.vel)
        g.set_npt(**cpl)
        g.run(warmup, dt, record=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ser = g.run(steps, dt, record=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        box = g.box()
        T = 2.0 * ser[-1, 1] / (I.KB_EV_PER_K * (3 * n - 3))
        out[tag] = {"value": n * steps / (ms / 1e3), "ms_per_step": ms / steps,
                    "box_rel_change": [float(b / b0 - 1.0) for b, b0 in zip(box, sysm.box)],
                    "temperature_K_last": float(T),
                    "kernel_launches_per_step": int(g.stats().kernel_launches_per_step)}
        g.close()
    return out


# ---------------------------------------------------------------- batched pool
def batch_systems(n_sys=512, lo=64, hi=20000, seed=11):
    """512 Si diamond / C graphene cells, atom counts log-uniform in [64, 20000] snapped to
    admissible lattices (total ~1.8M atoms), 300 K."""
    out = []
    for k, (kind, a, b, n) in enumerate(I.batch_sizes(n_sys, lo, hi, seed)):
        if kind == "si_diamond":
            s = I.si_diamond_tersoff(n=a, jitter_amp=0.05, seed_pos=1000 + k, seed_vel=2000 + k)
            out.append((s, 0))
        else:
            s = I.c_graphene_tersoff(nx=a, ny=b, jitter_amp=0.02, seed_pos=1000 + k, seed_vel=2000 + k)
            out.append((s, 1))
    return out


def run_batch(args, steps, warmup):
    import torch
    from paper_1610_03343_gb300 import md
    systems = batch_systems()
    cap = sum((s.n + 127) // 128 * 128 for s, _ in systems)
    n_tot = sum(s.n for s, _ in systems)
    out = {"n_systems": len(systems), "n_atoms": n_tot, "dt_fs": 0.5, "steps": steps}
    stream = torch.cuda.Stream()
    for prec, tag in ((md.MD_FP64, "fp64"), (md.MD_MIXED, "mixed")):
        pool = md.Pool(cap, len(systems), I.MD_TERSOFF, [I.TERSOFF_SI_1989, I.TERSOFF_C_1989],
                       [I.MASS_SI, I.MASS_C], precision=prec, stream=stream.cuda_stream)
        for s, pset in systems:
            pool.add(s.pos, s.vel, s.box, s.pbc, pset, np.full(s.n, pset, np.int32))
        if args.eager:
            md.md_set_graph_mode(pool.ctx, False)
        pool.run(1, 0.5)
        tuning = None
        if args.pool_tuning:
            pb, g = dict(zip(("fp64", "mixed"), args.pool_tuning.split(",")))[tag].split("x")
            md.md_set_tuning(pool.ctx, pair_block=int(pb), pool_blocks_per_sm=int(g))
            tuning = {"pair_block": int(pb), "pool_blocks_per_sm": int(g), "imposed": True}
        elif not args.no_tune:
            tuning = md.tuning_dict(md.md_autotune(pool.ctx, 5))
        pool.run(warmup, 0.5)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pool.run(steps, 0.5)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        r0 = md.md_get_stats(pool.ctx).n_rebuilds
        md.md_set_profiling(pool.ctx, True)
        pool.run(min(steps, 40), 0.5)
        kt = md.md_kernel_times(pool.ctx)
        md.md_set_profiling(pool.ctx, False)
        out[tag] = {"value": n_tot * steps / (ms / 1e3), "unit": "atom-steps/s", "ms_per_step": ms / steps,
                    "kernel_ms_per_step": {k: (v[1] / v[0] if v[0] else None) for k, v in kt.items()},
                    "rebuilds_per_step": (md.md_get_stats(pool.ctx).n_rebuilds - r0) / min(steps, 40),
                    "tuning": tuning}
        pool.close()
    return out


# ---------------------------------------------------------------- serving
class JobFactory:
    """Serving jobs: Tersoff (Si or C) or SW (Si) cells, atom count log-uniform in
    [64, 200000] snapped to a lattice, steps uniform in [100, 2000], NVE or damped
    relaxation (gamma = 0.01 / fs), 300 K, seeded.  Lattices are cached by shape; every
    job draws its own jitter and velocities."""

    def __init__(self, seed=21):
        self.rng = np.random.Generator(np.random.PCG64(seed))
        self.cache = {}

    def lattice(self, key):
        if key not in self.cache:
            kind, a, b = key
            if kind == "gr":
                self.cache[key] = I.graphene_positions(a, b, 1.42, 20.0)
            else:
                self.cache[key] = I.diamond_positions(a, 5.432 if kind == "si_t" else 5.431)
        return self.cache[key]

    def make(self, k):
        r = self.rng
        kind = I.MD_TERSOFF if r.random() < 0.5 else I.MD_SW
        elem = (0 if r.random() < 0.5 else 1) if kind == I.MD_TERSOFF else 0
        target = math.exp(r.uniform(math.log(64), math.log(200000)))
        if elem == 1:
            nx = max(3, int(round(math.sqrt(target / 4.0 / 1.732))))
            ny = max(3, int(round(1.732 * nx)))
            key = ("gr", nx, ny)
        else:
            n = max(2, int(round((target / 8.0) ** (1.0 / 3.0))))
            key = ("si_t" if kind == I.MD_TERSOFF else "si_s", n, n)
        pos0, box = self.lattice(key)
        pbc = np.array([1, 1, 1], np.int32)
        amp = 0.02 if elem == 1 else 0.05
        pos = I.wrap(pos0 + r.uniform(-amp, amp, size=pos0.shape), box, pbc)
        mass = I.MASS_C if elem == 1 else I.MASS_SI
        vel = I.maxwell_boltzmann(pos.shape[0], mass, 300.0, int(r.integers(1 << 30)))
        steps = int(r.integers(100, 2001))
        damp = 0.01 if r.random() < 0.5 else 0.0
        return dict(kind=kind, pset=elem, pos=pos, vel=vel, box=box, pbc=pbc, steps=steps, damp=damp,
                    types=np.full(pos.shape[0], elem, np.int32))


def run_serve(args, rate=None, n_requests=None, seed=31):
    """Poisson arrivals into the serving loop; a waiter thread collects results in
    submission order (and releases each job's output buffers) while submission goes on."""
    import queue
    from paper_1610_03343_gb300 import md
    rate = args.serve_rate if rate is None else rate
    n_requests = args.serve_requests if n_requests is None else n_requests
    rng = np.random.Generator(np.random.PCG64(seed))
    fac = JobFactory()
    jobs = [fac.make(k) for k in range(n_requests)]
    sizes = [(j["pos"].shape[0], j["steps"]) for j in jobs]
    kinds = [j["kind"] for j in jobs]
    gaps = rng.exponential(1.0 / rate, size=len(jobs))
    results = []
    with md.Server(precision=md.MD_MIXED, tersoff_atoms=12_000_000, sw_atoms=6_000_000, max_jobs_per_pool=1024,
                   tersoff_dt=0.5, sw_dt=1.0, chunk_steps=8, tersoff_sets=[I.TERSOFF_SI_1989, I.TERSOFF_C_1989],
                   tersoff_masses=[I.MASS_SI, I.MASS_C], sw_set=[I.SW_SI_1985], sw_mass=[I.MASS_SI]) as srv:
        q = queue.Queue()

        def waiter():
            while True:
                jid = q.get()
                if jid is None:
                    return
                results.append(srv.wait(jid)[0])

        th = threading.Thread(target=waiter, daemon=True)
        th.start()
        t_next = time.perf_counter()
        for k, gap in enumerate(gaps):
            t_next += gap
            while time.perf_counter() < t_next:
                time.sleep(min(0.002, max(0.0, t_next - time.perf_counter())))
            j = jobs[k]
            q.put(srv.submit(j["kind"], j["pos"], j["vel"], j["box"], j["pbc"], j["steps"], j["pset"],
                             j["types"], j["damp"], want_state=True))
            jobs[k] = None   # the server holds its own copy
        q.put(None)
        th.join()
        st = srv.stats()
    lat = np.array([r.t_done - r.t_submit for r in results])
    t0 = min(r.t_submit for r in results)
    t1 = max(r.t_done for r in results)
    t_last_submit = max(r.t_submit for r in results)
    work = sum(n * st_ for n, st_ in sizes)
    # queue stable: the server keeps up with the arrivals -- the work it completes per second,
    # from the first arrival to the last completion, is at least 90% of the work offered per
    # second over the arrival window (an overloaded queue falls behind and drains long after
    # the last arrival)
    drain = t1 - t_last_submit
    offered_rate = work / max(t_last_submit - t0, 1e-9)
    achieved_rate = work / max(t1 - t0, 1e-9)
    stable = bool(achieved_rate >= 0.9 * offered_rate)
    return {"requests": len(sizes), "rate_per_s": rate, "completed": int(st.completed), "queue_stable": stable,
            "failed": int(st.failed), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_atoms": float(np.mean([n for n, _ in sizes])), "value": work / (t1 - t0), "unit": "atom-steps/s",
            "offered": rate * work / len(sizes), "precision": "mixed", "wall_s": t1 - t0,
            "mean_job_atom_steps": work / len(sizes),
            "pool_seconds": {"busy": st.busy_seconds, "run": st.run_seconds, "admit": st.admit_seconds,
                             "harvest": st.harvest_seconds, "chunks": int(st.chunks)},
            "drain_s": drain, "kept_up": achieved_rate / offered_rate,
            # the two pools run concurrently: their run seconds add up to more than the wall time
            "resident_atom_steps_per_run_s": st.resident_atom_steps / max(st.run_seconds, 1e-9),
            "resident_atom_steps_per_wall_s": st.resident_atom_steps / max(t1 - t0, 1e-9),
            "work_by_kind": {"tersoff": float(sum(n * k for (n, k), j in zip(sizes, kinds) if j == I.MD_TERSOFF)),
                             "sw": float(sum(n * k for (n, k), j in zip(sizes, kinds) if j == I.MD_SW))}}


def precision_report(res, n, dt, box):
    """Energy drift of each path over the timed run and the heat-current autocorrelation
    (md_hcacf on each path's J series) of the mixed path against the fp64 path."""
    from paper_1610_03343_gb300 import md
    out = {}
    for tag in res:
        e = res[tag]["series"][:, 0] + res[tag]["series"][:, 1]
        out[f"energy_drift_ev_per_atom_{tag}"] = float((e[-1] - e[0]) / n)
    if "fp64" in res and "mixed" in res:
        rows = res["fp64"]["series"].shape[0]
        lags = max(1, min(200, rows // 2))
        c64, _ = md.green_kubo(res["fp64"]["series"], lags)
        cmx, _ = md.green_kubo(res["mixed"]["series"], lags)
        a64, amx = c64.sum(axis=1), cmx.sum(axis=1)
        out["hcacf_lags"] = lags
        out["hcacf_max_diff_rel_c0"] = float(np.abs(amx - a64).max() / abs(a64[0]))
        out["j_series_max_diff_rel"] = float(np.abs(res["mixed"]["series"][:, 2:5] - res["fp64"]["series"][:, 2:5]).max()
                                             / np.abs(res["fp64"]["series"][:, 2:5]).max())
    return out


def mixed_force_error():
    """Force error of the mixed path against the fp64 path on the serving job kinds."""
    from paper_1610_03343_gb300 import md
    worst = 0.0
    for s in (I.si_diamond_tersoff(n=6), I.c_graphene_tersoff(nx=20, ny=30), I.si_diamond_sw(n=6, jitter_amp=0.05)):
        f = []
        for prec in (md.MD_FP64, md.MD_MIXED):
            with md.from_inputs(s, precision=prec) as g:
                f.append(g.compute(want=("f",))["F"])
        worst = max(worst, float(np.abs(f[1] - f[0]).max() / np.abs(f[0]).max()))
    return worst


def measure_peaks():
    """FP64 and FP32 FMA peaks of this GPU (md_peak_flops: independent FMA chains on every SM,
    best of 8 launches timed with CUDA events), with the SM clock sampled meanwhile."""
    import torch
    from paper_1610_03343_gb300 import md
    out = {}
    clocks = ClockSampler(torch.cuda.current_device())
    with clocks:
        for tag, prec in (("fp64", md.MD_FP64), ("fp32", md.MD_MIXED)):
            tf, ms = md.md_peak_flops(prec, PEAK_ITERS[tag], 8)
            out[f"{tag}_tflops"] = tf
            out[f"{tag}_ms_per_launch"] = ms
    out["clocks"] = clocks.summary()
    out["how"] = ("md_peak_flops: independent FMA chains (8 per thread fp64, 16 fp32), 1024 threads per SM on every SM, "
                  "best of 8 launches timed with CUDA events, 2 flop per FMA")
    return out


def precision_vs_oracle():
    """Errors of the mixed path against the FP64 oracle: forces, per-atom energy, virial
    and heat current of one evaluation on the serving job kinds; and over a 200-step NVE run
    of a 2400-atom sheet (dt 0.5 fs) from the same state, the energy drift of each and the
    difference of their heat-current autocorrelations (both formed by the oracle's
    Green-Kubo routine, normalised by the oracle's C(0))."""
    import oracle
    from oracle import green_kubo as gk
    from paper_1610_03343_gb300 import md
    oracle.build()

    def rel(a, b):
        return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())

    out = {"evaluation": {}}
    for s in (I.si_diamond_tersoff(n=6), I.c_graphene_tersoff(nx=20, ny=30), I.si_diamond_sw(n=6, jitter_amp=0.05)):
        ref = oracle.compute(s.pos, s.box, s.pbc, s.kind, s.params, s.vel)
        with md.from_inputs(s, precision=md.MD_MIXED) as g:
            got = g.compute()
        out["evaluation"][s.name] = {k: rel(got[k], ref[k]) for k in ("F", "U", "W", "J")}
    out["force_err_max"] = max(e["F"] for e in out["evaluation"].values())
    s = I.c_graphene_tersoff(nx=20, ny=30)
    steps, dt = 200, 0.5
    _, _, ser_o = oracle.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, steps, dt)
    sers = {}
    for tag, prec in (("fp64", md.MD_FP64), ("mixed", md.MD_MIXED)):
        with md.from_inputs(s, precision=prec) as g:
            sers[tag] = g.run(steps, dt)
    e_o = ser_o[:, 0] + ser_o[:, 1]
    traj = {"system": s.name, "n_atoms": s.n, "steps": steps, "dt_fs": dt,
            "energy_drift_ev_per_atom_oracle": float((e_o[-1] - e_o[0]) / s.n)}
    lags = 100
    c_o = gk.hcacf(ser_o[:, 2:5], lags).sum(axis=1)
    for tag, ser in sers.items():
        e = ser[:, 0] + ser[:, 1]
        traj[f"energy_drift_ev_per_atom_{tag}"] = float((e[-1] - e[0]) / s.n)
        traj[f"energy_series_max_diff_ev_per_atom_{tag}"] = float(np.abs(e - e_o).max() / s.n)
        traj[f"j_series_max_diff_rel_{tag}"] = rel(ser[:, 2:5], ser_o[:, 2:5])
        traj[f"hcacf_max_diff_rel_c0_{tag}"] = float(np.abs(gk.hcacf(ser[:, 2:5], lags).sum(axis=1) - c_o).max()
                                                     / abs(c_o[0]))
    out["trajectory"] = traj
    return out


def run_sw_leg(args, steps, warmup, peaks):
    """Stillinger-Weber silicon, 40^3 cells (512,000 atoms), 300 K, dt 1 fs: fp64 and mixed
    atom-steps/s after 100 untimed steps (the crystal gains about one bond per atom as its
    second shell moves inside the cutoff), with the fp64 pair pass's roofline."""
    import torch
    from paper_1610_03343_gb300 import md
    sysm, dt = workload("sw_si_512k")
    n = sysm.n
    stream = torch.cuda.Stream()
    out = {"workload": "sw_si_512k", "n_atoms": n, "dt_fs": dt, "steps": steps, "equilibration_steps": 100}
    for prec, tag in ((md.MD_FP64, "fp64"), (md.MD_MIXED, "mixed")):
        g = md.System(sysm.box, sysm.pbc, n, sysm.kind, sysm.params, sysm.mass, precision=prec,
                      stream=stream.cuda_stream)
        g.set_positions(sysm.pos)
        g.set_velocities(sysm.vel)
        g.run(100, dt, record=False)
        md.md_autotune(g.ctx, 5)
        g.run(warmup, dt, record=True)
        pos0 = g.state()[0]
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.run(steps, dt, record=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        pos1 = g.state()[0]
        kt, _ = kernel_window(md, g, steps, warmup, dt, stream)
        g.close()
        rc = I.cutoff(sysm.kind, sysm.params)
        bst = [bond_statistics(p_, sysm.box, sysm.pbc, rc) for p_ in (pos0, pos1)]
        bonds, pairs = 0.5 * (bst[0][0] + bst[1][0]), 0.5 * (bst[0][1] + bst[1][1])
        pn, pms = kt.get("pair", (0, 0.0))
        leg = {"value": n * steps / (ms / 1e3), "unit": "atom-steps/s", "ms_per_step": ms / steps,
               "kernel_ms_per_step": {k: (v[1] / v[0] if v[0] else None) for k, v in kt.items()},
               "bonds_per_atom": round(bonds, 4), "bond_pairs_per_atom": round(pairs, 4)}
        if pn:
            t_pair = pms / pn / 1e3
            leg["pair_tflops_algorithmic"] = pair_flops_algorithmic(sysm.kind, bonds, pairs) * n / t_pair / 1e12
            if tag == "fp64":
                leg["pair_tflops_counted"] = pair_flops(sysm.kind, bonds, pairs) * n / t_pair / 1e12
                pm = pipe_model(sysm.kind, bonds, pairs, n, peaks)
                leg["pair_pipes"] = pm
                leg["pair_frac_of_pipe_model"] = pm["t_model_us"] * 1e-6 / t_pair
                leg["pair_launch_us"] = t_pair * 1e6
        out[tag] = leg
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--equilibrate", type=int, default=100,
                    help="untimed steps from the initial state before tuning and warm-up")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tersoff_c_graphene_1M")
    ap.add_argument("--scale", type=int, default=1,
                    help="divide the workload's cell counts per axis by this (profiling captures of smaller systems)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"])
    ap.add_argument("--eager", action="store_true",
                    help="launch each kernel eagerly instead of replaying graphs (for profilers)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shapes (no autotuner)")
    ap.add_argument("--pair-cap", type=int, default=0, choices=[0, 3, 4],
                    help="with --pair-block: bond slots of the fp64 Tersoff common-case pass (0 = 4)")
    ap.add_argument("--pair-block", default="",
                    help="impose the pair block size instead of autotuning: 'FP64,MIXED', e.g. 64,128")
    ap.add_argument("--pool-tuning", default="",
                    help="impose the batch leg's tuning: 'PBxBPS,PBxBPS' for fp64 and mixed, e.g. 64x16,128x16")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-npt", action="store_true")
    ap.add_argument("--no-sw", action="store_true", help="skip the Stillinger-Weber 512k-atom leg")
    ap.add_argument("--no-oracle-precision", action="store_true",
                    help="skip the mixed-path errors against the oracle (about 5 s of CPU work)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-requests-low", type=int, default=400,
                    help="requests of each below-capacity serving run (50%%, 80%% and 95%% of capacity)")
    ap.add_argument("--only", default="", choices=["", "batch", "serve"],
                    help="run one leg alone and print its JSON (diagnostics)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(args)))
        return
    if args.only == "batch":
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_batch(args, max(8, args.steps // 2), args.warmup)))
        return
    if args.only == "serve":
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_serve(args)))
        return

    n, dt, res, t_e2e, h2d, d2h, mixed_err = run_ours(args, rank, world)
    primary = "fp64" if "fp64" in res else "mixed"
    ms = res[primary]["ms"]
    ms_mixed = res["mixed"]["ms"] if "mixed" in res else 0.0
    ms, ms_mixed, t_e2e_max = reduce_max_over_ranks([ms, ms_mixed, t_e2e or 0.0], world, "cuda")
    t_e2e = t_e2e_max if t_e2e is not None else None
    value = job_value(world, n, args.steps, ms)
    if rank != 0:
        return
    kt = res[primary]["kt"]
    pair_n, pair_ms = kt.get("pair", (0, 0.0))
    sysm, _ = workload(args.workload, args.scale)
    peaks_hw = load_peaks()
    peaks = measure_peaks()
    fp64_peak = peaks["fp64_tflops"]
    # bonds at the first and the last step of the timed region (SW's count grows as the
    # crystal warms up); the pair pass's flops per launch use their mean
    rc = I.cutoff(sysm.kind, sysm.params)
    bstats = [bond_statistics(p, sysm.box, sysm.pbc, rc) for p in res[primary]["pos_window"]]
    bonds = 0.5 * (bstats[0][0] + bstats[1][0])
    bond_pairs = 0.5 * (bstats[0][1] + bstats[1][1])
    flops_alg = pair_flops_algorithmic(sysm.kind, bonds, bond_pairs) * n
    flops_cnt = pair_flops(sysm.kind, bonds, bond_pairs) * n
    pair_avg_s = pair_ms / pair_n / 1e3 if pair_n > 0 and pair_ms > 0 else None
    ach_alg = flops_alg / pair_avg_s / 1e12 if pair_avg_s else None
    ach_cnt = flops_cnt / pair_avg_s / 1e12 if pair_avg_s else None
    traffic = PAIR_TRAFFIC_BYTES.get(args.workload) if primary == "fp64" else None
    # The fp64 pass runs the method's arithmetic partly on the FP64 pipe (what needs 53 bits)
    # and partly as float pairs on the FP32 pipe: its roofline is the larger of the two pipe
    # times of its instruction mix at this GPU's measured rates; `peak` expresses that bound
    # as an algorithmic flop rate, so frac = model time / launch time.
    pm = pipe_model(sysm.kind, bonds, bond_pairs, n, peaks) if primary == "fp64" else None
    peak_mix = flops_alg / (pm["t_model_us"] * 1e-6) / 1e12 if pm else None
    roofline = {"bound": "alu", "kernel": f"pair ({primary})", "achieved": ach_alg, "peak": peak_mix,
                "unit": "TFLOP/s", "frac": ach_alg / peak_mix if (ach_alg and peak_mix) else None,
                "traffic": traffic, "flop_per_launch": flops_alg,
                "flop_model": "expression count of Eqs. 2-6 and dU_i/dr_ij: +,-,* 1 flop; division, "
                              "reciprocal, 1/sqrt 8; exp, log 16",
                "peak_model": "algorithmic flops / max(FP64-pipe time, issue time) of the launch's counted "
                              "instruction mix at the measured FP64 (md_peak_flops fp64) and issue "
                              "(md_peak_flops fp32 / 64) rates",
                "pipes": pm,
                "launch_us": pair_avg_s * 1e6 if pair_avg_s else None,
                "fp64_peak": fp64_peak,
                "vs_fp64_peak": ach_alg / fp64_peak if ach_alg else None,
                "fp64_peak_source": "measured on this GPU: md_peak_flops FP64 FMA chains "
                                    f"(SM clock median {peaks['clocks'].get('sm_mhz')} MHz)",
                "fp64_peak_nominal": FP64_PEAK_NOMINAL_TFLOPS,
                "counted": {"achieved": ach_cnt, "flop_per_launch": flops_cnt,
                            "frac_of_fp64_peak": ach_cnt / fp64_peak if ach_cnt else None,
                            "flop_model": "DADD + DMUL + 2 DFMA thread instructions of the kernel (ncu), "
                                          "per bond and per ordered bond pair"},
                "bonds_per_atom": [round(b[0], 4) for b in bstats],
                "bond_pairs_per_atom": [round(b[1], 4) for b in bstats]}
    out = {
        "metric": "atom-steps/s Tersoff FP64 vs mixed on 1 GB300",
        "value": value,
        "unit": "atom-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if primary == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n_atoms": n, "dt_fs": dt, "ensemble": "NVE",
                   "equilibration_steps": args.equilibrate,
                   "l2": "working set > L2 (no flush)", "launch": "eager" if args.eager else "graphs",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roofline,
        "peaks": peaks,
        "kernel_ms_per_step": {k: (v[1] / v[0] if v[0] else None) for k, v in kt.items()},
        "kernel_window": {"steps": args.steps, "ms_per_step": res[primary]["ms_events"] / args.steps,
                          "how": "kernel_ms_per_step and the rooflines' launch times come from a second "
                                 "window of the same number of steps right after the timed region, "
                                 "with a CUDA event pair around every kernel class of every step; the "
                                 "timed region runs without those event nodes, which cost time of "
                                 "their own (this window's ms_per_step)"},
        "gpu_launches": res[primary]["launches"],
        "rebuilds": res[primary]["rebuilds"],
        "clocks": res[primary]["clocks"],
        "tuning": res[primary]["tuning"],
    }
    if "mixed" in res and primary != "mixed":
        kmx = res["mixed"]["kt"]
        out["mixed"] = {"value": job_value(world, n, args.steps, ms_mixed), "ms_per_step": ms_mixed / args.steps,
                        "dtype": "f32+f64", "force_err_vs_fp64": mixed_err,
                        "kernel_ms_per_step": {k: (v[1] / v[0] if v[0] else None) for k, v in kmx.items()},
                        "kernel_window_ms_per_step": res["mixed"]["ms_events"] / args.steps,
                        "tuning": res["mixed"]["tuning"]}
        # the mixed step's largest kernel is the gather (memory-latency bound): its roofline
        # is HBM, on the algorithmic bytes one launch must move; the pair pass's is the FP32
        # pipe, on the expression-count flops
        gn, gms = kmx.get("gather", (0, 0.0))
        pn, pms = kmx.get("pair", (0, 0.0))
        hbm = peaks_hw["hbm_gbs"]
        rm = {"bound": "hbm", "kernel": "gather (mixed)", "unit": "GB/s", "peak": hbm,
              "peak_source": f"{peaks_hw['_source']} HBM copy bandwidth (MEASURED_PEAKS.json)",
              "traffic": GATHER_TRAFFIC_BYTES.get(args.workload), "traffic_note": GATHER_TRAFFIC_NOTE,
              "bytes_per_launch": gather_bytes_algorithmic(bonds) * n,
              "bytes_model": "per atom: mask 4 + list 5M + dU/dr 12M + r 12M + U 8 + type 4 + v 48 + F 24 "
                             "+ fused drift 72 (M in-cutoff bonds)"}
        if gn:
            t = gms / gn / 1e3
            rm["achieved"] = rm["bytes_per_launch"] / t / 1e9
            rm["frac"] = rm["achieved"] / hbm
            rm["launch_ms"] = t * 1e3
        if pn:
            t = pms / pn / 1e3
            a32 = pair_flops_algorithmic(sysm.kind, bonds, bond_pairs) * n / t / 1e12
            rm["pair"] = {"bound": "alu", "kernel": "pair (mixed, fp32)", "unit": "TFLOP/s", "achieved": a32,
                          "peak": peaks["fp32_tflops"], "frac": a32 / peaks["fp32_tflops"], "launch_ms": t * 1e3,
                          "peak_source": "measured on this GPU: md_peak_flops FP32 FMA chains"}
        out["roofline_mixed"] = rm
    out["precision"] = precision_report(res, n, dt, sysm.box)
    if not args.no_oracle_precision:
        out["precision"]["vs_oracle"] = precision_vs_oracle()
    if t_e2e is not None:
        out["e2e"] = {"value": world * n * args.steps / t_e2e, "unit": "atom-steps/s",
                      "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps}
    if not args.no_npt:
        out["npt"] = run_npt_leg(args, max(8, args.steps // 2), args.warmup)
    if not args.no_sw:
        out["sw"] = run_sw_leg(args, max(20, args.steps // 2), args.warmup, peaks)
    if not args.no_batch:
        out["batch"] = run_batch(args, max(8, args.steps // 2), args.warmup)
    if not args.no_serve:
        sv = run_serve(args)
        out["serve"] = sv
        sv["force_err_mixed_vs_fp64"] = mixed_force_error()
        if "vs_oracle" in out["precision"]:
            sv["force_err_mixed_vs_oracle"] = out["precision"]["vs_oracle"]["force_err_max"]
        # the device's capacity for this job mix, from the pool and SW rates measured above:
        # Tersoff work at the batched mixed rate, SW work at the SW leg's mixed rate
        wk = sv["work_by_kind"]
        if "batch" in out and "sw" in out and wk["tersoff"] + wk["sw"] > 0:
            rt, rs = out["batch"]["mixed"]["value"], out["sw"]["mixed"]["value"]
            est = (wk["tersoff"] + wk["sw"]) / (wk["tersoff"] / rt + wk["sw"] / rs)
            sv["mix_capacity_estimate"] = {"value": est, "unit": "atom-steps/s",
                                           "from": "batched Tersoff mixed and SW 512k mixed rates, weighted by "
                                                   "the job mix's atom-steps"}
            sv["fraction_of_mix_capacity"] = sv["value"] / est
        # capacity: the saturated throughput of the run above in jobs/s (arrivals faster than
        # the server); then the same job mix at 50%, 80% and 95% of it, each reporting whether
        # the queue kept up and its p50/p99
        keys = ("rate_per_s", "requests", "p50_s", "p99_s", "value", "queue_stable", "kept_up", "completed",
                "drain_s")
        cap_jobs = sv["value"] / sv["mean_job_atom_steps"]
        sv["capacity_jobs_per_s"] = cap_jobs
        sv["capacity_how"] = "saturated throughput of the 200/s run (atom-steps/s over the mean job's atom-steps)"
        sv["below_capacity"] = [
            {q: v for q, v in run_serve(args, rate=f * cap_jobs, n_requests=args.serve_requests_low,
                                        seed=41 + k).items() if q in keys} | {"fraction_of_capacity": f}
            for k, f in enumerate((0.5, 0.8, 0.95))]
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(out))


def _oracle_rate(sysm, dt, steps):
    import oracle
    t0 = time.perf_counter()
    oracle.run(sysm.pos, sysm.vel, sysm.mass, sysm.box, sysm.pbc, sysm.kind, sysm.params, steps, dt)
    t = time.perf_counter() - t0
    return sysm.n * steps / t, t


def cpu_sample(args):
    """A bounded sample of the bench workload for the oracle: a 250 x 250-cell patch
    (250,000 atoms) of the same sheet, or the same lattice at half the edge."""
    if "graphene" in args.workload:
        return I.c_graphene_tersoff(nx=250, ny=250)
    return workload(args.workload, 2)[0]


def cpu_baseline(args):
    """The oracle as it stands, single-threaded on a host core, on the bounded sample
    (about 10-15 s of CPU work: 24 velocity-Verlet steps)."""
    import oracle
    oracle.build()
    sysm = cpu_sample(args)
    _, dt = workload(args.workload)
    rate, t = _oracle_rate(sysm, dt, 24)
    return {"value": rate, "unit": "atom-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{sysm.n} atoms of the same lattice, 24 steps, {t:.1f} s"}


def reference_arm(args):
    """The oracle timed on the host as the reference arm: each step one velocity-Verlet
    step of the bounded sample (cpu_sample), at most 40 steps (about 20 s)."""
    import oracle
    oracle.build()
    sysm = cpu_sample(args)
    _, dt = workload(args.workload)
    steps = max(1, min(args.steps, 40))
    for _ in range(min(args.warmup, 1)):
        _oracle_rate(sysm, dt, 1)
    rate, t = _oracle_rate(sysm, dt, steps)
    return {"impl": "reference", "metric": "atom-steps/s Tersoff FP64 vs mixed on 1 GB300", "value": rate,
            "unit": "atom-steps/s", "n_gpus": 1, "steps": steps, "warmup": min(args.warmup, 1),
            "ms_per_step": t / steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample_atoms": sysm.n, "dt_fs": dt},
            "cpu_baseline": {"value": rate, "unit": "atom-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{sysm.n} atoms x {steps} steps"},
            "e2e": {"value": rate, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


if __name__ == "__main__":
    main()
