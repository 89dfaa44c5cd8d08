"""Throughput benchmark of the fused three-distribution MRT-LB step.

Default workload: the differentially heated porous cavity at 4096 x 4096
nodes, FP32 storage, per-node porosity U[0.3, 0.9] (seed 2) with the Ergun
medium at mean Da = 1e-3, Ra = 1e6, H = 100, conductivity ratio 10
(synthetic inputs).  A "step" is one lattice time step of all nodes: the
D2Q9 flow and both D2Q5 temperature distributions, collision, streaming and
walls.  MLUPS = nodes x steps / seconds.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Under torchrun (N > 1) every rank advances its own
cavity (independent replicas, weak scaling) and rank 0 prints.  At N = 1 the
line also carries, under "forms", compact runs of the other forms next to
the plain FP32 kernel: the same cavity at 1024 x 1024, the 256-cavity batch
(autotuned schedule), the forward + adjoint at 256 x 256 and the FP32 /
FP16 / BF16 storage forms at 8192 x 8192, each with its MLUPS, roofline
fraction, errors against the
oracle (whose timed run of the checked sample is that leg's CPU baseline)
and the clocks sampled while it was timed (--no-forms skips them).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1608_04118_gb300 import workloads as W  # noqa: E402

METRIC = "MLUPS (all 3 distributions fused)"
UNIT = "MLUPS"
# Algorithmic bytes per lattice update: read + write of 19 populations plus
# the per-node porosity read.
BYTES_PER_LUP = {"f32": 2 * 19 * 4 + 4, "f64": 2 * 19 * 8 + 8, "f16": 2 * 19 * 2 + 4,
                 "bf16": 2 * 19 * 2 + 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=500)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096, help="cavity side (nodes)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f64", "f16", "bf16"])
    ap.add_argument("--npt", type=int, default=0, choices=[0, 1, 2],
                    help="nodes per thread of the step kernel (0: the library default)")
    ap.add_argument("--block", default="",
                    help="block shape bx,by of the step kernel (default: the library's)")
    ap.add_argument("--staging", type=int, default=-1, choices=[-1, 0, 1],
                    help="two-node step fed from TMA-staged shared-memory tiles (1) or by "
                         "direct loads (0; -1: the library's default)")
    ap.add_argument("--cavities", type=int, default=256,
                    help="c3: number of cavities (the workload has 256; fewer for profiling)")
    ap.add_argument("--batch-schedule", default="",
                    help="c3: tile_x,tile_y,blocks,nodes_per_thread instead of the autotuned "
                         "schedule")
    ap.add_argument("--no-context", action="store_true",
                    help="c4: skip the 1024^2 context run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the compact batched / adjoint / reduced-storage legs of the "
                         "default line")
    ap.add_argument("--split", default="replicas", choices=["replicas", "slabs"],
                    help="N > 1: replicas (one independent cavity per rank, weak scaling; "
                         "default) or slabs (one cavity cut into N row slabs, halos exchanged "
                         "with NCCL after every step, strong scaling)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5"],
                    help="c2: single cavity (default, the headline line); c3: 256-cavity "
                         "batch; c4: forward + adjoint; c5: reduced-storage forms at 8192^2 "
                         "with their errors")
    return ap.parse_args()


def workload_config(n, storage):
    c = W.C2_THROUGHPUT
    return {"workload": "porous LTNE cavity %dx%d, per-node porosity U[%.1f,%.1f] seed %d, "
                        "Ergun K (mean Da %.0e), Ra %.0e, H %.0f, gamma_sf %.0f"
                        % (n, n, c["phi_lo"], c["phi_hi"], c["seed"], c["Da"], c["Ra"], c["H"],
                           c["gamma_sf"]),
            "nx": n, "ny": n, "storage": storage, "lattice": "D2Q9 + 2 x D2Q5 (MRT)",
            "l2": "inputs larger than L2 (%.2f GB of populations per buffer)"
                  % (19 * BYTES_PER_LUP[storage] / 38 * n * n / 1e9 if storage != "f64"
                     else 19 * 8 * n * n / 1e9)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, device=None):
    """Max of a per-rank value over all ranks of the default process group
    (the value itself when not distributed)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank, steps, world, t_max):
    """Lattice updates of all ranks (independent replicas) over the slowest
    rank's time, in millions per second."""
    return world * nodes_per_rank * steps / t_max / 1e6


def replica_seed(base, rank):
    """Porosity seed of rank `rank`'s cavity (rank 0 = the single-GPU input)."""
    return base + rank


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_traffic(storage, n, npt):
    """ncu DRAM bytes per launch of the step kernel (storage type, nodes per
    thread) from the committed profile summary, if it was taken on the
    current kernel source: (bytes, how) with how "measured at NxN" when the
    capture is of this lattice, else "scaled from NxN" (traffic grows with
    the node count), or (None, reason)."""
    p = os.path.join(ROOT, "profiles", "step_traffic.json")
    if not os.path.exists(p):
        return None, "no capture"
    try:
        with open(p) as fh:
            d = json.load(fh)
        from paper_1608_04118_gb300 import build as B

        if d.get("source_hash") != B.kernel_source_hash():
            return None, "capture predates the current kernel source"
        cands = [e for k, e in d["entries"].items() if k.startswith("%s/npt%d" % (storage, npt))]
        if not cands:
            return None, "no capture of this form"
        exact = [e for e in cands if int(e["nodes"]) == n * n]
        e = exact[0] if exact else max(cands, key=lambda e: int(e["nodes"]))
        side = int(round(float(e["nodes"]) ** 0.5))
        if exact:
            return float(e["dram_bytes_per_launch"]), "measured at %dx%d" % (side, side)
        return (float(e["dram_bytes_per_launch"]) * (n * n) / float(e["nodes"]),
                "scaled from %dx%d" % (side, side))
    except Exception as ex:  # a malformed summary reads as no capture
        return None, "unreadable capture (%s)" % type(ex).__name__


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline_oracle(n, target_s=12.0):
    """The FP64 oracle on the host cores, on a bounded sample of the
    workload: the same cavity physics on a 1024 x 1024 lattice for as many
    steps as fit in about target_s seconds."""
    import oracle
    from oracle import Oracle, OracleParams

    c = W.C2_THROUGHPUT
    m = min(n, 1024)
    phi = W.porosity_field(m, m, c["phi_lo"], c["phi_hi"], c["seed"]).reshape(-1)
    p = OracleParams.make(m, m, ergun_K=1, Ra=c["Ra"], Pr=c["Pr"], Da=c["Da"], H=c["H"],
                          gamma_sf=c["gamma_sf"], sigma=c["sigma"], T_hot=c["T_hot"],
                          T_cold=c["T_cold"], T_ref=c["T_ref"])
    def timed(o, secs):
        t0 = time.perf_counter()
        o.step(1)
        one = time.perf_counter() - t0
        k = max(1, int(secs / max(one, 1e-6)))
        t0 = time.perf_counter()
        o.step(k)
        return k, time.perf_counter() - t0

    cores = oracle.num_threads()
    k, dt = timed(Oracle(p, phi=phi).init(), target_s)
    # the same sample on one core, and the 64 x 64 FP64 configuration's
    # 10^4 steps on all cores
    oracle.set_num_threads(1)
    k1, dt1 = timed(Oracle(p, phi=phi).init(), target_s / 2)
    oracle.set_num_threads(cores)
    c1 = W.C1_PLAIN_64
    p1 = OracleParams.make(c1["nx"], c1["ny"], ergun_K=0,
                           **{q: c1[q] for q in ("Ra", "Pr", "Da", "porosity", "H", "gamma_sf",
                                                 "sigma", "T_hot", "T_cold", "T_ref")})
    o1 = Oracle(p1).init()
    t0 = time.perf_counter()
    o1.step(c1["steps"])
    dt_c1 = time.perf_counter() - t0
    return {"value": m * m * k / dt / 1e6, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": "FP64 oracle, %dx%d cavity with the same physics, %d steps (%.1f s)"
                      % (m, m, k, dt),
            "one_core": {"value": m * m * k1 / dt1 / 1e6, "unit": UNIT,
                         "sample": "%d steps (%.1f s)" % (k1, dt1)},
            "c1_64x64_1e4_steps_s": dt_c1}


def cpu_baseline_reduced(phys, m, steps):
    """CPU-baseline leg of the reduced-storage line: the FP64 oracle, timed
    on the host cores, on the down-sized parity run (m x m, `steps` steps of
    the same physics); its fields and observables are the reference the
    line's per-field errors are taken against."""
    import oracle
    from oracle import Oracle, OracleParams

    o = Oracle(OracleParams.make(m, m, **phys)).init()
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cpu = {"value": m * m * steps / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(),
           "kind": "oracle",
           "sample": "FP64 oracle, %dx%d cavity with the same physics, %d steps (%.1f s)"
                     % (m, m, steps, dt)}
    return cpu, o.macros(), o.observables()


def _events_time(stream, fn, clocks_gpu=None):
    """Run fn() (work enqueued on `stream`) between two CUDA events on that
    stream; seconds, plus the clocks sampled meanwhile (None if not asked)."""
    import torch

    sampler = ClockSampler(clocks_gpu) if clocks_gpu is not None else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    clocks = sampler.stop() if sampler else None
    return e0.elapsed_time(e1) / 1e3, clocks


def _field_err(got, ref):
    u = np.linalg.norm(np.stack([got["ux"] - ref["ux"], got["uy"] - ref["uy"]]))
    u /= np.linalg.norm(np.stack([ref["ux"], ref["uy"]]))
    return {"u": float(u), "Tf": float(np.linalg.norm(got["Tf"] - ref["Tf"])
                                      / np.linalg.norm(ref["Tf"])),
            "Ts": float(np.linalg.norm(got["Ts"] - ref["Ts"]) / np.linalg.norm(ref["Ts"]))}


def form_batched(stream, plain_mlups, peak, gpu, steps=200, check_steps=100):
    """Compact batched leg: the 256 cavities (seed 3) with the autotuned
    schedule, `steps` timed steps; the plain FP32 kernel on the same
    cavities one by one; errors of four cavities after `check_steps` steps
    against the oracle, whose run of them is this leg's CPU baseline."""
    import torch

    import oracle
    from oracle import Oracle, OracleParams
    from paper_1608_04118_gb300.autotune import tune_batch
    from paper_1608_04118_gb300.ltne import Batch, Cavity

    cavs = W.batch_cavities(256, seed=3)
    b = Batch(cavs, stream=stream)
    sched, _, table = tune_batch(b, steps=4, warmup=2)
    b.set_fields()
    with torch.cuda.stream(stream):
        b.step(3)
    l0 = b.launches
    t, clocks = _events_time(stream, lambda: b.step(steps), gpu)
    launches = b.launches - l0
    nodes = b.nodes
    value = nodes * steps / t / 1e6
    k_seq = 50
    singles = []
    for c in cavs:
        cc = Cavity(c["nx"], c["ny"], stream=stream, storage="f32",
                    **{k: v for k, v in c.items() if k not in ("nx", "ny")})
        singles.append(cc.set_fields())
    t_seq, _ = _events_time(stream, lambda: [cc.step(k_seq) for cc in singles])
    for cc in singles:
        cc.close()
    seq = nodes * k_seq / t_seq / 1e6
    # parity: four cavities of the batch against the oracle
    idx = [int(i) for i in np.random.default_rng(30).choice(len(cavs), 4, replace=False)]
    b.set_fields().step(check_steps)
    errs, t_orc, n_orc = [], 0.0, 0
    for i in idx:
        c = cavs[i]
        o = Oracle(OracleParams.make(c["nx"], c["ny"], **{k: v for k, v in c.items()
                                                           if k not in ("nx", "ny")}))
        t0 = time.perf_counter()
        o.init().step(check_steps)
        t_orc += time.perf_counter() - t0
        n_orc += c["nx"] * c["ny"] * check_steps
        errs.append(_field_err(b.fields(i), o.macros()))
    b.close()
    achieved = 152 * nodes * steps / t / 1e9
    return {"mlups": value, "steps": steps, "nodes": nodes, "cavities": len(cavs),
            "gpu_launches": int(launches),
            "schedule": {"tile_x": sched[0], "tile_y": sched[1], "blocks": sched[2],
                         "nodes_per_thread": sched[3], "trials": len(table)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "bytes_per_lup": 152},
            "one_by_one_plain_fp32_mlups": seq, "vs_plain_fp32_one_by_one": value / seq,
            "vs_plain_fp32_4096": value / plain_mlups,
            "errors_vs_oracle": {"cavities": [{"index": i, "nx": cavs[i]["nx"],
                                               "ny": cavs[i]["ny"], **e}
                                              for i, e in zip(idx, errs)],
                                 "steps": check_steps,
                                 "max": {k: max(e[k] for e in errs) for k in ("u", "Tf", "Ts")},
                                 "tolerance": 1e-5},
            "cpu_baseline": {"value": n_orc / t_orc / 1e6, "unit": UNIT,
                             "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "the four checked cavities, %d steps each (%.1f s)"
                                       % (check_steps, t_orc)},
            "clocks": clocks}


def form_adjoint(stream, peak, gpu):
    """Compact adjoint leg: forward 4000 steps + gradient of the hot-wall
    Nusselt average by the reverse kernels with 64-step checkpoints at
    256 x 256 (porosity U[0.4, 0.8] seed 4, Ra 1e5, Ergun mean Da 1e-3,
    H 50), next to the plain FP32 forward of the same cavity; accuracy on a
    20 x 16 cavity (120 steps) against the complex-step oracle, whose run is
    this leg's CPU baseline."""
    import math

    import torch

    import oracle
    from oracle import ComplexOracle, OracleParams
    from paper_1608_04118_gb300.ltne import Cavity, LTNE_K_ERGUN

    c = W.C4_ADJOINT
    nx, ny, steps = c["nx"], c["ny"], c["steps"]
    seg = int(math.ceil(math.sqrt(steps)))
    phi = W.porosity_field(nx, ny, c["phi_lo"], c["phi_hi"], c["seed"]).reshape(-1)
    kw = {k: c[k] for k in ("Ra", "Pr", "Da", "H", "gamma_sf", "sigma", "T_hot", "T_cold",
                            "T_ref")}
    cav = Cavity(nx, ny, stream=stream, storage="f32", permeability=LTNE_K_ERGUN,
                 porosity_field=1, **kw)
    cav.adjoint(phi, 2 * seg, segment=seg)  # warm-up
    out = {}
    t, clocks = _events_time(stream, lambda: out.update(
        r=cav.adjoint(phi, steps, segment=seg)), gpu)
    J, g, dH = out["r"]
    cav.set_fields(porosity=phi)
    with torch.cuda.stream(stream):
        cav.step(20)
    t_fwd, _ = _events_time(stream, lambda: cav.step(steps))
    cav.close()
    nodes = nx * ny
    # accuracy: the small cavity of the adjoint tests, FP32 gradient against
    # complex-step derivatives of the oracle (12 interior nodes and H)
    sm = dict(nx=20, ny=16, Ra=1e5, Pr=1.0, Da=1e-3, H=50.0, gamma_sf=3.0, sigma=1.2,
              T_hot=1.0, T_cold=0.0, T_ref=0.5)
    sphi = W.porosity_field(sm["nx"], sm["ny"], 0.4, 0.8, seed=44).reshape(-1)
    nodes_k = W.fd_nodes(sm["nx"], sm["ny"], 12, seed=45)
    p = OracleParams.make(sm["nx"], sm["ny"], ergun_K=1,
                          **{k: v for k, v in sm.items() if k not in ("nx", "ny")})
    ref = {}
    t0 = time.perf_counter()
    for k in list(nodes_k) + [-1]:
        o = ComplexOracle(p, phi=sphi).perturb(int(k), 1e-30).init().step(120)
        ref[int(k)] = o.objective()[1] / 1e-30
    t_orc = time.perf_counter() - t0
    sc = Cavity(sm["nx"], sm["ny"], stream=stream, storage="f32", permeability=LTNE_K_ERGUN,
                porosity_field=1, **{k: v for k, v in sm.items() if k not in ("nx", "ny")})
    _, gs, dHs = sc.adjoint(sphi, 120, segment=16)
    sc.close()
    gs = gs.double().cpu().numpy().reshape(-1)
    gref = np.array([ref[int(k)] for k in nodes_k])
    err_phi = float(np.abs(gs[nodes_k] - gref).max() / np.abs(gref).max())
    err_H = float(abs(dHs - ref[-1]) / abs(ref[-1]))
    plain = nodes * steps / t_fwd / 1e6
    value = nodes * steps / t / 1e6
    # algorithmic bytes per node-step: forward (156) + recompute (156) +
    # reverse (read the recorded state 76, adjoint populations 152, dJ/dphi 8)
    return {"mlups": value, "steps": steps, "segment": seg, "lattice": "%dx%d" % (nx, ny),
            "plain_fp32_forward_mlups": plain, "vs_plain_fp32": value / plain,
            "roofline": {"bound": "latency (one wave per reverse step at this size)",
                         "achieved": 548 * value * 1e6 / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": 548 * value * 1e6 / 1e9 / peak, "bytes_per_lup": 548},
            "J": J, "dJ_dH": dH, "max_abs_dJ_dphi": float(g.abs().max()),
            "errors_vs_oracle": {"case": "20x16, 120 steps, FP32 adjoint vs complex step",
                                 "dJ_dphi_max_rel": err_phi, "dJ_dH_rel": err_H,
                                 "tolerance": 1e-3},
            "cpu_baseline": {"value": sm["nx"] * sm["ny"] * 120 * len(ref) / t_orc / 1e6,
                             "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle (complex step)",
                             "sample": "%d complex-step runs of the 20x16 cavity, 120 steps "
                                       "(%.1f s)" % (len(ref), t_orc)},
            "clocks": clocks}


def form_plain_1024(stream, peak, gpu, steps=2000, warmup=500):
    """Compact leg of the throughput configuration at its smaller size:
    the 1024 x 1024 FP32 cavity with per-node porosity (seed 2, Ergun K at
    mean Da 1e-3, Ra 1e6, H 100, gamma_sf 10), default schedule, 500 warm-up
    and 2000 timed steps (two population buffers of 80 MB each, more than
    the L2 together but partly resident in it from step to step)."""
    import torch

    from paper_1608_04118_gb300.ltne import Cavity, LTNE_K_ERGUN

    c = W.C2_THROUGHPUT
    n = 1024
    kw = {k: c[k] for k in ("Ra", "Pr", "Da", "H", "gamma_sf", "sigma", "T_hot", "T_cold",
                            "T_ref")}
    phi = W.porosity_field(n, n, c["phi_lo"], c["phi_hi"], c["seed"]).reshape(-1)
    cav = Cavity(n, n, stream=stream, storage="f32", permeability=LTNE_K_ERGUN,
                 porosity_field=1, **kw).set_fields(porosity=phi)
    with torch.cuda.stream(stream):
        cav.step(warmup)
    l0 = cav.launches
    t, clocks = _events_time(stream, lambda: cav.step(steps), gpu)
    launches = int(cav.launches - l0)
    rate = n * n * steps / t / 1e6
    sched = list(cav.schedule)
    cav.close()
    achieved = BYTES_PER_LUP["f32"] * rate * 1e6 / 1e9
    return {"mlups": rate, "lattice": "%dx%d" % (n, n), "steps": steps, "warmup": warmup,
            "schedule": sched, "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "bytes_per_lup": BYTES_PER_LUP["f32"]},
            "clocks": clocks}


def form_reduced(stream, plain_mlups, peak, gpu, steps=200):
    """Compact reduced-storage leg: FP32 / FP16 / BF16 storage at 8192 x 8192
    (phi 0.6, Da 1e-2, Ra 1e6, H 1000), default schedules, `steps` timed
    steps each; per-field errors of the 512 x 512, 2000-step run against the
    oracle, whose run is this leg's CPU baseline."""
    import torch

    from paper_1608_04118_gb300.ltne import Cavity

    c = W.C5_REDUCED
    phys = {k: c[k] for k in ("Ra", "Pr", "Da", "porosity", "H", "gamma_sf", "sigma", "T_hot",
                              "T_cold", "T_ref")}
    n = c["nx"]
    rates, scheds, clocks, launches = {}, {}, {}, {}
    for st in ("f32", "f16", "bf16"):
        cav = Cavity(n, n, stream=stream, storage=st, **phys).set_fields()
        scheds[st] = list(cav.schedule)
        with torch.cuda.stream(stream):
            cav.step(3)
        l0 = cav.launches
        t, clocks[st] = _events_time(stream, lambda: cav.step(steps), gpu)
        launches[st] = int(cav.launches - l0)
        rates[st] = n * n * steps / t / 1e6
        cav.close()
        del cav
        torch.cuda.empty_cache()
    m = c["parity_n"]
    cpu, ref, robs = cpu_baseline_reduced(phys, m, c["steps"])
    errors = {}
    for st in ("f32", "f16", "bf16"):
        cav = Cavity(m, m, stream=stream, storage=st, **phys)
        cav.set_schedule(*scheds[st]).set_fields().step(c["steps"])
        got, gobs = cav.fields(), cav.observables()
        cav.close()
        e = _field_err(got, ref)
        e["Nu_max_rel"] = max(float(abs(gobs[k] - robs[k]) / abs(robs[k]))
                              for k in ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold"))
        errors[st] = e
    bpl = {"f32": 152, "f16": 76, "bf16": 76}
    return {"mlups": rates, "lattice": "%dx%d" % (n, n), "steps": steps, "schedules": scheds,
            "gpu_launches": launches,
            "vs_plain_fp32_storage": {st: rates[st] / rates["f32"] for st in rates},
            "roofline": {st: {"bound": "hbm", "achieved": bpl[st] * rates[st] / 1e3,
                              "peak": peak, "unit": "GB/s",
                              "frac": bpl[st] * rates[st] / 1e3 / peak,
                              "bytes_per_lup": bpl[st]} for st in rates},
            "errors_vs_oracle": {"run": "%dx%d, %d steps" % (m, m, c["steps"]),
                                 "fields": errors, "tolerance": 1e-3},
            "cpu_baseline": cpu, "clocks": clocks}


def run_reference(args):
    """Reference arm: the FP64 oracle, as it stands, on the host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from oracle import Oracle, OracleParams

    oracle.build()
    c = W.C2_THROUGHPUT
    m = min(args.n, 512)  # bounded sample per step so that the run ends in minutes
    phi = W.porosity_field(m, m, c["phi_lo"], c["phi_hi"], c["seed"]).reshape(-1)
    p = OracleParams.make(m, m, ergun_K=1, Ra=c["Ra"], Pr=c["Pr"], Da=c["Da"], H=c["H"],
                          gamma_sf=c["gamma_sf"], sigma=c["sigma"], T_hot=c["T_hot"],
                          T_cold=c["T_cold"], T_ref=c["T_ref"])
    o = Oracle(p, phi=phi).init()
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = m * m * args.steps / dt / 1e6
    sample = ("FP64 oracle on a %dx%d cavity with the same physics per step (bounded sample "
              "of the %dx%d workload)" % (m, m, args.n, args.n))
    # the lattice this arm actually runs; MLUPS is a per-node rate, so it
    # compares with the full-size line
    config = dict(workload_config(m, args.storage), storage="f64",
                  sample_of="%dx%d" % (args.n, args.n))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """256 independent cavities (sides 64..512, aspect 1-2, log-uniform Ra,
    Da, H, conductivity ratio; seed 3) advanced by the batched kernel with
    the autotuned schedule, against the same cavities run one by one through
    ltne_step()."""
    import torch

    torch.cuda.set_device(0)
    from paper_1608_04118_gb300 import build as B

    B.build()
    from paper_1608_04118_gb300.autotune import tune_batch
    from paper_1608_04118_gb300.ltne import Batch, Cavity

    cavs = W.batch_cavities(256, seed=3)[:args.cavities]
    stream = torch.cuda.Stream()
    b = Batch(cavs, stream=stream)
    t0 = time.perf_counter()
    if args.batch_schedule:
        sched, table = tuple(int(v) for v in args.batch_schedule.split(",")), []
        b.set_schedule(*sched)
    else:
        sched, t_best, table = tune_batch(b, steps=4, warmup=2)
    tune_s = time.perf_counter() - t0
    b.set_fields()
    with torch.cuda.stream(stream):
        b.step(max(args.warmup, 3))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = b.launches
    ev0.record(stream)
    b.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3
    nodes = b.nodes
    value = nodes * args.steps / t / 1e6
    obs = b.observables()
    # one by one: each cavity through the single-lattice path (its own
    # graph-replayed ltne_step), a shorter run -- MLUPS is a rate
    k_seq = min(args.steps, 200)
    singles = []
    for c in cavs:
        cc = Cavity(c["nx"], c["ny"], stream=stream, storage="f32",
                    **{k: v for k, v in c.items() if k not in ("nx", "ny")})
        cc.set_fields()
        singles.append(cc)
    torch.cuda.synchronize()
    ev0.record(stream)
    for cc in singles:
        cc.step(k_seq)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_seq = ev0.elapsed_time(ev1) / 1e3
    seq = nodes * k_seq / t_seq / 1e6
    peak, kind = load_peaks()
    per_launch = t / args.steps
    achieved = 152 * nodes / per_launch / 1e9
    line = {"metric": "MLUPS (batched, 256 cavities)", "value": value, "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_launch * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%d porous LTNE cavities, sides 64..512, aspect 1-2, "
                                   "seed 3" % len(cavs), "nodes": nodes,
                       "schedule": {"tile_x": sched[0], "tile_y": sched[1],
                                    "blocks": sched[2],
                                    "nodes_per_thread": sched[3] if len(sched) > 3 else 1,
                                    "tuning_s": tune_s,
                                    "trials": len(table)}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": kind, "bytes_per_lup": 152},
            "one_by_one": {"value": seq, "unit": UNIT, "steps": k_seq,
                           "note": "same cavities, ltne_step() per cavity in sequence"},
            "speedup_vs_one_by_one": value / seq,
            "gpu_launches": int(b.launches - l0),
            "nonfinite": int(sum(o["nonfinite"] for o in obs))}
    print(json.dumps(line), flush=True)


def run_reduced(args):
    """MLUPS of FP16 / BF16 / FP32 storage at 8192^2 (physics of the
    reduced-storage configuration) and their per-field errors against the
    FP64 oracle on the down-sized 512^2 run."""
    import torch

    torch.cuda.set_device(0)
    from paper_1608_04118_gb300 import build as B

    B.build()
    from paper_1608_04118_gb300.ltne import Cavity

    c = W.C5_REDUCED
    phys = {k: c[k] for k in ("Ra", "Pr", "Da", "porosity", "H", "gamma_sf", "sigma", "T_hot",
                              "T_cold", "T_ref")}
    n = args.n if args.n != 4096 else c["nx"]
    stream = torch.cuda.Stream()
    rates, rates_one_node, schedules = {}, {}, {}
    for st in ("f32", "f16", "bf16"):
        for one_node in (False, True):
            cav = Cavity(n, n, stream=stream, storage=st, **phys)
            if one_node:
                cav.set_schedule(64, 2, 1)
            schedules[(st, one_node)] = cav.schedule
            cav.set_fields()
            with torch.cuda.stream(stream):
                cav.step(max(args.warmup, 3))
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            cav.step(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            t = ev0.elapsed_time(ev1) / 1e3
            (rates_one_node if one_node else rates)[st] = n * n * args.steps / t / 1e6
            cav.close()
            del cav
            torch.cuda.empty_cache()
    m = c["parity_n"]
    cpu, ref, robs = cpu_baseline_reduced(phys, m, c["steps"])
    errors = {}
    for st in ("f32", "f16", "bf16"):
        # the schedule the MLUPS above were measured with
        cav = Cavity(m, m, stream=stream, storage=st, **phys)
        cav.set_schedule(*schedules[(st, False)]).set_fields().step(c["steps"])
        got, gobs = cav.fields(), cav.observables()
        e = {}
        un = np.linalg.norm(np.stack([ref["ux"], ref["uy"]]))
        e["u"] = float(np.linalg.norm(np.stack([got["ux"] - ref["ux"], got["uy"] - ref["uy"]])) / un)
        for k in ("Tf", "Ts"):
            e[k] = float(np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k]))
        e["rho_minus_1"] = float(np.linalg.norm(got["rho"] - ref["rho"])
                                 / np.linalg.norm(ref["rho"] - 1.0))
        for k in ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold"):
            e[k] = float(abs(gobs[k] - robs[k]) / abs(robs[k]))
        errors[st] = e
    peak, kind = load_peaks()
    bpl = {"f32": 152, "f16": 76, "bf16": 76}
    line = {"metric": "MLUPS (reduced-storage forms)", "value": rates["f16"], "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 math, f16 storage",
            "data": "synthetic",
            "config": {"workload": "porous LTNE cavity %dx%d, phi 0.6, Da 1e-2, Ra 1e6, H 1000"
                                   % (n, n), "parity_run": "%dx%d, %d steps vs FP64 oracle"
                                                           % (m, m, c["steps"])},
            "mlups": rates, "schedules": {st: list(schedules[(st, False)]) for st in rates},
            "mlups_one_node_per_thread": rates_one_node,
            "roofline": {st: {"achieved": bpl[st] * rates[st] * 1e6 / 1e9, "peak": peak,
                              "frac": bpl[st] * rates[st] * 1e6 / 1e9 / peak, "unit": "GB/s",
                              "peak_kind": kind} for st in rates},
            "errors_vs_fp64_oracle": errors, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """Reverse-mode form: 256 x 256 cavity, porosity U[0.4, 0.8] (seed 4),
    Ra 1e5, Da 1e-3 (Ergun), H 50; forward 4000 steps then the gradient of
    the hot-wall Nusselt average with respect to the per-node porosity and H
    (64-step checkpoint segments).  MLUPS = nodes x steps / (forward +
    recompute + reverse time), next to the plain FP32 forward."""
    import math

    import torch

    torch.cuda.set_device(0)
    from paper_1608_04118_gb300 import build as B

    B.build()
    from paper_1608_04118_gb300.ltne import Cavity, LTNE_K_ERGUN

    c = W.C4_ADJOINT
    nx, ny = (c["nx"], c["ny"]) if args.n == 4096 else (args.n, args.n)
    steps = args.steps if args.steps != 2000 else c["steps"]
    seg = int(math.ceil(math.sqrt(steps)))
    phi = W.porosity_field(nx, ny, c["phi_lo"], c["phi_hi"], c["seed"]).reshape(-1)
    kw = {k: c[k] for k in ("Ra", "Pr", "Da", "H", "gamma_sf", "sigma", "T_hot", "T_cold",
                            "T_ref")}
    stream = torch.cuda.Stream()
    cav = Cavity(nx, ny, stream=stream, storage="f32", permeability=LTNE_K_ERGUN,
                 porosity_field=1, **kw)
    cav.adjoint(phi, 64, segment=8)  # warm-up (kernels loaded, allocator primed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, g, dH = cav.adjoint(phi, steps, segment=seg)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    cav.set_fields(porosity=phi)
    with torch.cuda.stream(stream):
        cav.step(max(args.warmup, 3))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    cav.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_fwd = ev0.elapsed_time(ev1) / 1e3
    nodes = nx * ny

    # context: the same physics on a 1024^2 lattice (1000 steps), where a
    # step is several waves of blocks rather than one latency-bound wave
    def adjoint_mlups(n, k, sched):
        ph = W.porosity_field(n, n, c["phi_lo"], c["phi_hi"], c["seed"]).reshape(-1)
        cv = Cavity(n, n, stream=stream, storage="f32", permeability=LTNE_K_ERGUN,
                    porosity_field=1, **kw).set_adjoint_schedule(sched)
        sg = int(math.ceil(math.sqrt(k)))
        cv.adjoint(ph, 2 * sg, segment=sg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cv.adjoint(ph, k, segment=sg)
        torch.cuda.synchronize()
        cv.close()
        return n * n * k / (time.perf_counter() - t0) / 1e6

    def at_size(n, k):
        ph = W.porosity_field(n, n, c["phi_lo"], c["phi_hi"], c["seed"]).reshape(-1)
        cv = Cavity(n, n, stream=stream, storage="f32", permeability=LTNE_K_ERGUN,
                    porosity_field=1, **kw)
        sg = int(math.ceil(math.sqrt(k)))
        cv.adjoint(ph, 2 * sg, segment=sg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cv.adjoint(ph, k, segment=sg)
        torch.cuda.synchronize()
        ta = time.perf_counter() - t0
        cv.set_fields(porosity=ph)
        with torch.cuda.stream(stream):
            cv.step(20)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cv.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        tf = e0.elapsed_time(e1) / 1e3
        cv.close()
        return {"n": n, "steps": k, "segment": sg, "mlups": n * n * k / ta / 1e6,
                "plain_forward_mlups": n * n * k / tf / 1e6, "ratio_to_plain_forward": tf / ta}

    big = None if args.no_context else at_size(1024, 1000)
    # the two register budgets of the transposed collision (the default
    # picks by lattice size)
    forms = None if args.no_context else {
        "%dx%d" % (m, m): {"one_wave": adjoint_mlups(m, k, 1), "capped": adjoint_mlups(m, k, 2)}
        for m, k in ((nx, steps), (1024, 1000))}
    line = {"metric": "MLUPS (forward + adjoint, %dx%d)" % (nx, ny),
            "value": nodes * steps / t_adj / 1e6,
            "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "porous LTNE cavity %dx%d, porosity U[0.4,0.8] seed 4, "
                                   "Ergun mean Da 1e-3, Ra 1e5, H 50" % (nx, ny), "segment": seg,
                       "objective": "(Nu_f,hot + Nu_s,hot)/2 at the last step"},
            "seconds": t_adj, "plain_forward_mlups": nodes * steps / t_fwd / 1e6,
            "ratio_to_plain_forward": (nodes * steps / t_adj) / (nodes * steps / t_fwd),
            "J": J, "dJ_dH": dH, "max_abs_dJ_dphi": float(g.abs().max()),
            "same_physics_1024": big, "register_budgets_mlups": forms}
    print(json.dumps(line), flush=True)


def run_slabs(args):
    """The 4096 x 4096 cavity of the default line cut into one row slab per
    rank (strong scaling): every step is followed by the halo exchange of
    five populations per column and cut, through NCCL on the slab's stream;
    the observables are the slabs' FP64 accumulators combined in rank
    order.  Same timing rules as the default line (barrier, events on the
    stream, max over ranks)."""
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    torch.cuda.set_device(local if ws > 1 else 0)
    dist.init_process_group("nccl" if ws > 1 else "gloo", rank=rank, world_size=ws,
                            **({} if ws > 1 else {"init_method": "tcp://127.0.0.1:%d"
                                                  % _free_port()}))
    from paper_1608_04118_gb300 import build as B

    B.build()
    from paper_1608_04118_gb300.ltne import LTNE_K_ERGUN, ltne_ergun_diameter
    from paper_1608_04118_gb300.slabs import DistributedCavity

    c = W.C2_THROUGHPUT
    n = args.n
    phi = W.porosity_field(n, n, c["phi_lo"], c["phi_hi"], c["seed"]).reshape(-1)
    d = ltne_ergun_diameter(phi, n - 1, c["Da"])
    kw = dict(Ra=c["Ra"], Pr=c["Pr"], Da=c["Da"], H=c["H"], gamma_sf=c["gamma_sf"],
              sigma=c["sigma"], T_hot=c["T_hot"], T_cold=c["T_cold"], T_ref=c["T_ref"], d_p=d)
    stream = torch.cuda.Stream()
    dc = DistributedCavity(n, n, stream=stream, storage=args.storage, permeability=LTNE_K_ERGUN,
                           porosity_field=1, **kw)
    dc.set_fields(porosity=phi)
    dc.step(max(args.warmup, 3))
    torch.cuda.synchronize()
    dist.barrier()
    l0 = dc.slab.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    dc.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    t = ev0.elapsed_time(ev1) / 1e3
    t_max = max_over_ranks(t, torch.device("cuda", torch.cuda.current_device()))
    ob = dc.observables()
    # step kernels, plus the pack and unpack kernels of every step when the
    # slab has a neighbour
    launches = (dc.slab.launches - l0) * (3 if ws > 1 else 1)
    if rank == 0:
        value = n * n * args.steps / t_max / 1e6
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                "storage": args.storage, "data": "synthetic",
                "config": dict(workload_config(n, args.storage),
                               parallelism="row slabs x%d (one cavity, halo exchange per step)"
                                           % ws),
                "gpu_launches": int(launches),
                "observables": {"Nu_f_hot": ob["Nu_f_hot"], "nonfinite": ob["nonfinite"],
                                "step": ob["step"]}}
        print(json.dumps(line), flush=True)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.split == "slabs":
        run_slabs(args)
        return
    if args.workload == "c3":
        run_batch(args)
        return
    if args.workload == "c4":
        run_adjoint(args)
        return
    if args.workload == "c5":
        run_reduced(args)
        return
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1608_04118_gb300 import build as B

    B.build()
    from paper_1608_04118_gb300.ltne import Cavity, FIELD_KEYS, LTNE_HOST_IO_DIRECT, LTNE_K_ERGUN

    c = W.C2_THROUGHPUT
    n = args.n
    phi = W.porosity_field(n, n, c["phi_lo"], c["phi_hi"], replica_seed(c["seed"], rank)).reshape(-1)
    kw = dict(Ra=c["Ra"], Pr=c["Pr"], Da=c["Da"], H=c["H"], gamma_sf=c["gamma_sf"],
              sigma=c["sigma"], T_hot=c["T_hot"], T_cold=c["T_cold"], T_ref=c["T_ref"])
    stream = torch.cuda.Stream(dev)
    cav = Cavity(n, n, stream=stream, storage=args.storage, permeability=LTNE_K_ERGUN,
                 porosity_field=1, **kw)
    if args.block or args.npt:
        if args.block:
            bx, by = (int(v) for v in args.block.split(","))
        elif args.npt == 1:
            bx, by = 64, 2
        else:  # the library's two-node block shape for this storage (128 x 1 for FP32)
            bx, by = cav.schedule[:2] if cav.schedule[2] >= 2 else (128, 1)
        cav.set_schedule(bx, by, args.npt or cav.schedule[2])
    if args.staging >= 0:
        cav.set_staging(args.staging)
    schedule = cav.schedule
    cav.set_fields(porosity=phi)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident throughput ----
    with torch.cuda.stream(stream):
        cav.step(max(args.warmup, 3))
    barrier()
    sampler = None if args.no_clocks else ClockSampler(local)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    launches0 = cav.launches
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    cav.step(args.steps)
    ev1.record(stream)
    barrier()
    clocks = sampler.stop() if sampler else None
    t = ev0.elapsed_time(ev1) / 1e3
    launches = cav.launches - launches0
    t_max = max_over_ranks(t, dev)
    nodes = n * n
    value = whole_job_mlups(nodes, args.steps, ws, t_max)
    per_launch = t / args.steps
    peak, peak_kind = load_peaks()
    achieved = BYTES_PER_LUP[args.storage] * nodes / per_launch / 1e9
    traffic, traffic_how = kernel_traffic(args.storage, n, schedule[2])
    ob = cav.observables()
    # The FP64 observables: one ltne_observables call (the reduction pass
    # over the fields and the residual snapshot, its combination, the
    # 18-value read-back and the host finish), median of 5, each after a
    # one-step call so that the residual compares two different states.
    obs_t = []
    for _ in range(5):
        cav.step(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cav.observables()
        e1.record(stream)
        e1.synchronize()
        obs_t.append(e0.elapsed_time(e1) / 1e3)
    obs_s = sorted(obs_t)[2]
    esz = 8 if args.storage == "f64" else 4
    # reads: the 5 field planes, the porosity and the 4 snapshot planes (u_x,
    # u_y, T_f, T_s of the previous call's fields; nothing is written back)
    obs_bytes = (5 + 1 + 4) * esz * nodes

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not args.no_e2e:
        k = args.steps
        # the caller's host arrays, page-locked (torch pinned memory) and
        # reused from run to run: the porosity input and the five fields,
        # allocated and filled before one untimed run of the sequence
        def pinned(shape):
            return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()

        phi_in = pinned(phi.shape)
        phi_in[...] = phi
        host_out = {key: pinned((n, n)) for key in FIELD_KEYS}
        cav.set_fields(porosity=phi_in).step(1).fields(out=host_out)
        cav.observables()
        direct = cav.host_io == LTNE_HOST_IO_DIRECT
        barrier()
        t0 = time.perf_counter()
        cav.set_fields(porosity=phi_in)  # H2D of the porosity; fields at rest, T = T_ref
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        cav.step(k)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        cav.fields(out=host_out)      # D2H of the fields
        host_ob = cav.observables()   # D2H of the observables
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        te = t3 - t0
        tt = max_over_ranks(te, dev)
        # bytes crossing to and from the host: the porosity plane and the five
        # fields, as the caller's FP64 values (direct: kernels read and write
        # the host arrays) or in the compute type (staged copies); the
        # initial fields are the defaults, zero deviations set on the device;
        # plus the observables' accumulators
        hsz = 8 if direct else esz
        h2d = nodes * hsz
        d2h = 5 * nodes * hsz + 18 * 8
        e2e = {"value": whole_job_mlups(nodes, k, ws, tt), "unit": UNIT,
               "h2d_bytes_per_step": h2d / k, "d2h_bytes_per_step": d2h / k,
               "note": "whole run through the C ABI: set_fields from a host array, %d steps, "
                       "get_fields + observables to host; the caller's float64 arrays are "
                       "page-locked and reused" % k,
               "host_io": "direct (kernels read and write the host arrays)" if direct
                          else "staged (pinned buffers, host conversion)",
               "phases_s": {"set_fields": t1 - t0, "steps": t2 - t1,
                            "get_fields_and_observables": t3 - t2}}
        assert host_ob["nonfinite"] == 0 and np.isfinite(host_out["Tf"]).all()

    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    cpu = None if (args.no_cpu_baseline or ws > 1) else cpu_baseline_oracle(n)
    forms = None
    if not args.no_forms and ws == 1:
        del cav
        torch.cuda.empty_cache()
        gpu = None if args.no_clocks else local
        forms = {"plain_fp32_1024": form_plain_1024(stream, peak, gpu),
                 "batched_256_cavities": form_batched(stream, value, peak, gpu),
                 "adjoint_256": form_adjoint(stream, peak, gpu),
                 "reduced_storage_8192": form_reduced(stream, value, peak, gpu)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.storage == "f64" else "f32", "storage": args.storage,
        "data": "synthetic",
        "config": dict(workload_config(n, args.storage),
                       schedule={"block": [schedule[0], schedule[1]],
                                 "nodes_per_thread": schedule[2]}),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "frac_of_8TBs": achieved / 8000.0,
                     "bytes_per_lup": BYTES_PER_LUP[args.storage],
                     "traffic": traffic, "traffic_source": traffic_how,
                     # the ncu-counted bytes of one launch over the launch time
                     "achieved_dram": None if traffic is None else traffic / per_launch / 1e9,
                     "kernel": "%s<%s> (one launch = one step of %d nodes)"
                               % ("k_step_pair" if schedule[2] == 2 else "k_step", args.storage,
                                  nodes)},
        "observables_reduction": {"ms": obs_s * 1e3,
                                  "note": "one ltne_observables call after a one-step call: "
                                          "both passes, the read-back and its synchronisation",
                                  "bytes_per_node": obs_bytes // nodes,
                                  "achieved_GBps": obs_bytes / obs_s / 1e9,
                                  "frac_of_peak": obs_bytes / obs_s / 1e9 / peak},
        "gpu_launches": int(launches),
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
        "observables": {"Nu_f_hot": ob["Nu_f_hot"], "Nu_s_hot": ob["Nu_s_hot"],
                        "nonfinite": ob["nonfinite"], "step": ob["step"]},
        "forms": forms,
    }
    if ws > 1:
        line["config"]["parallelism"] = "replicas x%d (independent cavities)" % ws
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
