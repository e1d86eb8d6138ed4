#!/usr/bin/env python3
"""MD throughput of the Allegro-FM energy/force path on GB300 (one JSON line on stdout).

Workload (default): the large NVE MD system, a 4,194,304-atom SiO2-like amorphous solid
(1,398,101 Si + 2,796,203 O on a jittered 162^3 lattice, 2.2 g/cm^3, periodic cube of
398.75 A), l<=2 / 3-layer / 32-channel model (rc 6 A, skin 1 A, seeded random-init
weights) with BF16 tensor-core MLPs and the FP32 adjoint; velocity Verlet at 1 fs from
300 K.  One step = kick, drift, neighbour maintenance, energies (per atom and per system)
+ forces (forward + hand-written adjoint), kick.  After the BF16 timing the same
workload is timed on the plain FP32 path (a few steps) and both force fields are
compared with the FP64 oracle on sampled atoms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--precision 0|1] [--fp32-steps K32]

Under torchrun (N > 1) every rank runs an independent replica (weak scaling); rank 0
prints the line with the max-over-ranks time.  --impl reference times the FP64 CPU
oracle on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

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

import synth  # noqa: E402

# the headline metric; both arms print it on the same workload, unit and direction
METRIC = "MD atom-steps/s (E+F, 1 GB300) at stated force error vs FP64 oracle; % roofline"
UNIT = "atom-steps/s"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.070 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
L2_FLUSH_BYTES = 512 << 20

WORKLOADS = {
    "water12288": dict(desc="4,096 H2O (12,288 atoms), periodic cube 49.67 A, 1.0 g/cm3",
                       make=lambda: synth.water_system(4096, L=49.67, seed=1001),
                       model="fm_water", nu="water12288"),
    "water4095": dict(desc="1,365 H2O (4,095 atoms), periodic cube 34.44 A, 1.0 g/cm3",
                      make=lambda: synth.water_system(1365, L=34.44, seed=1001),
                      model="fm_water", nu="water4095"),
    "csh131072": dict(desc="C-S-H-like solid, 131,072 atoms, 2.6 g/cm3",
                      make=lambda: synth.csh_system(False, 1002), model="fm_water",
                      nu="csh131072"),
    "cubic96": dict(desc="96 atoms, cubic 10 A, l<=1 model", make=synth.config1_system,
                    model="small", nu="cubic96"),
    "sio2_4194304": dict(desc="SiO2-like solid, 4,194,304 atoms, 2.2 g/cm3, L = 398.75 A",
                         make=lambda: synth.sio2_system(162, 4194304, 1004),
                         model="fm_water", nu="sio2_4194304", dt_fs=1.0),
    "csh_np6326": dict(desc="C-S-H nanoparticle in H2O/CO2, 6,326 atoms (267 C, 90 Ca, 133 Si, "
                            "2,577 O, 3,259 H), periodic (45.7 A)^3",
                       make=lambda: synth.nanoparticle_mixture_system(1005), model="fm_water",
                       nu="csh_np6326"),
    "molecules1024": dict(desc="1,024 organic molecules (7-23 heavy atoms + H), non-periodic",
                          make=lambda: synth.molecules_system(1024, 1003), model="fm_water",
                          nu="molecules1024"),
}


def model_hp(wl):
    hp = synth.preset(WORKLOADS[wl]["model"])
    hp["avg_num_neighbors"] = synth.NU[WORKLOADS[wl]["nu"]]
    return hp


def gemm_flops_per_edge(hp):
    """Algorithmic FLOPs of the MLP matrix products per edge and E+F evaluation: every
    dense layer of the two-body (after the embedding/radial input layer), environment
    and latent MLPs, forward (x W) and the adjoint's input gradient (g W^T)."""
    tb, lat = hp["two_body"], hp["latent"]
    D = tb[-1]
    C, lmax = hp["channels"], hp["lmax"]
    ldw = (lmax + 1) * C
    ldx = D + (lmax + 1) * C
    mac = sum(tb[k - 1] * tb[k] for k in range(1, len(tb)))
    per_layer = D * ldw + ldx * lat[0] + sum(lat[k - 1] * lat[k] for k in range(1, len(lat)))
    mac += hp["n_layers"] * per_layer
    return 2 * 2 * mac


def method_flops_per_edge(hp):
    """Algorithmic FLOPs per edge of one E+F evaluation on the matrix units: every dense
    layer of the method counted as the model defines it -- the radial input layer of the
    two-body MLP (n_basis -> first width; the species one-hot rows are lookups), its hidden
    layers, per interaction layer the environment projection and the latent MLP over
    [x | scalars], and the edge-energy MLP (hidden widths -> 1) -- forward plus the
    adjoint's input gradients of the same shapes (2 FLOP per multiply-add, x2 for the
    adjoint).  Recomputation and the folding of the linear readout into one vector are
    implementation choices and are not counted."""
    tb, lat, ee = hp["two_body"], hp["latent"], list(hp["edge_eng"])
    D = tb[-1]
    C, lmax = hp["channels"], hp["lmax"]
    ldw = (lmax + 1) * C
    mac = hp["n_basis"] * tb[0]
    mac += sum(tb[k - 1] * tb[k] for k in range(1, len(tb)))
    fan = D + ldw
    per_layer = D * ldw
    for w in lat:
        per_layer += fan * w
        fan = w
    mac += hp["n_layers"] * per_layer
    fan = D
    for w in ee + [1]:
        mac += fan * w
        fan = w
    return 2 * 2 * mac


def gemm_bytes_per_edge(hp, precision):
    """Compulsory HBM bytes per edge of all MLP GEMM launches of one E+F evaluation: each
    operand read once, each epilogue input read once, each output written once, in the
    storage types of the path.  Precision 0: FP32 everywhere; the adjoint's latent-input
    and env-weight products are two GEMMs.  Precision 1: BF16 GEMM operands, stored
    pre-activations, residual stream and env weights (the env projection's output), FP32
    gradients; the last latent GEMM carries the
    edge-energy readout (per-edge energy, envelope seed and bf16 dE/dz out, no latent
    stored) when D <= 256; the adjoint computes the scalar gradients first and then one
    GEMM over the concatenated [dE/dz | dE/dw]."""
    tb, lat = hp["two_body"], hp["latent"]
    D = tb[-1]
    C, lmax, NL = hp["channels"], hp["lmax"], hp["n_layers"]
    ldw = (lmax + 1) * C
    ldx = D + (lmax + 1) * C
    tc = precision == 1
    head = tc and D <= 256
    sa = 2 if tc else 4                      # bytes of a GEMM operand element
    sz = 2 if tc else 4                      # bytes of a stored pre-activation
    cp = 2 if tc else 0                      # extra bf16 copy of the residual stream
    sx = 2 if tc else 4                      # bytes of a stored residual-stream element
    sw = 2 if tc else 4                      # bytes of a stored env weight
    b = 0
    for k in range(1, len(tb)):              # two-body hidden layers
        b += tb[k - 1] * sa + tb[k] * sz
        b += (tb[k] * sx + 4) if k == len(tb) - 1 else tb[k] * sa
    for L in range(1, NL + 1):
        b += D * sa + ldw * sw               # environment projection
        fan = ldx
        for k, w in enumerate(lat):
            b += fan * sa
            if k < len(lat) - 1:
                b += w * sz + w * sa
            elif head and L == NL:
                b += D * sx + 4 + D * 2 + 4 + 4   # residual, f; dE/dz, E_e, envelope seed
            else:
                fp32_copy = D * 4 if (tc and L == NL) else 0   # x^N for the readout
                b += w * sz + 2 * D * sx + fp32_copy + 4
            fan = w
    for L in range(NL, 0, -1):               # adjoint
        for k in range(len(lat) - 1, 0, -1):
            b += lat[k] * sa + lat[k - 1] * sz + lat[k - 1] * sa
        res = 0 if L == NL else D * 4
        if tc:
            b += lat[0] * sa + (ldx - D) * 4                 # scalar gradients
            b += lat[0] * sa + ldw * sa + res + D * 4        # [dE/dz | dE/dw] product
        else:
            b += lat[0] * sa + res + ldx * 4
            b += ldw * sa + 2 * D * 4
    for k in range(len(tb) - 1, 0, -1):
        b += tb[k] * sa + tb[k - 1] * sz + tb[k - 1] * (sa if k > 1 else 4)
    return b


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        """Summary of the samples taken between mark('t0') and mark('t1')."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        t0 = getattr(self, "t0", 0.0)
        t1 = getattr(self, "t1", float("inf"))
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            parts = [p.strip() for p in ln.split(",")][1:]
            if len(parts) < 7 or not (t0 - 0.25 <= ts <= t1 + 0.25):
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


def traffic_per_edge(kernel):
    """DRAM bytes per edge of a kernel class from the committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", "traffic_per_edge.txt")
    try:
        for ln in open(path):
            parts = ln.split()
            if len(parts) >= 2 and parts[0] == kernel and not ln.startswith("#"):
                return float(parts[1])
    except OSError:
        pass
    return None


# ------------------------------------------------------------------------- oracle arm
def oracle_leg(wl, pos, F_paths, n_atoms=24, workers=None):
    """Time the FP64 oracle (spawn pool over all host cores) on the centres that the
    forces of `n_atoms` sampled atoms need, and compare those oracle forces with each
    force field in F_paths ({name: F [n, 3]}, all at positions `pos`)."""
    from oracle import neighbors, pool
    s = WORKLOADS[wl]["make"]()
    hp = model_hp(wl)
    workers = workers or os.cpu_count() or 1
    atoms = np.linspace(0, s.n - 1, n_atoms).astype(int).tolist()
    nl = neighbors.neighbor_list(pos, s.box, s.pbc, hp["rc"], 0.0, s.sys_ptr, centres=atoms)
    need = set(atoms)
    for m in atoms:
        need.update(int(j) for j in nl[m][0])
    centres = sorted(need)
    t0 = time.perf_counter()
    terms = pool.centre_terms(hp, 42, pos, s.Z, s.box, s.pbc, centres, s.sys_ptr,
                              workers=workers)
    dt = time.perf_counter() - t0
    F_ref = {}
    for m in atoms:
        Fm = terms[m][3].sum(axis=0)
        for i in sorted(set(int(j) for j in nl[m][0])):
            col, g = terms[i][1], terms[i][3]
            Fm = Fm - g[col == m].sum(axis=0)
        F_ref[m] = Fm
    cpu = {"value": len(centres) / dt, "unit": UNIT, "cores": workers,
           "kind": "oracle",
           "sample": f"E+F of {len(centres)} centres of {wl} (the neighbourhoods of {n_atoms} "
                     f"atoms), {dt:.1f} s on a spawn pool of {workers} processes"}
    ferrs = {}
    for name, F in F_paths.items():
        d = np.array([F[m] - F_ref[m] for m in atoms])
        ferrs[name] = {"rmse_meV_per_A": float(np.sqrt((d ** 2).mean()) * 1e3),
                       "max_meV_per_A": float(np.abs(d).max() * 1e3),
                       "sample": f"forces on {n_atoms} atoms at the final positions vs the "
                                 "FP64 oracle"}
    return cpu, ferrs


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import pool
    wl = args.workload
    s = WORKLOADS[wl]["make"]()
    hp = model_hp(wl)
    workers = os.cpu_count() or 1
    # size one step (E+F of a sample of centres) so the whole run takes about 3 minutes
    probe = list(range(min(s.n, 2 * workers)))
    t0 = time.perf_counter()
    pool.centre_terms(hp, 42, s.pos, s.Z, s.box, s.pbc, probe, workers=workers)
    t_probe = time.perf_counter() - t0
    per_step = 150.0 / max(1, args.steps + args.warmup)
    n = int(min(s.n, max(len(probe), len(probe) * per_step / max(t_probe, 1e-3))))
    centres = list(range(n))
    for _ in range(args.warmup):
        pool.centre_terms(hp, 42, s.pos, s.Z, s.box, s.pbc, centres, workers=workers)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pool.centre_terms(hp, 42, s.pos, s.Z, s.box, s.pbc, centres, workers=workers)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded), random-init weights",
        "config": {"workload": wl, "desc": WORKLOADS[wl]["desc"], "model": WORKLOADS[wl]["model"],
                   "atoms": s.n, "dt_fs": WORKLOADS[wl].get("dt_fs", 0.5),
                   "parallelism": f"{workers} host processes (rank 0)",
                   "sample_atoms_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers,
                         "kind": "oracle",
                         "sample": f"E+F of centres 0..{n - 1} of {wl} per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2502_06073_gb300 as ff

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl = args.workload
    s = WORKLOADS[wl]["make"]()
    hp = model_hp(wl)
    model = ff.FFModel(hp, seed=42, precision=args.precision)
    x = torch.tensor(s.pos, dtype=torch.float64, device=dev)
    Z = torch.tensor(s.Z, dtype=torch.int32, device=dev)
    mass = torch.tensor(s.masses, dtype=torch.float64, device=dev)
    v0 = synth.maxwell_boltzmann(s.masses, 300.0, seed=7)
    v = torch.tensor(v0, dtype=torch.float64, device=dev)
    multi = s.sys_ptr.shape[0] > 2
    sys_ptr = s.sys_ptr if multi else None
    model.bind(x, Z, s.box, s.pbc, sys_ptr)
    tuned = None
    if args.autotune and args.precision == 1:
        tuned = model.autotune(x)
    if args.graph:
        model.set_graph(True)
    # 0.5 fs (the paper's MD step) unless the workload states its own
    dt_fs = WORKLOADS[args.workload].get("dt_fs", 0.5)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # nvidia-smi starts before the warm-up: its start-up stalls the GPU for tens of ms
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)
    for _ in range(args.warmup):
        model.md(x, v, mass, 1, dt_fs, energies=True)
    torch.cuda.synchronize()
    E_edges = model.edges()[1].shape[0]

    # ---- timed region: K MD steps (energies per atom and per system + forces each step),
    # device-timed per step, L2 flushed between steps
    def timed_steps(nsteps, profile):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        if profile:
            ff.profile_enable(True)
            ff.profile_read()
        for k in range(nsteps):
            flush.zero_()
            ev[k][0].record(stream)
            model.md(x, v, mass, 1, dt_fs, energies=True)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        prof = None
        if profile:
            prof = ff.profile_read()
            ff.profile_enable(False)
        return [a.elapsed_time(b) for a, b in ev], prof

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark("t0")
    l0 = model.launches()
    step_ms, _ = timed_steps(args.steps, False)
    launches = model.launches() - l0
    clocks.mark("t1")
    clk = clocks.stop()
    # a few steps again with every launch bracketed by events (per-kernel durations for the
    # roofline; kept out of the headline timing).  A graph replay carries no per-launch
    # events, so with --graph this pass launches the same kernels eagerly (one untimed step
    # first, which evaluates the forces at the current positions)
    if args.graph:
        model.set_graph(False)
        model.md(x, v, mass, 1, dt_fs, energies=True)
    n_prof = min(args.steps, args.profile_steps)
    prof_ms, prof = timed_steps(n_prof, True)
    E_prof = model.edges()[1].shape[0] if args.graph else E_edges
    if args.graph:
        model.set_graph(True)
    t_total = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([t_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_total = float(t.item())
        dist.barrier()
    value = world * s.n * args.steps / t_total

    # ---- e2e: same steps through the C ABI with host buffers (H2D inputs, D2H results)
    xh = x.cpu().pin_memory()
    vh = v.cpu().pin_memory()
    xo = torch.empty_like(xh).pin_memory()
    vo = torch.empty_like(vh).pin_memory()
    eo = torch.empty(1, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        x.copy_(xh, non_blocking=True)
        v.copy_(vh, non_blocking=True)
        Ep, _ = model.md(x, v, mass, 1, dt_fs, energies=True)
        xo.copy_(x, non_blocking=True)
        vo.copy_(v, non_blocking=True)
        eo.copy_(Ep[:1], non_blocking=True)
        xh, xo = xo, xh
        vh, vo = vo, vh
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = e0.elapsed_time(e1) / 1e3
    if world > 1:
        t = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = float(t.item())
    e2e = world * s.n * args.steps / t_e2e
    h2d = 2 * s.n * 3 * 8
    d2h = 2 * s.n * 3 * 8 + 8

    # ---- roofline of the dominant kernel class (per-kernel CUDA events of the profiled
    # pass); the contraction classes are measured against the matrix-unit work the method
    # defines (method_flops_per_edge), not against what this implementation stores
    pk, pk_kind = peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_launch, dom_ms) = dom
    method_flop = method_flops_per_edge(hp) * E_prof * n_prof
    if dom_name == "gemm_f32":
        achieved = method_flop / (dom_ms / 1e3) / 1e12
        peak = FP32_PEAK_TFLOPS
        roof = {"kernel": "gemm_f32 (all FP32 MLP GEMM launches)", "bound": "alu",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.070 GHz",
                "flop_per_edge": method_flops_per_edge(hp),
                "launches": dom_launch, "avg_launch_us": 1e3 * dom_ms / max(dom_launch, 1)}
        tpe = traffic_per_edge("gemm_f32")
        roof["traffic"] = (tpe * E_prof * n_prof / max(dom_launch, 1)) if tpe else None
    elif dom_name == "gemm_bf16":
        t_s = dom_ms / 1e3
        achieved = method_flop / t_s / 1e12
        byts = gemm_bytes_per_edge(hp, 1) * E_prof * n_prof
        roof = {"kernel": "gemm_bf16 (tcgen05, all MLP GEMM launches)", "bound": "tensor",
                "achieved": achieved, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                "frac": achieved / pk["bf16_tflops"],
                "peak_source": f"bf16_tflops burst ({pk_kind})",
                "frac_of_sustained": achieved / pk["bf16_tflops_sustained"],
                "flop_per_edge": method_flops_per_edge(hp),
                "unfused_gemm_bytes_per_edge": gemm_bytes_per_edge(hp, 1),
                "unfused_bytes_hbm_frac": byts / t_s / 1e9 / pk["hbm_gbs"],
                "launches": dom_launch, "avg_launch_us": 1e3 * dom_ms / max(dom_launch, 1)}
        tpe = traffic_per_edge("gemm_bf16")
        roof["traffic"] = (tpe * E_prof * n_prof / max(dom_launch, 1)) if tpe else None
    else:
        roof = {"kernel": dom_name, "bound": "hbm", "achieved": None, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": None, "traffic": None}
    # the whole step against the same matrix-unit work (what the fused design is bound by)
    step_flop = method_flops_per_edge(hp) * E_edges * args.steps
    tensor_peak = pk["bf16_tflops"] if args.precision == 1 else FP32_PEAK_TFLOPS
    roof["step_tensor_tflops"] = step_flop / t_total / 1e12
    roof["step_tensor_frac"] = step_flop / t_total / 1e12 / tensor_peak

    # ---- NVE energy drift (optional): linear fit of E_pot + E_kin per atom over a run
    drift = None
    if args.drift_steps > 0 and rank == 0:
        try:
            Ep, Ek = model.md(x, v, mass, args.drift_steps, dt_fs, energies=True)
            et = (Ep + Ek).cpu().numpy() / s.n
            tt = np.arange(1, args.drift_steps + 1) * dt_fs * 1e-6            # ns
            slope = float(np.polyfit(tt, et, 1)[0])
            drift = {"eV_per_atom_per_ns": slope, "steps": args.drift_steps, "dt_fs": dt_fs,
                     "fluctuation_eV_per_atom": float(et.std()),
                     "E_tot_first_last_eV_per_atom": [float(et[0]), float(et[-1])]}
        except ff.FFError as exc:      # e.g. the random-weight system collapsing
            drift = {"error": str(exc), "steps": args.drift_steps}

    # forces of this path at the final positions (compared with the oracle below)
    x_end = x.clone()
    _, _, F_main = model.energy_forces(x_end, E_atom=False)
    F_main = F_main.double().cpu().numpy()
    model.close()
    del model
    torch.cuda.empty_cache()

    # ---- the plain FP32 path on the same workload (a few steps from the same state)
    fp32 = None
    F_32 = None
    if args.precision == 1 and args.fp32_steps > 0:
        m32 = ff.FFModel(hp, seed=42, precision=0)
        m32.bind(x_end, Z, s.box, s.pbc, sys_ptr)
        _, _, F32 = m32.energy_forces(x_end, E_atom=False)
        F_32 = F32.double().cpu().numpy()
        x32, v32 = x_end.clone(), v.clone()
        m32.md(x32, v32, mass, 1, dt_fs, energies=True)               # untimed warm-up step
        torch.cuda.synchronize()
        ev32 = []
        for _ in range(args.fp32_steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record(stream)
            m32.md(x32, v32, mass, 1, dt_fs, energies=True)
            b.record(stream)
            ev32.append((a, b))
        torch.cuda.synchronize()
        ms32 = [a.elapsed_time(b) for a, b in ev32]
        fp32 = {"value": s.n * len(ms32) / (sum(ms32) / 1e3), "unit": UNIT,
                "ms_per_step": sum(ms32) / len(ms32), "steps": len(ms32), "warmup": 2,
                "dtype": "f32", "bf16_speedup": (sum(ms32) / len(ms32)) /
                                                 (1e3 * t_total / args.steps)}
        m32.close()
        del m32
        torch.cuda.empty_cache()

    # ---- CPU-baseline leg: the FP64 oracle on a bounded sample of this workload (the
    # neighbourhoods of a few atoms at the final positions), timed; the same oracle
    # results give the force error of each path on those atoms
    cpu = ferr = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        Fs = {"main": F_main}
        if F_32 is not None:
            Fs["fp32"] = F_32
        cpu, ferrs = oracle_leg(wl, x_end.cpu().numpy(), Fs)
        ferr = ferrs["main"]
        if fp32 is not None:
            fp32["force_error"] = ferrs["fp32"]

    if rank == 0:
        line = {
            "metric": METRIC, "value": value,
            "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == 0 else "bf16-mlp/f32",
            "data": "synthetic (seeded), random-init weights",
            "config": {"workload": wl, "desc": WORKLOADS[wl]["desc"],
                       "model": WORKLOADS[wl]["model"], "atoms": s.n, "edges": E_edges,
                       "dt_fs": dt_fs, "parallelism": f"replicas x{world}",
                       "path": "CUDA graph on the frozen Verlet list" if args.graph
                               else "per-step filtered list",
                       "gemm_tiles": tuned or "default",
                       "l2": "flushed between timed steps (512 MiB write); per-step inputs "
                             "far larger than L2"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            "kernel_ms_per_step": {k: round(v[1] / n_prof, 4) for k, v in prof.items()
                                   if v[0]},
            "profiled_steps": n_prof,
            "profiled_ms_per_step": sum(prof_ms) / n_prof,
            "step_ms": [round(t, 3) for t in step_ms],
            "force_error": ferr,
            "fp32": fp32,
            "nve_drift": drift,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sio2_4194304", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1],
                    help="1: BF16 tensor-core MLPs (default); 0: plain FP32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp32-steps", type=int, default=2,
                    help="with --precision 1: time this many steps of the plain FP32 path on "
                         "the same workload after the main timing (0: skip)")
    ap.add_argument("--profile-steps", type=int, default=3,
                    help="steps of the per-kernel event pass that feeds the roofline")
    ap.add_argument("--drift-steps", type=int, default=0,
                    help="after timing, run this many NVE steps and fit the energy drift")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the tensor-core GEMM tile configuration before timing")
    ap.add_argument("--graph", action="store_true",
                    help="MD steps replay a captured CUDA graph on the frozen Verlet list")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
