"""Throughput of the fused D3Q19 TRT + CLI step (fluid MLUPS and HBM roofline).

Workload: the 256x256x512 channel with a porous layer z < 256 of r = 8 sphere
packings at porosities {0.4, 0.6, 0.8, 0.9} (one solver per porosity, FP32
storage); one bench step = one lattice time step of all four solvers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores instead (the
only other program here; see the "cpu_baseline" key).  Multi-GPU runs are
independent replicas (one process per GPU, no data exchange): the LBM of one
box runs on one GPU.
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

from paper_1507_06565_gb300 import workloads as W  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
METRIC = "fluid MLUPS (D3Q19 TRT + CLI stream-collide; HBM roofline fraction in 'roofline')"
WORKLOAD = ("256x256x512 channel, walls z=0/511, porous layer z<256 of overlapping r=8 spheres, "
            "porosity sweep {0.4,0.6,0.8,0.9} (one solver each); one step = one time step of all four")
# measured DRAM read + write bytes per fluid cell of one launch (FP32 storage,
# neighbour table outside the dense tiles): ncu on one full-size solver of the
# sweep (porosity 0.6, 26.7 M fluid cells), applied per fluid cell to all four
# (profiles/step_kernels_channel_256x256x512_phi06_dram.txt)
MEASURED_DRAM_B_PER_FLUP = {"even": 153.1, "odd": 180.3}
# the same for the batched REV cubes (table-only odd step), taken on the first
# 8 cubes (11.2 M fluid cells, far above L2) and applied per fluid cell to the
# 64-cube batch (profiles/step_kernels_rev_8cubes_dram.txt)
MEASURED_DRAM_B_PER_FLUP_REV = {"even": 153.2, "odd": 222.3}
# bounded samples of the workload for the CPU oracle: same sphere radius,
# porosity and channel structure at a reduced box
SAMPLE = W.Channel("W2-shaped sample 128x128x256 r=8 phi=0.6", 128, 128, 256, 1.0, 128.0, 8.0, 8.0, 0.6, True, 2060)
SAMPLE_STEP = W.Channel("W2-shaped sample 64x64x128 r=8 phi=0.6", 64, 64, 128, 1.0, 64.0, 8.0, 8.0, 0.6, True, 2060)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, device: str = "cuda") -> float:
    """The largest of `value` over all ranks (the slowest rank's time); the
    value itself without a process group."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ms: float, world: int) -> float:
    """Millions of units per second over the whole job: every rank processes
    the same units (replicas, weak scaling), the job takes the slowest rank's
    time."""
    return units_per_rank * world / (ms * 1e-3) / 1e6


def _peak_hbm():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_sample(steps: int, warmup: int):
    """FP64 oracle on the host cores over the small W2-shaped sample channel."""
    import oracle as O

    sp, _, rc = O.place_spheres(*SAMPLE_STEP.sphere_args())
    assert rc == 0
    lat = O.Lattice(SAMPLE_STEP.nx, SAMPLE_STEP.ny, SAMPLE_STEP.nz, False, sp, SAMPLE_STEP.tau, SAMPLE_STEP.lam,
                    SAMPLE_STEP.g).init()
    nf = int((lat.solid() == 0).sum())
    lat.step(warmup)
    t0 = time.perf_counter()
    lat.step(steps)
    dt = time.perf_counter() - t0
    return nf, dt, O.threads()


def cpu_baseline(seconds_hint: float = 15.0):
    import oracle as O

    sp, _, _ = O.place_spheres(*SAMPLE.sphere_args())
    lat = O.Lattice(SAMPLE.nx, SAMPLE.ny, SAMPLE.nz, False, sp, SAMPLE.tau, SAMPLE.lam, SAMPLE.g).init()
    nf = int((lat.solid() == 0).sum())
    t0 = time.perf_counter()
    lat.step(1)
    one = time.perf_counter() - t0
    n = max(2, min(200, int(seconds_hint / max(one, 1e-3))))
    t0 = time.perf_counter()
    lat.step(n)
    dt = time.perf_counter() - t0
    cores = O.threads()
    # the same oracle on one core, over the small sample, for a few seconds
    O.set_threads(1)
    try:
        sp1, _, _ = O.place_spheres(*SAMPLE_STEP.sphere_args())
        lat1 = O.Lattice(SAMPLE_STEP.nx, SAMPLE_STEP.ny, SAMPLE_STEP.nz, False, sp1, SAMPLE_STEP.tau, SAMPLE_STEP.lam,
                         SAMPLE_STEP.g).init()
        nf1 = int((lat1.solid() == 0).sum())
        lat1.step(1)
        t1 = time.perf_counter()
        lat1.step(3)
        dt1 = time.perf_counter() - t1
    finally:
        O.set_threads(cores)
    return {"value": nf * n / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{SAMPLE.name} ({nf} fluid cells), FP64 dense two-array oracle, {n} steps after 1 warm-up",
            "single_core": {"value": nf1 * 3 / dt1 / 1e6, "unit": "MLUPS", "cores": 1,
                            "sample": f"{SAMPLE_STEP.name} ({nf1} fluid cells), 3 steps after 1 warm-up"}}


def workload_name(args):
    name = None
    if args.workload == "channel":
        name = WORKLOAD
    if args.workload == "channel-half":
        name = (WORKLOAD.replace("256x256x512", "128x128x256").replace("z=0/511", "z=0/255")
                .replace("z<256", "z<128"))
    if name is not None:
        if getattr(args, "phi", None) is not None:
            name = name.replace("porosity sweep {0.4,0.6,0.8,0.9} (one solver each); one step = one time step of all four",
                                f"porosity {args.phi:g} (one solver)")
        return name
    if args.workload == "w0":
        return ("151^3 periodic cube, one centred sphere of diameter 90 (the paper's per-core block), "
                + ("simple bounce-back on every link" if args.bounce_back else "CLI walls"))
    if args.workload == "large":
        return ("512x512x1024 channel, walls z=0/1023, porous layer z<512 of overlapping r=8 spheres, porosity 0.6 "
                "(seed 3060); one step = one time step of the box")
    return (f"{args.cubes} periodic REV cubes (edge U[48,160], r U[3,10], porosity U[0.35,0.95], seeds 4000+i) "
            "as one batch: one launch per step for all cubes")


# Packings on which the cli-stability sweep (60,000 steps from a perturbed
# rest state, Eq. (CLI) wherever x_f2 exists) saw a perturbation grow: with
# --wall-rule auto these run with the corner safeguards
# (LBM_FLAG_CLI_SAFEGUARDS), every other packing with the paper's rule.  A
# batch takes the safeguards when any of its boxes needs them.
PAPER_CLI_UNSTABLE = {"W2 256x256x512 r=8 phi=0.4", "W3 512x512x1024 r=8 phi=0.6", "W4 cube 5 edge=149",
                      "W4 cube 17 edge=151", "W4 cube 47 edge=52"}
# workloads that always take the safeguards: the REV batch (cubes 5 and 17
# grow), the warm-start channels (held-out channel 600006 diverges) and the
# resolution studies (their D = 4 packing diverges under flow)
SAFEGUARDED_WORKLOADS = ("rev", "surrogate", "grid-study", "re-sweep")


def wall_rule(args, cases=()) -> str:
    rule = getattr(args, "wall_rule", "auto")
    if rule == "auto":
        if getattr(args, "workload", "channel") in SAFEGUARDED_WORKLOADS:
            return "safeguards"
        rule = "safeguards" if any(c.name in PAPER_CLI_UNSTABLE for c in cases) else "paper"
    return rule


def odd_flags(args, cases=()) -> int:
    """Library flags of a run: the odd-step neighbour source, forced simple
    bounce-back or staged even step, and the wall rule for these packings."""
    import paper_1507_06565_gb300 as L

    flags = {"auto": 0, "table": L.LBM_FLAG_NEIGHBOUR_TABLE, "rows": L.LBM_FLAG_ROW_NEIGHBOURS,
             "staged": L.LBM_FLAG_STAGED_NEIGHBOURS,
             "derived": L.LBM_FLAG_DERIVED_NEIGHBOURS}[getattr(args, "odd", "auto")]
    if getattr(args, "bounce_back", False):
        flags |= L.LBM_FLAG_SIMPLE_BOUNCE_BACK
    if getattr(args, "even", "auto") == "staged":
        flags |= L.LBM_FLAG_STAGED_EVEN
    refs = getattr(args, "plane_references", "auto")
    if refs == "on":
        flags |= L.LBM_FLAG_PLANE_REFERENCES
    elif refs == "off":
        flags |= L.LBM_FLAG_NO_PLANE_REFERENCES
    if wall_rule(args, cases) == "safeguards":
        flags |= L.LBM_FLAG_CLI_SAFEGUARDS
    return flags


def fallback_fraction(solver) -> dict:
    """Wall links of a solver and the fraction of them that take simple
    bounce-back instead of Eq. (CLI) under its wall rule."""
    fb = solver.link_fallback()
    return {"links": int(fb.size), "bounce_back_fraction": float(fb.mean()) if fb.size else 0.0}


def run_converge(args):
    """Time to steady state: run the workload until the plane-profile residual
    (largest over the parts) is below --tol, re-centring the density at every
    check; report wall time, steps and the permeability of every box."""
    import torch

    import paper_1507_06565_gb300 as L
    from paper_1507_06565_gb300.build import build

    build()
    L.load_library()
    if args.workload == "rev":
        cases = [W.W4_cube(i) for i in range(args.cubes)]
        geoms = [L.lbm_geometry_from_spheres(*c.sphere_args()) for c in cases]
        solvers = [L.BatchSolver(geoms, cases[0].tau, cases[0].lam, cases[0].g, args.storage,
                                 flags=odd_flags(args, cases))]
    else:
        phis = W.W2_POROSITIES if args.phi is None else [args.phi]
        cases = [W.W2(phi) if args.workload == "channel" else W.W2_half(phi) for phi in phis]
        geoms = [L.lbm_geometry_from_spheres(*c.sphere_args()) for c in cases]
        solvers = [L.Solver(g, c.tau, c.lam, c.g, args.storage, flags=odd_flags(args, [c]))
                   for g, c in zip(geoms, cases)]
    out = []
    total_s = 0.0
    for s, c in zip(solvers, cases):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, n, res = s.run_until(args.tol, args.interval, args.max_steps, criterion="profile")
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        total_s += dt
        rec = {}
        if isinstance(s, L.BatchSolver):
            k = s.permeabilities().tolist()
        else:
            k = [s.permeability(*c.perm_window)]
            # plane-averaged superficial u_x and porosity, every 8th plane (Sec. 3.1 profiles)
            pa = s.plane_average()
            rec = {"profile_z_every8": list(range(0, c.nz, 8)), "u_sup_every8": pa[::8, 0].tolist(),
                   "porosity_every8": pa[::8, 2].tolist()}
        out.append({"case": c.name, "wall_rule": wall_rule(args, [c]), "status": L.status_string(rc), "steps": n,
                    "residual": res, "seconds": dt, "mlups": s.info()["n_fluid"] * n / dt / 1e6,
                    "permeability": k, "schedule": s.schedule(), **rec})
    line = {"metric": f"time to steady state (plane-profile residual < {args.tol:g})", "value": total_s, "unit": "s",
            "higher_is_better": False, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": workload_name(args)}, "runs": out}
    print(json.dumps(line), flush=True)


def run_precision_check(args):
    """Converged error of FP16/BF16 storage (the reduced-precision
    configuration): for each porosity, the channel in FP32 storage is run to
    the profile tolerance from rest; FP16 and BF16 solvers then start from its
    velocity field and run to the same tolerance.  Reports the permeability
    and plane-profile differences of each against the FP32 result.  With
    --oracle-steps N the FP64 oracle (host cores) continues the converged FP32
    state for N steps and reports how far its profile moves, which bounds how
    far the FP32 steady state lies from the oracle's."""
    import torch

    import paper_1507_06565_gb300 as L
    from paper_1507_06565_gb300.build import build

    build()
    L.load_library()
    phis = W.W2_POROSITIES if args.phi is None else [args.phi]
    rows = []
    for phi in phis:
        c = W.W2(phi) if args.workload == "channel" else W.W2_half(phi)
        geom = L.lbm_geometry_from_spheres(*c.sphere_args())
        flags = odd_flags(args, [c])
        out = {"case": c.name, "wall_rule": wall_rule(args, [c]), "plane_references": args.plane_references}
        s32 = L.Solver(geom, c.tau, c.lam, c.g, "f32", flags=flags)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, n, res = s32.run_until(args.tol, args.interval, args.max_steps, criterion="profile")
        torch.cuda.synchronize()
        out["f32"] = {"status": L.status_string(rc), "steps": n, "residual": res, "seconds": time.perf_counter() - t0,
                      "permeability": s32.permeability(*c.perm_window)}
        pa32 = s32.plane_average()[:, 0]
        out["f32"]["u_sup_every8"] = pa32[::8].tolist()
        _, u32 = s32.moments()
        for st in ("f16", "bf16"):
            s = L.Solver(geom, c.tau, c.lam, c.g, st, u0=u32, flags=flags)
            t0 = time.perf_counter()
            rc, n, res = s.run_until(args.tol, args.interval, args.rp_max_steps, criterion="profile")
            torch.cuda.synchronize()
            k = s.permeability(*c.perm_window)
            pa = s.plane_average()[:, 0]
            out[st] = {"status": L.status_string(rc), "steps": n, "residual": res,
                       "seconds": time.perf_counter() - t0, "permeability": k,
                       "k_rel_vs_f32": k / out["f32"]["permeability"] - 1.0,
                       "profile_l2_rel_vs_f32": float(np.linalg.norm(pa - pa32) / np.linalg.norm(pa32)),
                       "profile_max_rel_vs_f32": float(np.max(np.abs(pa - pa32)) / np.max(np.abs(pa32)))}
            del s
        if args.oracle_steps > 0:
            import oracle as O

            lat = O.Lattice(c.nx, c.ny, c.nz, False, geom.spheres(), c.tau, c.lam, c.g,
                            cli_safeguards=wall_rule(args, [c]) == "safeguards")
            # the FP32 state as full populations f = h + w (lbm_populations
            # gives h for every fluid cell)
            h = s32.populations().cpu().numpy().astype(np.float64)
            fluid = s32.export_lists()["fluid_cell"]
            _, w = O.velocity_set()
            f = np.zeros((19, c.nz * c.ny * c.nx))
            f[:, fluid] = h + w[:, None]
            lat.set_f(f)
            p0 = lat.plane_average()[:, 0]
            t0 = time.perf_counter()
            lat.step(args.oracle_steps)
            p1 = lat.plane_average()[:, 0]
            out["oracle_continuation"] = {
                "steps": args.oracle_steps, "seconds": time.perf_counter() - t0, "threads": O.threads(),
                "profile_change_l2_rel": float(np.linalg.norm(p1 - p0) / np.linalg.norm(p1)),
                "profile_vs_gpu_l2_rel": float(np.linalg.norm(p0 - pa32) / np.linalg.norm(pa32)),
                "permeability_after": float(O.Lattice.permeability(lat, *c.perm_window))}
        rows.append(out)
        del s32
        torch.cuda.empty_cache()
    line = {"metric": f"converged FP16/BF16 error against FP32 (profile residual < {args.tol:g})", "unit": "relative",
            "value": max(abs(r[st]["k_rel_vs_f32"]) for r in rows for st in ("f16", "bf16")), "higher_is_better": False,
            "data": "synthetic", "config": {"workload": workload_name(args), "tol": args.tol}, "runs": rows}
    print(json.dumps(line), flush=True)


def unet_conv_flops(n, nz, ny, nx) -> float:
    """Multiply-adds x 2 of the 3x3x3 convolutions of one forward pass
    (27 taps x c_in x c_out per voxel of each layer's level)."""
    from paper_1507_06565_gb300.workloads import UNET_LAYERS

    level = {"enc1": 0, "enc2": 1, "enc3": 2, "bott": 3, "dec3": 2, "dec2": 1, "dec1": 0}
    v0 = n * nz * ny * nx
    return float(sum(2 * 27 * co * ci * v0 / 8 ** level[name[:4]] for name, co, ci in UNET_LAYERS))


def run_unet(args):
    """Training steps of the warm-start U-Net (forward, backward, Adam) on a
    batch of 4 seeded 64x64x128 fields, the warm-start training shape."""
    import torch

    import paper_1507_06565_gb300 as L
    from paper_1507_06565_gb300.build import build

    build()
    L.load_library()
    n, nz, ny, nx = 4, 128, 64, 64
    net = L.UNet(n, nz, ny, nx, params=W.unet_init(0))
    gen = torch.Generator(device="cuda").manual_seed(1)
    sdf = torch.rand((n, nz, ny, nx), device="cuda", generator=gen) * 2 - 1
    tgt = torch.rand((n, 3, nz, ny, nx), device="cuda", generator=gen) * 0.1
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        net.forward(sdf)
        net.backward(tgt)
        net.adam_step(1e-3)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fw = bw = 0.0
    for _ in range(args.steps):
        ev[0].record(stream)
        net.forward(sdf)
        ev[1].record(stream)
        net.backward(tgt)
        net.adam_step(1e-3)
        ev[2].record(stream)
        torch.cuda.synchronize()
        fw += ev[0].elapsed_time(ev[1])
        bw += ev[1].elapsed_time(ev[2])
    fw, bw = fw / args.steps, bw / args.steps
    flops = unet_conv_flops(n, nz, ny, nx)
    try:
        with open(PEAKS_FILE) as fh:
            peak, kind = float(json.load(fh)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        peak, kind = 1900.0, "fallback"
    achieved = 3 * flops / ((fw + bw) * 1e-3) / 1e12
    line = {"metric": "U-Net training step (forward, backward, Adam)", "value": 1e3 / (fw + bw),
            "unit": "steps/s", "higher_is_better": True, "ms_per_step": fw + bw, "forward_ms": fw,
            "backward_ms": bw, "steps": args.steps, "warmup": args.warmup, "dtype": "bf16 (fp32 accumulate)",
            "data": "synthetic",
            "config": {"workload": f"batch {n} of {nz}x{ny}x{nx} fields, 16/32/64/128 channels"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "peak_kind": kind,
                         "flops": "3 x forward convolution FLOPs (forward, input and weight gradients) per step"}}
    print(json.dumps(line), flush=True)


def run_unet_layers(args):
    """Per-layer throughput of the U-Net's tensor-core contractions (the
    training shape: batch 4 of 64x64x128 fields): every 3x3x3 layer's forward
    convolution, its input gradient (the same kernel with the transposed
    weights) and its weight gradient, each timed alone with CUDA events over
    --steps launches, as TFLOP/s against the bf16 peak and as GB/s of the
    activations it must read and write once."""
    import torch

    import paper_1507_06565_gb300 as L
    from paper_1507_06565_gb300.build import build
    from paper_1507_06565_gb300.workloads import UNET_LAYERS

    build()
    L.load_library()
    n, nz, ny, nx = 4, 128, 64, 64
    level = {"enc1": 0, "enc2": 1, "enc3": 2, "bott": 3, "dec3": 2, "dec2": 1, "dec1": 0}
    try:
        with open(PEAKS_FILE) as fh:
            peak, kind = float(json.load(fh)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        peak, kind = 1900.0, "fallback"
    hbm, _ = _peak_hbm()
    gen = torch.Generator(device="cuda").manual_seed(0)
    stream = torch.cuda.current_stream()
    rows = []
    for name, co, ci in UNET_LAYERS:
        lv = level[name[:4]]
        dims = (n, nz >> lv, ny >> lv, nx >> lv)
        V = int(np.prod(dims))
        x = (torch.rand((V, ci), device="cuda", generator=gen) - 0.5).to(torch.bfloat16)
        dy = (torch.rand((V, co), device="cuda", generator=gen) - 0.5).to(torch.bfloat16)
        w = ((torch.rand((27, co, ci), device="cuda", generator=gen) - 0.5) * 0.1).to(torch.bfloat16)
        wt = w.flip(0).transpose(1, 2).contiguous()   # the input gradient's weights
        b = torch.zeros(co, device="cuda")
        y = torch.empty((V, co), dtype=torch.bfloat16, device="cuda")
        dx = torch.empty((V, ci), dtype=torch.bfloat16, device="cuda")
        dw = torch.zeros((27, co, ci), device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        flops = 2.0 * 27 * co * ci * V
        rec = {"layer": name, "level": lv, "c_in": ci, "c_out": co, "voxels": V, "gflop": flops / 1e9}
        for kind_, fn, io in (
                ("forward", lambda: L.unet_conv3d(x, w, b, co, dims, True, out=y, status=status), V * (ci + co) * 2),
                ("input_grad", lambda: L.unet_conv3d(dy, wt, None, ci, dims, False, out=dx, status=status),
                 V * (ci + co) * 2),
                ("weight_grad", lambda: L.unet_conv3d_wgrad(dy, x, dims, dw=dw, status=status), V * (ci + co) * 2)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            tf = flops / (ms * 1e-3) / 1e12
            rec[kind_] = {"ms": ms, "tflops": tf, "frac_bf16": tf / peak, "gbs_io": io / (ms * 1e-3) / 1e9,
                          "frac_hbm_io": io / (ms * 1e-3) / 1e9 / hbm}
        assert int(status.item()) == 0, "a tensor-core wait gave up"
        rows.append(rec)
    tot_ms = sum(r[k]["ms"] for r in rows for k in ("forward", "input_grad", "weight_grad"))
    tot_fl = sum(3 * r["gflop"] for r in rows) * 1e9
    line = {"metric": "U-Net layer contractions (forward, input gradient, weight gradient)", "unit": "TFLOP/s",
            "value": tot_fl / (tot_ms * 1e-3) / 1e12, "higher_is_better": True, "dtype": "bf16 (fp32 accumulate)",
            "data": "synthetic", "peak": peak, "peak_kind": kind, "steps": args.steps,
            "config": {"workload": f"batch {n} of {nz}x{ny}x{nx} fields, the 14 3x3x3 layers"}, "layers": rows}
    print(json.dumps(line), flush=True)


def run_glbm(args):
    """Steps of the homogenised porous-medium LBM (Sec. 4) on a dense
    256x256x512 box: walls z = 0/511, lower half a porous layer (eps = 0.6,
    K = 1, nu_eff = nu / eps), body force 1e-6; MLUPS over the fluid cells
    and the roofline of the 152 B/FLUP algorithmic traffic."""
    import torch

    import paper_1507_06565_gb300 as L
    from paper_1507_06565_gb300.build import build

    build()
    L.load_library()
    nx, ny, nz, nu = 256, 256, 512, 0.1
    z = np.arange(nz)
    porous = (z >= 1) & (z < nz // 2)
    eps = np.where(porous, 0.6, 1.0)
    inv_k = np.where(porous, 1.0, 0.0)
    solver = L.GLBM(nx, ny, nz, eps, inv_k, 3 * nu / eps + 0.5, nu, 0.0, (1e-6, 0.0, 0.0))
    stream = torch.cuda.current_stream()
    solver.step(args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for i in range(args.steps):
        solver.step(1)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    durs = np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)])
    ms = float(durs.sum())
    nf = solver.n_fluid
    peak, peak_kind = _peak_hbm()
    first_parity = args.warmup & 1
    parity = {("even" if (first_parity + off) % 2 == 0 else "odd"): float(nf * 152 / (durs[off::2].mean() * 1e-3) / 1e9)
              for off in (0, 1) if durs[off::2].size}
    achieved = float(nf * 152 / (durs.mean() * 1e-3) / 1e9)
    line = {"metric": "fluid MLUPS of the homogenised porous-medium LBM (Sec. 4, Guo & Zhao GLBM)",
            "value": nf * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "higher_is_better": True,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"dense {nx}x{ny}x{nz} box, walls z=0/{nz - 1}, porous lower half eps=0.6 K=1, "
                                   "nu_eff=nu/eps, G=1e-6", "fluid_cells": nf},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "bytes_per_flup": 152, "peak_kind": peak_kind, "by_parity": parity,
                         "kernel": "k_glbm_even/k_glbm_odd"},
            "clocks": clk, "gpu_launches": args.steps}
    print(json.dumps(line), flush=True)


def run_homogenised(args):
    """Sec. 4's comparison on synthetic data: the pore-scale channel (half-size
    W2 shape, porosity 0.6) run to a steady profile; its plane porosity
    eps(z) and permeability K_b (porous window) drive the homogenised LBM
    on the same channel, with K(z) = K_b * CK(eps(z)) / CK(eps_b) (Carman-Kozeny
    scaling, CK(e) = e^3 / (1 - e)^2, eps_b the mean porosity of the window;
    K = infinity where eps = 1), Stokes regime (no Forchheimer term), run to
    steady state with nu_eff = nu (standard GLBM) and nu_eff = nu / eps (the
    paper's proposal).  Reports the deviation of each homogenised profile
    from the plane-averaged pore-scale one."""
    import torch

    import paper_1507_06565_gb300 as L
    from paper_1507_06565_gb300.build import build

    build()
    L.load_library()
    case = W.W2_half(0.6)
    geom = L.lbm_geometry_from_spheres(*case.sphere_args())
    dns = L.Solver(geom, case.tau, case.lam, case.g)
    t0 = time.perf_counter()
    rc, n_dns, res = dns.run_until(args.tol, args.interval, args.max_steps, criterion="profile")
    torch.cuda.synchronize()
    t_dns = time.perf_counter() - t0
    pa = dns.plane_average()
    u_dns, eps = pa[:, 0], pa[:, 2]
    k_b = dns.permeability(*case.perm_window)
    z0, z1 = case.perm_window
    eps_b = float(eps[z0:z1].mean())
    ck = lambda e: e ** 3 / np.maximum(1.0 - e, 1e-12) ** 2
    nz = case.nz
    eps_h = np.where(eps > 0, np.clip(eps, 1e-3, 1.0), 1.0)
    eps_h[0] = eps_h[-1] = 1.0
    inv_k = np.where(eps_h < 1.0 - 1e-9, ck(eps_b) / (k_b * ck(eps_h)), 0.0)
    nu = (case.tau - 0.5) / 3.0
    fluid = slice(1, nz - 1)
    out = {}
    for name, tau in (("nu_eff = nu", np.full(nz, case.tau)), ("nu_eff = nu / eps", 3.0 * nu / eps_h + 0.5)):
        h = L.GLBM(4, 4, nz, eps_h, inv_k, tau, nu, 0.0, case.g)
        prev, steps = None, 0
        while steps < 2_000_000:
            h.step(20_000)
            steps += 20_000
            prof = h.plane_average()
            if prev is not None and np.linalg.norm(prof - prev) <= 1e-8 * np.linalg.norm(prof):
                break
            prev = prof
        dev = np.abs(prof[fluid] - u_dns[fluid])
        ref = np.max(np.abs(u_dns[fluid]))
        out[name] = {"steps": steps, "max_dev_rel": float(dev.max() / ref),
                     "l2_dev_rel": float(np.linalg.norm(prof[fluid] - u_dns[fluid]) / np.linalg.norm(u_dns[fluid])),
                     "porous_max_dev_rel": float(dev[: z1 - 1].max() / ref),
                     "u_every8": prof[::8].tolist()}
    # two-domain interface parameters from the pore-scale profile (Sec. 3.2),
    # at the first all-fluid plane and two planes below it
    from paper_1507_06565_gb300 import interface as I

    zc = np.arange(nz, dtype=float)
    z_top = nz - 1.5
    fits = {}
    zi0 = I.interface_position(zc[1:-1], eps[1:-1])
    for zi in (zi0, zi0 - 2.0):
        try:
            f = I.fit_interface(zc[1:-1], u_dns[1:-1], zi, k_b, nu, nu_eff=nu / eps_b)
            fits[f"z_int={zi:g}"] = {"u_s": f.u_s, "du_free": f.du_free, "du_porous": f.du_porous, "u_m": f.u_m,
                                     "alpha_bj": f.alpha_bj, "alpha_bjs": f.alpha_bjs, "beta_otw": f.beta_otw}
        except ValueError as exc:
            fits[f"z_int={zi:g}"] = {"error": str(exc)}
    # the single-domain Brinkman closed form (two layers, nu_eff = nu / eps_b,
    # K and eps_b from the run) against the pore-scale profile; the sharp
    # interface sits where a layer of porosity eps_b holds the same solid
    # volume as the measured plane porosities
    z_bot = 0.5
    z_sharp = z_bot + float(np.sum(1.0 - eps[1:-1])) / (1.0 - eps_b)
    u_br = I.profile_brinkman_layer(zc, z_bot, z_sharp, z_top, k_b, eps_b, nu, case.g[0])
    dev_br = np.abs(u_br[fluid] - u_dns[fluid])
    brinkman = {"z_int": z_sharp, "max_dev_rel": float(dev_br.max() / np.max(np.abs(u_dns[fluid]))),
                "l2_dev_rel": float(np.linalg.norm(u_br[fluid] - u_dns[fluid]) / np.linalg.norm(u_dns[fluid])),
                "u_every8": u_br[::8].tolist()}
    line = {"metric": "homogenised vs pore-scale plane-averaged velocity (Sec. 4)", "unit": "relative deviation",
            "value": out["nu_eff = nu / eps"]["l2_dev_rel"], "higher_is_better": False, "data": "synthetic",
            "config": {"workload": f"{case.name}: pore-scale to profile residual {args.tol:g}, then GLBM with its "
                                   "plane porosity and permeability"},
            "dns": {"status": L.status_string(rc), "steps": n_dns, "seconds": t_dns, "permeability": k_b,
                    "eps_bulk": eps_b, "u_every8": u_dns[::8].tolist(), "eps_every8": eps[::8].tolist()},
            "homogenised": out, "brinkman_closed_form": brinkman, "interface": fits, "z_top_wall": z_top}
    print(json.dumps(line), flush=True)


def run_grid_study(args):
    """Grid study of the pore-scale profile (Sec. 3.1): the same packing at
    sphere diameters D = 4, 8, 16, 32 lattice units, the force scaled as
    1/scale^3 to keep Re_D = u_max D / nu near 2; the normalised profiles
    are compared on the coarsest heights."""
    import paper_1507_06565_gb300 as L
    from paper_1507_06565_gb300.build import build

    from paper_1507_06565_gb300 import studies as S

    build()
    L.load_library()
    runs, prof = [], {}
    for scale in (1, 2, 4, 8):
        t0 = time.perf_counter()
        h, un, n, umax, re, st = S.run_case(scale, S.G1 / scale ** 3, args.tol, args.interval, args.max_steps,
                                            flags=odd_flags(args))
        prof[scale] = (h, un)
        runs.append({"D": 4 * scale, "steps": n, "status": st, "u_max": umax, "Re_D": re,
                     "layer_porosity": S.layer_porosity(scale), "seconds": time.perf_counter() - t0})
    h1 = prof[1][0]
    diffs = {f"D{4 * a}-D{4 * b}": S.profile_change(prof[a], prof[b], h1) for a, b in ((1, 2), (2, 4), (4, 8))}
    line = {"metric": "pore-scale profile change between resolutions (u/u_max on z/H)", "unit": "relative L2",
            "value": diffs["D16-D32"], "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "16x16x32 channel packing (overlapping D=4 spheres, porosity 0.6, lower half) "
                                   "scaled x1, x2, x4, x8; Re_D ~ 2", "tol": args.tol},
            "runs": runs, "profile_change": diffs,
            "profiles_every_coarse_plane": {f"D{4 * k}": np.interp(h1, *v).tolist() for k, v in prof.items()}}
    print(json.dumps(line), flush=True)


def run_re_sweep(args):
    """Reynolds-number sweep of the pore-scale profile (Sec. 3.1): the D = 16
    packing of the grid study, the force scaled to Re_D ~ 0.2 .. 16 (viscosity
    and geometry fixed); reports where the normalised profile peaks and how
    much flow enters the porous half."""
    import paper_1507_06565_gb300 as L
    from paper_1507_06565_gb300.build import build

    from paper_1507_06565_gb300 import studies as S

    build()
    L.load_library()
    runs = []
    for factor in (0.1, 1.0, 3.0, 8.0):
        h, un, n, umax, re, st = S.run_case(4, factor * S.G1 / 64, args.tol, args.interval, args.max_steps,
                                            flags=odd_flags(args))
        runs.append({"force_factor": factor, "Re_D": re, "u_max": umax, "steps": n, "status": st,
                     "z_max_over_H": float(h[int(np.argmax(un))]),
                     "porous_half_mean_u_over_max": float(un[h < 0.5].mean()),
                     "profile_every4": un[::4].tolist()})
    line = {"metric": "pore-scale profile vs Re_D (peak height and porous-layer flow)", "unit": "z/H",
            "value": runs[-1]["z_max_over_H"], "higher_is_better": None, "data": "synthetic",
            "config": {"workload": "64x64x122 channel (D=16 packing of the grid study)", "tol": args.tol},
            "runs": runs}
    print(json.dumps(line), flush=True)


def run_surrogate(args):
    """Time to steady state with and without the learned warm start: solver-
    generated training data, training with the library's U-Net kernels, and
    cold versus warm runs of held-out packings to the same tolerance."""
    import torch

    import paper_1507_06565_gb300 as L
    from paper_1507_06565_gb300 import surrogate as S
    from paper_1507_06565_gb300.build import build

    build()
    L.load_library()
    shape = tuple(int(v) for v in args.shape.split("x"))
    t0 = time.perf_counter()
    data = S.generate(range(500000, 500000 + args.train_samples), shape, tol=args.label_tol)
    tr = S.train(data, epochs=args.epochs, lr=2e-3, batch=args.batch)
    params = tr.net.params().cpu().numpy()
    rows = S.warm_vs_cold(params, range(600000, 600000 + args.heldout), shape, tol=args.tol)
    cold = sum(r["cold"]["seconds"] for r in rows)
    warm = sum(r["warm"]["seconds"] for r in rows)
    line = {"metric": f"time to steady state (plane-profile residual < {args.tol:g}), surrogate warm vs cold",
            "value": warm, "unit": "s", "higher_is_better": False, "cold_s": cold, "speedup": cold / warm,
            "steps_cold": [r["cold"]["steps"] for r in rows], "steps_warm": [r["warm"]["steps"] for r in rows],
            "k_rel_diff_max": max(r["k_rel_diff"] for r in rows),
            "k_err_warm_max": max(r["k_err_warm"] for r in rows),
            "k_err_cold_max": max(r["k_err_cold"] for r in rows),
            "k_reference": "cold run continued, untimed, for 4 decay times of the slowest viscous mode",
            "dtype": "f32 LBM, bf16/fp32 network", "data": "synthetic",
            "config": {"workload": f"{shape[0]}x{shape[1]}x{shape[2]} channels, lower half overlapping r=4 spheres at "
                                   "porosity U[0.6,0.8]; train seeds 500000+, held-out seeds 600000+",
                       "train_samples": args.train_samples, "heldout": args.heldout, "epochs": args.epochs,
                       "batch": args.batch, "label_tol": args.label_tol, "wall_rule": "safeguards"},
            "training": {"data_steps": data.steps, "data_s": data.seconds, "train_s": tr.seconds,
                         "samples": tr.samples, "loss_first": tr.losses[0], "loss_last": float(np.mean(tr.losses[-8:]))},
            "rows": rows, "total_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def _stability_sets():
    """Every packing the benchmarks and studies run, grouped as solvers: name,
    geometry builder, cases (one solver per entry; a list is one batch)."""
    sets = [("W1 32x32x64 RSA r=4", [W.W1])]
    sets += [(c.name, [c]) for c in (W.W2(phi) for phi in W.W2_POROSITIES)]
    sets += [(W.W2_half(phi).name, [W.W2_half(phi)]) for phi in W.W2_POROSITIES]
    sets.append(("W0 151^3 one sphere D=90", [W.W0]))
    sets.append(("W4 64 REV cubes", [W.W4_cube(i) for i in range(64)]))
    from paper_1507_06565_gb300 import surrogate as S

    sets.append(("W5 warm-start channels 64x64x128 r=4 (seeds 500000-500015)",
                 [S.channel_case(sd) for sd in range(500000, 500016)]))
    sets.append(("W5 held-out channels 64x64x128 r=4 (seeds 600000-600009)",
                 [S.channel_case(sd) for sd in range(600000, 600010)]))
    sets.append(("W3 512x512x1024 r=8 phi=0.6", [W.W3_LARGE]))
    from paper_1507_06565_gb300 import studies as St

    for scale in (1, 2, 4, 8):
        sets.append((f"grid-study packing D={4 * scale}", [St.BASE], scale))
    return sets


def run_cli_stability(args):
    """Stability of the wall rule on every packing: g = 0, a white-noise
    perturbation of the rest state (velocity amplitude 1e-6 per cell), and the
    largest |u| of each box after 2000 steps, half of --stability-steps and
    all of them.  The white noise also excites the lattice's undamped
    period-two modes, which keep their amplitude (ratio ~1.00); Eq. (CLI) in a
    corner where it is unstable makes the perturbation grow without bound.  A
    box counts as growing when its largest |u| rises by more than 1% over the
    second half.  Reports, per box, both ratios, the cell of the largest |u|
    at the end, and the fraction of wall links that take simple bounce-back."""
    import torch

    import paper_1507_06565_gb300 as L
    from paper_1507_06565_gb300.build import build

    build()
    L.load_library()
    rows = []
    first = 2000
    from paper_1507_06565_gb300 import studies as St

    for name, cases, *scale in _stability_sets():
        if cases[0] is W.W0:
            geoms = [L.lbm_geometry_from_list(*W.W0_BOX, True, W.W0_SPHERES)]
        elif scale:
            (nx, ny, nz), sc = St.scaled_spheres(scale[0])
            geoms = [L.lbm_geometry_from_list(nx, ny, nz, False, sc)]
            cases = [W.Channel(name, nx, ny, nz, 0.0, 0.0, 0.0, 0.0, 0.0, True, 0)]
        else:
            geoms = [L.lbm_geometry_from_spheres(*c.sphere_args()) for c in cases]
        cells = sum(g.info()["n_cells"] for g in geoms)
        gen = torch.Generator(device="cuda").manual_seed(1)
        u0 = 1e-6 * torch.randn(3 * cells, device="cuda", generator=gen)
        kw = dict(tau=cases[0].tau, lam=cases[0].lam, g=(0.0, 0.0, 0.0), storage="f32",
                  flags=odd_flags(args, cases))
        if len(geoms) > 1:
            s = L.BatchSolver(geoms, u0=u0, **kw)
            offs = [s.part_info(b)["cell_offset"] for b in range(len(geoms))]
        else:
            s = L.Solver(geoms[0], u0=u0, **kw)
            offs = [0]
        offs.append(cells)
        del u0
        links = fallback_fraction(s)

        def part_max():
            _, u = s.moments()
            a = u.abs().amax(dim=0).reshape(-1)
            return [(float(a[offs[b]:offs[b + 1]].max()), int(a[offs[b]:offs[b + 1]].argmax()))
                    for b in range(len(geoms))]

        t0 = time.perf_counter()
        half = args.stability_steps // 2
        s.step(first)
        m0 = part_max()
        s.step(half - first)
        m1 = part_max()
        s.step(args.stability_steps - half)
        m2 = part_max()
        torch.cuda.synchronize()
        parts = []
        for b, c in enumerate(cases):
            def ratio(a, e):
                return e / a if a > 0 and np.isfinite(e) else float("inf")
            cell = m2[b][1]
            nx, ny = geoms[b].shape[2], geoms[b].shape[1]
            parts.append({"box": c.name, "ratio": ratio(m0[b][0], m2[b][0]),
                          "ratio_late": ratio(m1[b][0], m2[b][0]), "max_u_end": m2[b][0],
                          "argmax_xyz": [cell % nx, (cell // nx) % ny, cell // (nx * ny)]})
        worst = max(p["ratio_late"] for p in parts)
        rows.append({"set": name, "worst_ratio_late": worst, "worst_ratio": max(p["ratio"] for p in parts),
                     "stable": bool(worst <= 1.01),
                     "growing_boxes": [p for p in parts if not p["ratio_late"] <= 1.01], "links": links,
                     "seconds": time.perf_counter() - t0})
        del s
        torch.cuda.empty_cache()
    line = {"metric": "growth of a rest-state perturbation under the wall rule (max|u| ratio over the second half)",
            "value": max(r["worst_ratio_late"] for r in rows), "unit": "ratio", "higher_is_better": False,
            "data": "synthetic", "config": {"wall_rule": args.wall_rule, "steps": args.stability_steps,
                                            "first": first, "perturbation": "white noise, |u| ~ 1e-6, g = 0"},
            "sets": rows}
    print(json.dumps(line), flush=True)


def run_reference(args, world, rank):
    if rank != 0:
        return
    nf, dt, cores = _oracle_sample(args.steps, args.warmup)
    value = nf * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": SAMPLE_STEP.name, "fluid_cells": nf},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{SAMPLE_STEP.name}: one oracle time step per bench step"},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch

    import paper_1507_06565_gb300 as L
    from paper_1507_06565_gb300.build import build

    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    L.load_library()
    stream = torch.cuda.current_stream()

    phis = W.W2_POROSITIES if args.phi is None else [args.phi]
    if args.workload == "channel":
        cases = [W.W2(phi) for phi in phis]
    elif args.workload == "channel-half":   # the same channel at half the size, for profiler captures
        cases = [W.W2_half(phi) for phi in phis]
    elif args.workload == "large":   # one 512x512x1024 channel (W2's structure, porosity 0.6)
        cases = [W.W3_LARGE]
    elif args.workload == "w0":   # the paper's single-sphere block: 151^3 periodic, one sphere D = 90
        cases = [W.W0]
    else:   # rev: the periodic REV cubes as one batch
        cases = [W.W4_cube(i) for i in range(args.cubes)]
    if args.workload == "w0":
        geoms = [L.lbm_geometry_from_list(*W.W0_BOX, True, W.W0_SPHERES)]
    else:
        geoms = [L.lbm_geometry_from_spheres(*c.sphere_args()) for c in cases]
    c0 = cases[0]
    if args.workload == "rev":
        solvers = [L.BatchSolver(geoms, c0.tau, c0.lam, c0.g, args.storage, flags=odd_flags(args, cases))]
    else:
        solvers = [L.Solver(g, c.tau, c.lam, c.g, args.storage, flags=odd_flags(args, [c]))
                   for g, c in zip(geoms, cases)]
    nfs = [s.info()["n_fluid"] for s in solvers]
    nf_total = sum(nfs)
    lib = L.load_library()
    # set-up: let the launch-schedule tuner finish its timed trial launches
    # before the warm-up, so the timed steps use the final schedule
    for s in solvers:
        while not s.schedule()["tuned"] and s.steps < 256:
            s.step(2)
    schedules = [s.schedule() for s in solvers]
    links = [fallback_fraction(s) for s in solvers]

    def one_step(events=None):
        for s in solvers:
            if events is not None:
                events[0].append(torch.cuda.Event(enable_timing=True))
                events[1].append(torch.cuda.Event(enable_timing=True))
                events[0][-1].record(stream)
            rc = lib.lbm_step(s.handle, 1)
            if rc:
                raise L.LBMError(rc, "lbm_step")
            if events is not None:
                events[1][-1].record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = ([], [])
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        one_step(ev)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1))
    durs = np.array([a.elapsed_time(b) for a, b in zip(*ev)]).reshape(args.steps, len(solvers))
    first_parity = args.warmup & 1   # parity of the first timed step
    # per-launch algorithmic bytes: 19 loads + 19 stores of the stored type per fluid cell
    bytes_per_flup = 19 * 2 * (4 if args.storage == "f32" else 2)
    bytes_per_launch = np.array(nfs, dtype=np.float64) * bytes_per_flup
    # algorithmic bytes of all timed launches over their summed event time
    # (a launch-weighted rate; the gaps between launches are in ms_per_step)
    achieved = float(bytes_per_launch.sum() * args.steps / (durs.sum() * 1e-3) / 1e9)
    peak, peak_kind = _peak_hbm()
    parity = {}
    for off in (0, 1):
        sel = durs[off::2]
        if sel.size:
            name = "even" if (first_parity + off) % 2 == 0 else "odd"
            gbs = float(bytes_per_launch.sum() * sel.shape[0] / (sel.sum() * 1e-3) / 1e9)
            parity[name] = {"achieved": gbs, "frac": gbs / peak, "share": float(sel.sum() / durs.sum())}
    value = whole_job_rate(nf_total * args.steps, ms, world)
    # DRAM bytes per fluid cell and launch of the step kernels as they stand,
    # from ncu captures (dram__bytes_read.sum + dram__bytes_write.sum) of one
    # solver of this workload: only for the configuration they were taken on
    traffic = None
    if args.storage == "f32" and args.odd == "auto" and args.even == "auto":
        if args.workload == "channel":
            traffic = float(np.mean(nfs)) * 0.5 * (MEASURED_DRAM_B_PER_FLUP["even"] + MEASURED_DRAM_B_PER_FLUP["odd"])
        elif args.workload == "rev" and args.cubes == 64:
            traffic = float(np.mean(nfs)) * 0.5 * (MEASURED_DRAM_B_PER_FLUP_REV["even"]
                                                   + MEASURED_DRAM_B_PER_FLUP_REV["odd"])

    # end to end through the public API with host buffers: lbm_init from the
    # host geometry (mask and sphere bins copied host->device, lists and
    # links built on the device), the steps through lbm_step (the schedule
    # tuner's trial launches included), plane averages copied back to the
    # host; at least 200 steps so that the set-up is amortised as in a run
    e2e_steps = max(200, args.steps)
    torch.cuda.synchronize()
    te = time.perf_counter()
    h2d = 0
    d2h = 0
    setup_s = 0.0
    groups = [geoms] if args.workload == "rev" else [[g] for g in geoms]
    grp_case = {id(g): c for g, c in zip(geoms, cases)}
    for grp in groups:
        t_in = time.perf_counter()
        if args.workload == "rev":
            s2 = L.BatchSolver(grp, c0.tau, c0.lam, c0.g, args.storage, flags=odd_flags(args, cases))
        else:
            s2 = L.Solver(grp[0], c0.tau, c0.lam, c0.g, args.storage, flags=odd_flags(args, [grp_case[id(grp[0])]]))
        setup_s += time.perf_counter() - t_in
        s2.step(e2e_steps)
        pa = s2.plane_average()
        h2d += sum(g.mask().nbytes for g in grp)
        d2h += pa.nbytes
        del s2
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - te
    e2e_value = nf_total * e2e_steps / e2e_s / 1e6

    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": {"workload": workload_name(args), "fluid_cells": nfs, "storage": args.storage,
                   "odd_neighbours": args.odd, "even_step": args.even,
                   "wall_rule": ([wall_rule(args, cases)] if args.workload == "rev"
                                 else [wall_rule(args, [c]) for c in cases]),
                   "wall_links": links, "schedule": schedules,
                   "l2": "inputs larger than L2 ({:.1f}-{:.1f} GB of populations and indices per solver)".format(
                       *(n * (19 * (4 if args.storage == "f32" else 2) + 76) / 1e9 for n in (min(nfs), max(nfs)))),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_step_even/k_step_odd (fused AA stream-collide + CLI)",
                     "bytes_per_flup": bytes_per_flup, "peak_kind": peak_kind, "by_kernel": parity,
                     "wall_frac": value * 1e6 / world * bytes_per_flup / 1e9 / peak},
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d / e2e_steps,
                "d2h_bytes_per_step": d2h / e2e_steps, "steps": e2e_steps, "seconds": e2e_s,
                "setup_seconds": setup_s,
                "what": f"lbm_init from host geometry + {e2e_steps} steps + plane averages to host, every solver"},
        "clocks": clk,
        "gpu_launches": args.steps * len(solvers),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--odd", choices=["auto", "table", "rows", "staged", "derived"], default="auto",
                    help="neighbour indices of the odd step (library default, int32 table, row bitmasks, row words "
                         "staged per tile, x-neighbours derived from the table's other entries)")
    ap.add_argument("--even", choices=["auto", "staged"], default="auto",
                    help="even-step kernel: autotuned, or always the TMA-staged one")
    ap.add_argument("--bounce-back", action="store_true",
                    help="simple bounce-back on every wall link instead of CLI (Eq. (noslip), q = 1/2 forced)")
    ap.add_argument("--wall-rule", choices=["auto", "paper", "safeguards"], default="auto",
                    help="Eq. (CLI) wherever x_f2 exists (paper), or with the corner safeguards (q < 0.1 and "
                         "two-cell gaps bounce back); auto: paper on the workloads where it was found stable")
    ap.add_argument("--stability-steps", type=int, default=60000,
                    help="cli-stability: steps per packing")
    ap.add_argument("--storage", choices=["f32", "f16", "bf16"], default="f32",
                    help="population storage (FP32 collision in every case)")
    ap.add_argument("--workload", choices=["channel", "channel-half", "large", "w0", "rev", "surrogate", "unet", "glbm",
                                           "homogenised", "grid-study", "re-sweep", "cli-stability", "unet-layers"],
                    default="channel",
                    help="channel: the 256x256x512 sweep (the benchmark); channel-half: 128x128x256, for "
                         "profiling; large: one 512x512x1024 channel; rev: the batched REV cubes; surrogate: "
                         "warm versus cold start; unet: U-Net training steps; glbm: the homogenised model; "
                         "homogenised: the homogenised model against the pore-scale profile; grid-study, "
                         "re-sweep: the resolution and Reynolds-number studies of the pore-scale profile; "
                         "cli-stability: growth of a perturbation of the rest state on every packing")
    ap.add_argument("--cubes", type=int, default=64, help="number of REV cubes (rev workload)")
    ap.add_argument("--phi", type=float, default=None,
                    help="channel workloads: one porosity of the sweep instead of all four")
    ap.add_argument("--precision-check", action="store_true",
                    help="--converge: FP16/BF16 runs started from the converged FP32 field, errors against it")
    ap.add_argument("--rp-max-steps", type=int, default=400_000,
                    help="--precision-check: step limit of the FP16/BF16 runs (their profile residual floor can "
                         "lie above --tol)")
    ap.add_argument("--plane-references", choices=["auto", "on", "off"], default="auto",
                    help="plane reference equilibria: the library default (on for FP16/BF16 storage), or forced")
    ap.add_argument("--oracle-steps", type=int, default=0,
                    help="--precision-check: FP64 oracle steps from the converged FP32 state")
    ap.add_argument("--converge", action="store_true",
                    help="instead of timing steps, run to steady state and report the time and permeabilities")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--train-samples", type=int, default=96)
    ap.add_argument("--heldout", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--shape", default="64x64x128", help="surrogate: channel nx x ny x nz")
    ap.add_argument("--batch", type=int, default=4, help="surrogate: training batch")
    ap.add_argument("--label-tol", type=float, default=1e-6, help="surrogate: profile residual of the labels")
    ap.add_argument("--interval", type=int, default=500)
    ap.add_argument("--max-steps", type=int, default=2_000_000)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "surrogate":
        run_surrogate(args)
    elif args.workload == "unet":
        run_unet(args)
    elif args.workload == "glbm":
        run_glbm(args)
    elif args.workload == "unet-layers":
        run_unet_layers(args)
    elif args.workload == "homogenised":
        run_homogenised(args)
    elif args.workload == "grid-study":
        run_grid_study(args)
    elif args.workload == "re-sweep":
        run_re_sweep(args)
    elif args.workload == "cli-stability":
        run_cli_stability(args)
    elif args.converge and args.precision_check:
        run_precision_check(args)
    elif args.converge:
        run_converge(args)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
