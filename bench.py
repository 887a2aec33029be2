"""Benchmark of the rendering hot path: phasor terms/s for forward + adjoint.

One step = one pass of the whole hot path over one batch of synthetic input
(stratified sampling, MLP fields with gradient tangents, lensless blending,
signal tracing, matched filter + L2 loss, and the adjoints of all of them down
to the MLP parameter gradient). Headline workload (default, the largest
single-GPU configuration): 128x128 array at 2 mm, 256 frequencies over
77-81 GHz, 256^3 stratified samples of a 10 cm cube, SDF/reflectiveness MLP
4x128 (softplus, PE 6 octaves) in BF16 on the tcgen05 tensor cores with FP32
accumulation, FP32 phasor sums, 64^3 heatmap against a synthetic target
(sphere + point reflector). The same line carries the 64x64-array, 128-bin,
128^3-sample FP32 step ("c2"), the per-bin recurrence measured beside the
default Chebyshev form, the signal tracing bank, the training-step comparison
of proposal against uniform sampling and the paper's own training
configuration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
                  [--workload c3|c2|c3-small|c2-small]

N > 1 runs under torchrun, one independent replica per GPU (no collective on
the data path; weak scaling); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "point·antenna·freq phasor terms/s fwd+adj; train-step ms at ≤2e-3 rel err"
WORKLOADS = {
    "c3": ("128x128 array @2mm, 256 freqs 77-81 GHz, 256^3 stratified samples, MLP 4x128 bf16 on tcgen05 "
           "(fp32 accumulate), 64^3 heatmap, forward + adjoint of every step"),
    "c2": ("64x64 array @2mm, 128 freqs 77-81 GHz, 128^3 stratified samples, MLP 4x128 fp32, "
           "64^3 heatmap, forward + adjoint of every step"),
    "c3-small": "c3 array, band and bf16 MLP on 64x64x16 stratified samples, 32^3 heatmap (profiling size)",
    "c2-small": "c2 array, band and fp32 MLP on 64x64x16 stratified samples, 32^3 heatmap (profiling size)",
}
DTYPES = {"fp32": "f32", "bf16": "f32 phasor sums + bf16 MLP (fp32 accumulate)"}
# Algorithmic FP32 flops (FMA = 2) of the phasor sums.
# Per-bin recurrence, per (point, antenna, bin) term: real amplitude times the
# unit phasor into a complex sum (2 FMA) and the angle-addition step (2 MUL +
# 2 FMA) = 10 flops (render, filter adjoint); complex coefficients summed by
# Horner's rule over a 32-bin block = 4 FMA = 8 flops (filter, render adjoint).
# Chebyshev form, per (point, antenna) pair and order k: the three-term
# recurrence of T_k (1 FMA) and the complex moment or series sum (2 FMA) =
# 6 flops per order.
# Besides the orders, the Chebyshev form does fixed arithmetic per pair, FP32
# flops (FMA = 2) counted from its steps: the range as a double-single from
# split coordinates in carrier cycles (differences 9, |dh|^2 5, cross term 11,
# sum, square root product and Newton correction 6: 32), the carrier phase's
# fractional cycle and angle (3), x and 2x (4), and the call's own terms:
# render, the amplitude w (T'/r)^2 D and its product with the phasor (15);
# render adjoint, Re(conj(g) x the series sum) and the chain rule of
# A = w T'^2 gamma D into its five sums (30); filter, the phasor-rotated series
# sum into M (8); filter adjoint, the complex amplitude times the phasor (6).
FLOPS_PER_TERM = {"render": 10, "filter_backward": 10, "filter": 8, "render_backward": 8}
CHEB_FLOPS_PER_ORDER = 6
CHEB_FLOPS_PER_PAIR = {"render": 54, "render_backward": 69, "filter": 47, "filter_backward": 45}
PHASOR_CALLS = ("render", "render_backward", "filter", "filter_backward")
MLP_CALLS = ("fields", "fields_backward")
TIMED_CALLS = PHASOR_CALLS + MLP_CALLS
# DRAM bytes (read + write) per launch of a call's main kernel from one ncu
# capture: (bytes, what the count scales with, units in the captured case,
# the workload that case stands for). A capture of a smaller case is scaled by
# the points or voxels processed (the records and partials grow in
# proportion). Only kernels unchanged since their capture are listed.
NCU_DRAM = {}
# Captures whose traffic does not grow in proportion to the points (stated, not
# scaled): the render adjoint's DRAM reads are mostly its point groups' antenna
# rows, whose size depends on the group count and the antennas, not the points.
NCU_DRAM_UNSCALED = {
    ("c3", "render_backward"): "ncu capture of cheb_points_kernel<1,3> on the same array, band and part "
                               "rules at 2^20 points (bench.py --phasor-case 128,128,64): 9.32e9 B per launch, "
                               "9.13e9 B of it the 512 groups' antenna rows (the same 512 groups at 2^24 points); "
                               "not scaled",
}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def cpu_baseline_sample(geo, xyz, grad, w, t_eff, c_ant, max_pts=16384, n_ant=1024, n_vox=8192, filt_ant=1024):
    """Times the FP64 oracle's four phasor sums on a bounded sample of the
    workload (first max_pts points x first n_ant antennas x all bins for the
    tracing pair; first n_vox voxels x first filt_ant antennas for the filter
    pair). Returns (terms/s, seconds, terms, description)."""
    import numpy as np
    from oracle import geraf_oracle as O
    import geraf_inputs as gi
    b = gi.Band(geo.band.f0, geo.band.df, geo.band.n_f)
    h = lambda t: t.detach().cpu().numpy()
    X, Gr, W, Te = h(xyz)[:, :max_pts], h(grad)[:, :max_pts], h(w)[:max_pts], h(t_eff)[:max_pts]
    A, C = h(geo.ant)[:, :n_ant], h(c_ant)[:n_ant]
    V = h(geo.vox)[:, :n_vox]
    Af = h(geo.ant)[:, :filt_ant]
    rng = np.random.default_rng(0)
    g = gi.complex_normal(rng, (n_ant, b.n_f))
    t0 = time.perf_counter()
    s = O.render(X, Gr, W, Te, A, C, b)
    O.render_backward(X, Gr, W, Te, A, C, b, g)
    sf = gi.complex_normal(rng, (filt_ant, b.n_f))
    M, P = O.filter_forward(sf, Af, V, b)
    O.filter_backward(M, np.ones(n_vox), Af, V, b)
    dt = time.perf_counter() - t0
    terms = 2 * X.shape[1] * n_ant * b.n_f + 2 * n_vox * filt_ant * b.n_f
    desc = (f"oracle render+render_backward on {X.shape[1]} points x {n_ant} antennas x {b.n_f} bins, "
            f"filter+filter_backward on {n_vox} voxels x {filt_ant} antennas x {b.n_f} bins (FP64 C, OpenMP)")
    del s
    return terms / dt, dt, terms, desc


def oracle_threads():
    try:
        return int(os.environ.get("OMP_NUM_THREADS", "")) or os.cpu_count()
    except ValueError:
        return os.cpu_count()


def run_reference(args, rank):
    """The oracle as the reference arm: K bounded samples of the workload on
    the host cores, timed like steps."""
    if rank != 0:
        return
    import torch  # noqa: F401  (CUDA not needed)
    import numpy as np
    import geraf_inputs as gi
    from oracle import geraf_oracle as O
    wl = gi.workload(args.workload)
    b = gi.band(77e9, 81e9, wl.n_f)
    xyz, apr = O.sample(wl.grid, gi.SAMPLE_STRATIFIED, seed=0, step=0)
    n_pts, n_ant, n_vox, filt_ant = 16384, 128, 2048, 256
    X = xyz[:, :n_pts]
    rng = np.random.default_rng(0)
    Gr = rng.standard_normal((3, n_pts))
    W, Te = rng.uniform(0, 1e-3, n_pts), np.full(n_pts, 2.0)
    A = gi.antenna_array(wl.array_n, wl.array_n, wl.array_pitch)[:, :n_ant]
    Af = gi.antenna_array(wl.array_n, wl.array_n, wl.array_pitch)[:, :filt_ant]
    V, _ = O.sample(wl.heat, gi.SAMPLE_UNIFORM)
    V = V[:, :n_vox]
    g = gi.complex_normal(rng, (n_ant, b.n_f))
    sf = gi.complex_normal(rng, (filt_ant, b.n_f))

    def step():
        O.render(X, Gr, W, Te, A, np.ones(n_ant), b)
        O.render_backward(X, Gr, W, Te, A, np.ones(n_ant), b, g)
        M, _ = O.filter_forward(sf, Af, V, b)
        O.filter_backward(M, np.ones(n_vox), Af, V, b)

    terms = 2 * n_pts * n_ant * b.n_f + 2 * n_vox * filt_ant * b.n_f
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = terms * args.steps / dt
    cores = oracle_threads()
    desc = (f"per step: oracle render+render_backward {n_pts} points x {n_ant} antennas x {b.n_f} bins, "
            f"filter+filter_backward {n_vox} voxels x {filt_ant} antennas (FP64 C + OpenMP, host cores)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "sample": "bounded oracle sample"},
            "cpu_baseline": {"value": value, "unit": "terms/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, world: int, device) -> float:
    """Largest value of x over all ranks (the job's time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seeds(rank: int) -> dict:
    """Each rank runs an independent replica: its own sampling seed and MLP init."""
    return {"sample": 7 + 1000 * rank, "mlp": 1234 + rank}


def job_rate(units_per_step_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: units processed by all ranks over the slowest rank's time."""
    return units_per_step_per_rank * steps * world / (max_ms * 1e-3)


def train_step_compare(dev, warmup=1, steps=2, c_warmup=2, c_steps=3, r_max=2, prop_steps=800,
                       m_table=(24, 26, 27, 28, 30), dilates=(1, 2), gshape=(64, 64, 128)):
    """Training step on the random-scene workload (1-8 ellipsoids and boxes
    behind a 0.5 occluder, 10 dB noise; 64x64 array, 128 bins, 64^3 heatmap):
    2^24 stratified samples (256^2 columns x 256 depths) against the same
    grid's own samples in the m proposal cells (of 128 per column, 2 depths
    each) ranked first plus r_max run-closing samples per column (2 m + r_max
    samples per column). First the proposal is trained on the blended weights T alpha of
    dense renders of the analytic scene (the converged geometry); then, at
    fixed parameters, the heatmap relative L2 of the cell-subset pass against
    the dense pass (identical samples in the kept cells) on that scene, for the
    trained proposal and for the exact dense weight histogram, against m and
    the ranking's dilation (cells ranked by the largest q within `dilate`
    cells). Then the training steps are timed on the MLP field at each m (each
    with its Adam update; the cell steps also update the proposal from their
    own pass), and the MLP-field heatmap error and gradient cosine are
    reported. The operating point is the fewest samples whose trained-proposal
    error on the converged geometry is at most 2e-3 (fallback to uniform
    sampling when none is)."""
    import torch
    import geraf_inputs as gi
    import paper_2605_29097_gb300 as G
    from paper_2605_29097_gb300 import pipeline as PL
    wl = gi.workload("c4")
    geo = PL.make_geometry(wl, dev)
    scene = gi.c4_scene(4)
    target = PL.scene_target(geo, scene, noise_seed=4, device=dev)
    s_fine = geo.n_z // gshape[2]
    prop, pm = PL.init_proposal(gshape=gshape, depth=16, seed=5, device=dev)
    ptrain = PL.ProposalTrainer(prop, pm, lr=1e-2)
    afield = PL.scene_field(scene, dev)
    ploss = None
    for k in range(prop_steps):
        dp, df, ploss = PL.proposal_signal_dense(geo, afield, prop, seed=41, step=k)
        ptrain.step(dp, df)

    def rel(a, b):
        return float(torch.linalg.norm(a.double() - b.double()) / torch.linalg.norm(b.double()))

    # fixed parameters, identical samples in the kept cells (seed 31, step 0)
    _, q_prop, _ = G.geraf_proposal_density(prop, keep_saved=False)
    q_prop = q_prop.clone()
    q_best = PL.dense_weight_histogram(geo, afield, gshape, seed=31, step=0)
    Pu = PL.forward_backward(geo, afield, target, seed=31, step=0).P
    table = []
    for mm in m_table:
        for dil in dilates:
            row = {"m": mm, "dilate": dil, "samples_per_column": mm * s_fine + r_max,
                   "kept_fraction": (mm * s_fine + r_max) / geo.n_z}
            for name, q in (("trained_proposal", q_prop), ("exact_histogram", q_best)):
                Pc = PL.cells_forward_backward(geo, afield, prop, target, mm, r_max, seed=31, step=0, q=q,
                                               train_proposal=False, dilate=dil).P
                row[name] = rel(Pc, Pu)
            table.append(row)
        torch.cuda.empty_cache()
    del Pu, q_best

    # training steps on the MLP field
    spec = gi.MLPSpec(center=(0.0, 0.0, 0.15), half=0.06)
    p0 = gi.mlp_init(spec, seed=11, sdf_bias=0.02)
    p = torch.as_tensor(p0, device=dev)
    field = G.MLPField(p, center=spec.center, half=spec.half)
    master = p.clone().requires_grad_(True)
    opt = torch.optim.Adam([master], lr=1e-3)

    def apply(d):
        opt.zero_grad(set_to_none=False)
        master.grad = d.clone()
        opt.step()
        with torch.no_grad():
            p.copy_(master)

    def timed(fn, w, n, k0):
        for i in range(w):
            fn(k0 + i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(n):
            fn(k0 + w + i)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    ms_u = timed(lambda k: apply(PL.forward_backward(geo, field, target, seed=21, step=k).d_params), warmup, steps, 0)
    torch.cuda.empty_cache()
    ok = sorted((r for r in table if r["trained_proposal"] <= 2e-3), key=lambda r: (r["m"], r["trained_proposal"]))
    op = ok[0] if ok else min(table, key=lambda r: r["trained_proposal"])
    timed_m = {}
    for mm in m_table:
        def cells_step(k, mm=mm):
            r = PL.cells_forward_backward(geo, field, prop, target, mm, r_max, seed=23, step=k, dilate=op["dilate"])
            apply(r.d_params)
            dp, df, _ = r.proposal
            ptrain.step(dp, df)
        ms_c = timed(cells_step, c_warmup, c_steps, 100)
        timed_m[mm] = {"cells_step_ms": ms_c, "speedup": ms_u / ms_c,
                       "samples": geo.n_ray * (mm * s_fine + r_max)}
        torch.cuda.empty_cache()
    m_op = op["m"]
    with torch.no_grad():
        p.copy_(torch.as_tensor(p0, device=dev))
    ru = PL.forward_backward(geo, field, target, seed=31, step=0)
    rc = PL.cells_forward_backward(geo, field, prop, target, m_op, r_max, seed=31, step=0, q=q_prop,
                                   train_proposal=False, dilate=op["dilate"])
    gu, gc = ru.d_params.double(), rc.d_params.double()
    cos = float((gu @ gc) / (torch.linalg.norm(gu) * torch.linalg.norm(gc)))
    torch.cuda.synchronize()
    return {"workload": "random ellipsoids/boxes behind a 0.5 occluder, 10 dB noise; 64x64 array, 128 freqs, "
                        "MLP 4x128 fp32, 64^3 heatmap",
            "uniform_samples": wl.grid.n_pts, "cells_of_column": gshape[2], "r_max": r_max,
            "proposal_training_steps_on_scene": prop_steps, "proposal_kl_after_training": float(ploss),
            "uniform_step_ms": ms_u, "cells_steps": timed_m,
            "heatmap_rel_l2_table_converged_geometry": table,
            "operating_point": {"m": m_op, "dilate": op["dilate"], "samples_per_column": op["samples_per_column"],
                                "heatmap_rel_l2_converged_geometry": op["trained_proposal"],
                                "speedup": timed_m.get(m_op, {}).get("speedup")},
            "heatmap_rel_l2_mlp_field_at_init": rel(rc.P, ru.P), "grad_cosine_mlp_field_at_init": cos,
            "tolerance": 2e-3, "fallback_to_uniform": not ok,
            "steps": {"uniform": steps, "cells": c_steps}}


def paper_config_step(dev, warmup=3, steps=5, precision="fp32"):
    """The paper's own training configuration (App. C "Training Setup";
    section 5.3; section 9): N_ray = 1024 primary rays x N_z = 32 depths,
    SDF network 8 x 256 and a separate reflectivity network 4 x 256 on a
    10-octave encoding (FP32), the FMCW chirp read as 64 stepped frequencies,
    a signal tracing bank of 3200-antenna patches (a 160 x 160 array at 2 mm in
    8 patches of 80 x 40), 32^3 heatmap voxels (as many as the paper's
    matched-filter points). One step traces one patch, filters the whole bank
    and runs the adjoints of the patch and of both networks."""
    import dataclasses
    import torch
    import geraf_inputs as gi
    import paper_2605_29097_gb300 as G
    from paper_2605_29097_gb300 import pipeline as PL
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.12, (32, 32, 32))
    wl = gi.Workload("paper", 160, 0.002, 64, g, g, gi.SAMPLE_STRATIFIED, "mlp", "fp32", sharpness=2.0 / g.pitch[2])
    geo = PL.make_geometry(wl, dev)
    fb = gi.fmcw_band()
    geo = dataclasses.replace(geo, band=G.Band(fb.f0, fb.df, fb.n_f))
    nets = gi.paper_nets(center=(0.0, 0.0, 0.15), half=0.06)
    params = torch.as_tensor(gi.nets_init(nets, seed=3, sdf_bias=0.02), device=dev)
    field = G.MLPField(params, n_levels=10, width=256, n_hidden=8, beta=nets.sdf.beta, center=nets.sdf.center,
                       half=nets.sdf.half, refl_hidden=4, refl_width=256,
                       precision=G.PREC_BF16 if precision == "bf16" else G.PREC_FP32)
    target = PL.scene_target(geo, gi.c4_scene(4), noise_seed=4, device=dev)
    bank = PL.SignalBank(geo, (160, 160), (80, 40))
    bank.fill(field, 0, 0)
    names = ["render", "render_backward", "filter", "filter_backward", "fields_backward"]
    for k in range(warmup):
        PL.forward_backward_bank(bank, field, target, 0, k)
    torch.cuda.synchronize()
    ev = [{nm: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for nm in names}
          for _ in range(steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(steps):
        PL.forward_backward_bank(bank, field, target, 0, warmup + k, timers=ev[k])
    e1.record()
    torch.cuda.synchronize()
    G.geraf_poll_device_error()
    ms = e0.elapsed_time(e1) / steps
    n_pts, nf = g.n_pts, fb.n_f
    n_ant, n_vox = int(geo.ant.shape[1]), int(geo.vox.shape[1])
    terms = 2 * n_pts * bank.patch_size * nf + n_vox * n_ant * nf + n_vox * bank.patch_size * nf
    return {"workload": "paper training configuration: 1024 rays x 32 depths, SDF net 8x256 + reflectivity net "
                        f"4x256, PE 10 octaves, {precision}" + (" on tcgen05" if precision == "bf16" else "")
                        + "; FMCW 64 samples (3.59 GHz); 160x160 array @2mm in 3200-antenna bank patches; 32^3 heatmap",
            "n_pts": n_pts, "patch_antennas": bank.patch_size, "n_antennas": n_ant, "n_f": nf, "n_vox": n_vox,
            "ms_per_step": ms, "terms_per_step": terms, "terms_per_s": terms / (ms * 1e-3),
            "per_call_ms": {nm: round(sum(e[nm][0].elapsed_time(e[nm][1]) for e in ev) / steps, 3) for nm in names},
            "paper_context": "50,000 iterations in 32 h on one H100 (about 2.3 s per iteration, whole training "
                             "step, App. C); other hardware and code: context, not a target"}


def mlp_bench(n_pts=1 << 21, reps=5):
    """Fields kernels alone on n_pts points (4x128 MLP, PE 6 octaves, value +
    3 gradient tangents): FP32 CUDA-core forward, BF16 tensor-core forward and
    the adjoint, with algorithmic TFLOP/s (2 flops per MAC of the 4-stream GEMMs)."""
    import numpy as np
    import torch
    import geraf_inputs as gi
    import paper_2605_29097_gb300 as G
    from paper_2605_29097_gb300 import _build
    _build.build()
    spec = gi.MLPSpec()
    rng = np.random.default_rng(0)
    xyz = torch.as_tensor((np.array(spec.center)[:, None] + rng.uniform(-spec.half, spec.half, (3, n_pts)))
                          .astype(np.float32), device="cuda")
    p = torch.as_tensor(gi.mlp_init(spec, seed=1), device="cuda")
    macs = 4 * (spec.in_dim * 128 + (spec.n_hidden - 1) * 128 * 128) + 128 * 5
    out = {"mode": "mlp", "n_pts": n_pts, "mac_per_point": macs}
    for name, prec in (("fp32", G.PREC_FP32), ("bf16", G.PREC_BF16)):
        field = G.MLPField(p, precision=prec)
        for _ in range(2):
            f, grad, a, saved = G.geraf_fields(field, xyz, keep_saved=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            G.geraf_fields(field, xyz)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[f"forward_{name}_ms"] = ms
        out[f"forward_{name}_tflops"] = 2 * macs * n_pts / (ms * 1e-3) / 1e12
        d = torch.ones(n_pts, device="cuda")
        dg = torch.ones(3, n_pts, device="cuda")
        G.geraf_fields_backward(field, xyz, saved, d, dg, d)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            G.geraf_fields_backward(field, xyz, saved, d, dg, d)
        e1.record()
        torch.cuda.synchronize()
        out[f"backward_{name}_ms"] = e0.elapsed_time(e1) / reps
    G.geraf_poll_device_error()
    print(json.dumps(out), flush=True)


def blend_case(shape, reps=3, seed=0):
    """Lensless alpha blending and its adjoint on n_ray columns x n_z depths
    (SDF falling through zero along each column, reflectiveness in [0.2, 1]):
    two untimed calls, then `reps` timed with CUDA events; prints the times and
    the achieved bandwidth in the algorithmic bytes (blend: f and a read, alpha,
    T, w and t_eff written, 24 B per point; adjoint: f, a, alpha, T, dL/dw and
    dL/dT' read, dL/df and dL/da written, 32 B per point)."""
    import torch
    import paper_2605_29097_gb300 as G
    from paper_2605_29097_gb300 import _build
    _build.build()
    dev = torch.device("cuda:0")
    n_ray, n_z = shape
    gen = torch.Generator(device=dev).manual_seed(seed)
    z = torch.linspace(0.1, 0.2, n_z, device=dev)[:, None]
    sdf = (0.15 - z + 0.01 * torch.randn(n_z, n_ray, device=dev, generator=gen)).reshape(-1).contiguous()
    refl = (0.2 + 0.8 * torch.rand(n_z * n_ray, device=dev, generator=gen)).contiguous()
    apr = 0.02 * torch.rand(n_ray, device=dev, generator=gen)
    antf = 0.02 * torch.rand(1024, device=dev, generator=gen)
    d_w = torch.randn(n_z * n_ray, device=dev, generator=gen)
    d_t = torch.randn(n_z * n_ray, device=dev, generator=gen)
    s_, atx = 300.0, 1.0
    for _ in range(2):
        out = G.geraf_blend(sdf, refl, n_ray, n_z, apr, antf, s_, atx)
        G.geraf_blend_backward(sdf, refl, out[0], out[1], n_ray, n_z, s_, atx, d_w, d_t)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tf = tb = 0.0
    for _ in range(reps):
        ev[0].record()
        out = G.geraf_blend(sdf, refl, n_ray, n_z, apr, antf, s_, atx)
        ev[1].record()
        G.geraf_blend_backward(sdf, refl, out[0], out[1], n_ray, n_z, s_, atx, d_w, d_t)
        ev[2].record()
        torch.cuda.synchronize()
        tf += ev[0].elapsed_time(ev[1])
        tb += ev[1].elapsed_time(ev[2])
    n = n_ray * n_z
    tf, tb = tf / reps, tb / reps
    print(json.dumps({"mode": "blend_case", "n_pts": n, "blend_ms": tf, "blend_gbs": 24 * n / (tf * 1e-3) / 1e9,
                      "blend_backward_ms": tb, "blend_backward_gbs": 32 * n / (tb * 1e-3) / 1e9}), flush=True)


def phasor_case(shape, reps=3, seed=0):
    """Render and render adjoint of the 256^3-sample workload's array and band
    (128x128 antennas at 2 mm, 256 bins) against a `shape` stratified grid of
    its 10 cm cube, random gradients, weights and transmittances, and
    a random signal adjoint: two untimed calls of each, then `reps` timed with
    CUDA events; prints their mean times and the Chebyshev work."""
    import torch
    import geraf_inputs as gi
    import paper_2605_29097_gb300 as G
    from paper_2605_29097_gb300 import _build
    _build.build()
    dev = torch.device("cuda:0")
    wl = gi.workload("c3")
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.10, shape)
    xyz, _ = G.geraf_sample(G.make_grid(g.lo, g.pitch, g.n), gi.SAMPLE_STRATIFIED, seed=1, step=0)
    n = xyz.shape[1]
    gen = torch.Generator(device=dev).manual_seed(seed)
    grad = torch.randn(3, n, device=dev, generator=gen)
    w = torch.rand(n, device=dev, generator=gen)
    t_eff = 0.3 + 1.7 * torch.rand(n, device=dev, generator=gen)
    ant = torch.as_tensor(gi.antenna_array(wl.array_n, wl.array_n, wl.array_pitch), device=dev)
    c_ant = 0.1 * torch.rand(ant.shape[1], device=dev, generator=gen)
    b = gi.band(77e9, 81e9, wl.n_f)
    band = G.Band(b.f0, b.df, b.n_f)
    g_s = torch.view_as_complex(torch.randn(ant.shape[1], wl.n_f, 2, device=dev, generator=gen)).contiguous()
    for _ in range(2):
        G.geraf_render(xyz, grad, w, t_eff, ant, c_ant, band)
        G.geraf_render_backward(xyz, grad, w, t_eff, ant, c_ant, band, g_s)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tr = tb = 0.0
    for _ in range(reps):
        ev[0].record()
        G.geraf_render(xyz, grad, w, t_eff, ant, c_ant, band)
        ev[1].record()
        G.geraf_render_backward(xyz, grad, w, t_eff, ant, c_ant, band, g_s)
        ev[2].record()
        torch.cuda.synchronize()
        tr += ev[0].elapsed_time(ev[1])
        tb += ev[1].elapsed_time(ev[2])
    G.geraf_poll_device_error()
    work = {k: G.geraf_chebyshev_work(xyz, ant, band, tp) for k, tp in (("render", False), ("render_backward", True))}
    print(json.dumps({"mode": "phasor_case", "n_pts": n, "n_ant": ant.shape[1], "n_f": wl.n_f,
                      "render_ms": tr / reps, "render_backward_ms": tb / reps, "work": work}), flush=True)


def mlp_backward_macs(spec) -> int:
    """MACs per point of the MLP adjoint: weight gradients of every layer and
    input adjoints of the hidden layers above the first, over the 4 streams
    (value and 3 tangents), plus the head."""
    w = 128
    weight = 4 * w * (spec.in_dim + (spec.n_hidden - 1) * w)
    inputs = 4 * w * w * (spec.n_hidden - 1)
    head = 4 * w * 2 * 2
    return weight + inputs + head


def mlp_forward_macs(spec) -> int:
    """MACs per point of the MLP forward: every hidden layer over the 4 streams
    (value and 3 tangents), the head's two outputs on the value stream and f
    on the 3 tangents."""
    w = 128
    return 4 * (spec.in_dim * w + (spec.n_hidden - 1) * w * w) + w * 5


def call_flops(name, pairs, n_f, order, mlp_macs=0, n_mlp_pts=0):
    """Algorithmic flops of one call (see FLOPS_PER_TERM; MLP calls: 2 per MAC)."""
    if name in MLP_CALLS:
        return 2 * mlp_macs * n_mlp_pts
    if order > 0:
        return pairs * (order * CHEB_FLOPS_PER_ORDER + CHEB_FLOPS_PER_PAIR[name])
    return pairs * n_f * FLOPS_PER_TERM[name]


def _events(names, steps):
    import torch
    return [{nm: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for nm in names}
            for _ in range(steps)]


def _per_call(ev, names, steps):
    return {nm: sum(e[nm][0].elapsed_time(e[nm][1]) for e in ev) / steps for nm in names}


def measure_workload(name, steps, warmup, dev, world, rank, headline):
    """Times `steps` hot-path steps of one workload (after `warmup` untimed
    ones) with CUDA events on the launching stream, max over ranks; with
    `headline` also the end-to-end leg through host buffers and the clocks
    during the timed region; for the 128-bin workload also the same step
    with the per-bin recurrence forced and the signal tracing bank."""
    import dataclasses
    import torch
    import torch.distributed as dist
    import geraf_inputs as gi
    import paper_2605_29097_gb300 as G
    from paper_2605_29097_gb300 import pipeline as PL

    def barrier():
        if world > 1:
            dist.barrier()

    wl = gi.workload(name)
    geo = PL.make_geometry(wl, dev)
    spec = gi.MLPSpec()
    seeds = replica_seeds(rank)
    params_np = gi.mlp_init(spec, seed=seeds["mlp"])
    params = torch.as_tensor(params_np, device=dev)
    prec = G.PREC_BF16 if wl.precision == "bf16" else G.PREC_FP32
    field = G.MLPField(params, precision=prec)
    target = PL.synthetic_target(geo, dev)
    torch.cuda.synchronize()
    n_pts = wl.grid.n_pts
    terms = PL.terms_per_step(geo, n_pts)
    seed = seeds["sample"]
    step_id = 0
    for _ in range(warmup):
        PL.forward_backward(geo, field, target, seed, step_id)
        step_id += 1
    G.geraf_poll_device_error()
    torch.cuda.synchronize()

    ev = _events(TIMED_CALLS, steps)
    clk = ClockSampler(torch.cuda.current_device()) if headline else None
    if clk:
        clk.start()
    barrier()
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record()
    for k in range(steps):
        PL.forward_backward(geo, field, target, seed, step_id, timers=ev[k])
        step_id += 1
    t_end.record()
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop() if clk else None
    G.geraf_poll_device_error()
    ms = max_over_ranks(t_start.elapsed_time(t_end), world, dev)
    out = {"name": name, "wl": wl, "n_pts": n_pts, "n_ant": int(geo.ant.shape[1]), "n_vox": int(geo.vox.shape[1]),
           "n_f": geo.band.n_f, "terms": terms, "steps": steps, "ms": ms,
           "value": job_rate(terms, steps, world, ms), "per_call": _per_call(ev, TIMED_CALLS, steps),
           "clocks": clocks, "launches": PL.launches_per_step(field, geo.band) * steps,
           "precision": wl.precision, "mlp_fwd_macs": mlp_forward_macs(spec),
           "mlp_bwd_macs": mlp_backward_macs(spec)}

    if headline:
        # end to end through the public API with host buffers: per step the
        # inputs (MLP parameters, target heatmap, antenna positions) go host ->
        # device from pinned memory and the results (loss, parameter gradient,
        # scalar gradients) come back.
        h_params = torch.as_tensor(params_np).pin_memory()
        h_target = target.cpu().pin_memory()
        h_ant = geo.ant.cpu().pin_memory()
        h_loss = torch.empty((), dtype=torch.float64).pin_memory()
        h_dp = torch.empty_like(h_params).pin_memory()
        h_sc = torch.empty(2).pin_memory()
        d_params = torch.empty_like(params)
        d_target = torch.empty_like(target)
        d_ant = torch.empty_like(geo.ant)
        geo_e = dataclasses.replace(geo, ant=d_ant)
        field_e = G.MLPField(d_params, precision=prec)
        e_steps = max(1, min(steps, 3))
        barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(e_steps):
            d_params.copy_(h_params, non_blocking=True)
            d_target.copy_(h_target, non_blocking=True)
            d_ant.copy_(h_ant, non_blocking=True)
            r = PL.forward_backward(geo_e, field_e, d_target, seed, step_id)
            step_id += 1
            h_loss.copy_(r.loss, non_blocking=True)
            h_dp.copy_(r.d_params, non_blocking=True)
            h_sc.copy_(r.d_scalars, non_blocking=True)
            torch.cuda.synchronize()
        e_s = time.perf_counter() - w0
        barrier()
        out["e2e"] = {"value": job_rate(terms, e_steps, world, 1e3 * max_over_ranks(e_s, world, dev)),
                      "unit": "terms/s",
                      "h2d_bytes_per_step": (h_params.numel() + h_target.numel() + h_ant.numel()) * 4,
                      "d2h_bytes_per_step": 8 + h_dp.numel() * 4 + h_sc.numel() * 4}
        del geo_e, field_e, d_params, d_target, d_ant, r

    if geo.band.n_f <= 128 and name in ("c2", "c2-small"):
        # the same step with the per-bin recurrence forced (for comparison)
        b0 = geo.band
        geo_rec = dataclasses.replace(geo, band=G.Band(b0.f0, b0.df, b0.n_f, G.PHASOR_RECURRENCE))
        PL.forward_backward(geo_rec, field, target, seed, step_id)
        rec_steps = 2
        ev_rec = _events(TIMED_CALLS, rec_steps)
        torch.cuda.synchronize()
        for k in range(rec_steps):
            PL.forward_backward(geo_rec, field, target, seed, step_id + k, timers=ev_rec[k])
        torch.cuda.synchronize()
        out["per_call_rec"] = _per_call(ev_rec, TIMED_CALLS, rec_steps)
        # the paper's signal tracing bank: 16 x 16-antenna patches, one traced
        # per step, the others from the bank
        bank = PL.SignalBank(geo, (wl.array_n, wl.array_n), (16, 16))
        bank.fill(field, seed, 0)
        for k in range(warmup):
            PL.forward_backward_bank(bank, field, target, seed, step_id + k)
        torch.cuda.synchronize()
        eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        eb0.record()
        for k in range(steps):
            PL.forward_backward_bank(bank, field, target, seed, step_id + warmup + k)
        eb1.record()
        torch.cuda.synchronize()
        bank_ms = eb0.elapsed_time(eb1) / steps
        nf, na, nv = geo.band.n_f, out["n_ant"], out["n_vox"]
        out["bank_step"] = {"patch_antennas": bank.patch_size, "n_patches": bank.n_patch, "ms_per_step": bank_ms,
                            "full_trace_ms_per_step": ms / steps, "speedup": (ms / steps) / bank_ms,
                            "terms_per_step": 2 * n_pts * bank.patch_size * nf + nv * na * nf
                            + nv * bank.patch_size * nf}
        del bank
    xyz_o, _ = G.geraf_sample(geo.grid, geo.mode, seed, 0, device=dev)
    out["orders"] = {"points": G.geraf_chebyshev_order(xyz_o, geo.ant, geo.band),
                     "voxels": G.geraf_chebyshev_order(geo.vox, geo.ant, geo.band)}
    # orders each Chebyshev call evaluates (per split or point group; the mean
    # over the points of the orders per pair the running kernel instance computes)
    out["cheb_work"] = {"render": G.geraf_chebyshev_work(xyz_o, geo.ant, geo.band, False),
                        "render_backward": G.geraf_chebyshev_work(xyz_o, geo.ant, geo.band, True),
                        "filter": G.geraf_chebyshev_work(geo.vox, geo.ant, geo.band, True),
                        "filter_backward": G.geraf_chebyshev_work(geo.vox, geo.ant, geo.band, False)}
    if headline and rank == 0 and not getattr(measure_workload, "no_cpu", False):
        # intermediate arrays of one step for the oracle sample
        f, grad, a, _ = G.geraf_fields(field, xyz_o)
        _, apr = G.geraf_sample(geo.grid, geo.mode, seed, 0, device=dev)
        fa, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
        fn, _, _, _ = G.geraf_fields(field, geo.ant, want_grad=False, want_refl=False)
        _, _, w, t_eff, c_ant = G.geraf_blend(f, a, geo.n_ray, geo.n_z, fa, fn, geo.sharpness, geo.a_tx)
        tps, secs, cterms, desc = cpu_baseline_sample(geo, xyz_o, grad, w, t_eff, c_ant)
        out["cpu_baseline"] = {"value": tps, "unit": "terms/s", "cores": oracle_threads(), "kind": "oracle",
                               "sample": desc + f"; {cterms:.3g} terms in {secs:.1f} s"}
        del f, grad, a, fa, fn, w, t_eff, c_ant, apr
    del xyz_o, geo, field, target, params
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def roofline_of(m, peaks, sm_count):
    """Per-call roofline figures of a measured workload (measure_workload) and
    the dominant call: the one with the largest event time inside the timed
    region, over every timed call (phasor sums and MLP)."""
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sm_count * 128 * 2 * max_mhz * 1e6 / 1e12       # FMA = 2 flops per lane per clock
    bf16_peak = peaks.get("bf16_tflops_sustained")
    n_pts, n_ant, n_vox, n_f = m["n_pts"], m["n_ant"], m["n_vox"], m["n_f"]
    pairs = {"render": n_pts * n_ant, "render_backward": n_pts * n_ant, "filter": n_vox * n_ant,
             "filter_backward": n_vox * n_ant, "fields": n_pts, "fields_backward": n_pts}
    cw = m["cheb_work"]
    order_of = {nm: cw[nm][3] for nm in PHASOR_CALLS}
    whole = {"render": m["orders"]["points"], "render_backward": m["orders"]["points"],
             "filter": m["orders"]["voxels"], "filter_backward": m["orders"]["voxels"]}
    macs = {"fields": m["mlp_fwd_macs"], "fields_backward": m["mlp_bwd_macs"]}
    tensor = m["precision"] == "bf16" and bf16_peak

    def roof(nm, ms, order):
        fl = call_flops(nm, pairs[nm], n_f, order, macs.get(nm, 0), n_pts)
        tf = fl / (ms * 1e-3) / 1e12
        if nm in MLP_CALLS and tensor:
            r = {"bound": "tensor", "peak": bf16_peak, "peak_basis": "MEASURED_PEAKS bf16_tflops_sustained"}
        else:
            r = {"bound": "alu", "peak": fp32_peak, "peak_basis": "FP32 FMA units x max SM clock"}
        r.update(ms=round(ms, 3), tflops=tf, frac=tf / r["peak"])
        if nm in PHASOR_CALLS and order > 0:
            fw = call_flops(nm, pairs[nm], n_f, whole[nm])
            fo = pairs[nm] * order * CHEB_FLOPS_PER_ORDER
            r.update(orders_per_pair=round(order, 3), whole_set_order=whole[nm],
                     frac_orders_only=fo / (ms * 1e-3) / 1e12 / fp32_peak,
                     frac_whole_set_order=fw / (ms * 1e-3) / 1e12 / fp32_peak)
        return r

    calls = {nm: roof(nm, m["per_call"][nm], order_of.get(nm, 0)) for nm in TIMED_CALLS}
    dom = max(TIMED_CALLS, key=lambda k: m["per_call"][k])
    return calls, dom, fp32_peak, max_mhz, order_of


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the C2 step, the training-step comparison and the paper configuration")
    ap.add_argument("--mlp-bench", type=int, default=0, metavar="N_PTS",
                    help="time only the fields kernels on N_PTS points and exit")
    ap.add_argument("--paper-config", action="store_true",
                    help="time only the paper's own training configuration and exit")
    ap.add_argument("--train-step", action="store_true",
                    help="run only the uniform vs proposal-cell training-step comparison and exit")
    ap.add_argument("--blend-case", default="", metavar="N_RAY,N_Z",
                    help="time only blend and its adjoint on N_RAY columns x N_Z depths and exit")
    ap.add_argument("--phasor-case", default="", metavar="NX,NY,NZ",
                    help="time only render and render adjoint of the 256^3-sample workload's array and band "
                         "against an NX x NY x NZ stratified grid of its cube (the profiling case) and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.mlp_bench:
        mlp_bench(args.mlp_bench)
        return
    if args.blend_case:
        blend_case(tuple(int(v) for v in args.blend_case.split(",")), reps=args.steps)
        return
    if args.phasor_case:
        phasor_case(tuple(int(v) for v in args.phasor_case.split(",")), reps=args.steps)
        return
    if args.train_step:
        import torch
        from paper_2605_29097_gb300 import _build
        _build.build()
        print(json.dumps({"mode": "train_step", **train_step_compare(torch.device("cuda", local))}), flush=True)
        return
    if args.paper_config:
        import torch
        from paper_2605_29097_gb300 import _build
        _build.build()
        dev = torch.device("cuda", local)
        print(json.dumps({"mode": "paper_config", "fp32": paper_config_step(dev),
                          "bf16": paper_config_step(dev, precision="bf16")}), flush=True)
        return

    import torch
    import torch.distributed as dist
    from paper_2605_29097_gb300 import _build

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    _build.build()
    measure_workload.no_cpu = args.no_cpu_baseline

    m = measure_workload(args.workload, args.steps, args.warmup, dev, world, rank, headline=True)
    extras = {}
    if not args.no_extras and args.workload == "c3":
        extras["c2"] = measure_workload("c2", min(args.steps, 10), 3, dev, world, rank, headline=False)

    if rank == 0:
        peaks = measured_peaks()
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        calls, dom, fp32_peak, max_mhz, order_of = roofline_of(m, peaks, sm_count)
        fam = "c3" if args.workload.startswith("c3") else "c2"
        traffic, traffic_basis = None, NCU_DRAM_UNSCALED.get((fam, dom), "no ncu capture of this kernel version")
        if (fam, dom) in NCU_DRAM:
            b_cap, unit, n_cap, basis = NCU_DRAM[(fam, dom)]
            n_full = m["n_pts"] if unit == "points" else m["n_vox"]
            traffic = b_cap * n_full / n_cap
            traffic_basis = basis + (f", scaled by {unit} from {n_cap} to {n_full}" if n_cap != n_full else "")
        d = calls[dom]
        line = {
            "metric": METRIC, "value": m["value"], "unit": "terms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[m["precision"]], "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n_pts": m["n_pts"], "n_ant": m["n_ant"],
                       "n_f": m["n_f"], "n_vox": m["n_vox"], "terms_per_step": m["terms"],
                       "l2": "inputs larger than L2 (the per-step MLP activations alone are gigabytes)",
                       "parallelism": f"replicas x{world}"},
            "per_call_ms": {k: round(v, 3) for k, v in m["per_call"].items()},
            "roofline": {"bound": d["bound"], "kernel": dom, "achieved": d["tflops"], "peak": d["peak"],
                         "unit": "TFLOP/s", "frac": d["frac"], "traffic": traffic, "traffic_basis": traffic_basis,
                         "peak_basis": (f"{sm_count} SMs x 128 FP32 lanes x 2 flops (FMA) x {max_mhz:.0f} MHz"
                                        if d["bound"] == "alu" else d["peak_basis"]),
                         "work_basis": ("Chebyshev phasor sums: pairs x (the form's fixed per-pair flops "
                                        f"{CHEB_FLOPS_PER_PAIR} + 6 flops x orders evaluated per pair) (the "
                                        "running instance's orders per split or point group, mean over the "
                                        "points, geraf_chebyshev_work; calls[*].frac_orders_only counts the "
                                        "orders alone, calls[*].frac_whole_set_order one expansion of the "
                                        "whole set's order instead); per-bin "
                                        "recurrence: terms x 10 (render, filter adjoint) or 8 (filter, render "
                                        f"adjoint) flops; MLP forward 2 x {m['mlp_fwd_macs']} and adjoint "
                                        f"2 x {m['mlp_bwd_macs']} flops per point"),
                         "calls": calls,
                         "mlp": {nm: calls[nm] for nm in MLP_CALLS}},
            "phasor_method": {"chebyshev_order": m["orders"],
                              "chebyshev_work": {nm: {"whole_set_order": w[0], "max_part_order": w[1],
                                                      "instance_orders": w[2], "orders_per_pair": round(w[3], 3)}
                                                 for nm, w in m["cheb_work"].items()}},
            "cpu_baseline": m.get("cpu_baseline"),
            "e2e": m["e2e"],
            "gpu_launches": m["launches"],
            "clocks": m["clocks"],
        }
        for src in [m] + list(extras.values()):
            if "per_call_rec" in src:
                # the per-bin recurrence forced on the same step: per-call times and roofline
                rec = {}
                for nm in PHASOR_CALLS:
                    pr = src["n_pts"] if nm.startswith("render") else src["n_vox"]
                    t_ms = src["per_call_rec"][nm]
                    tf = call_flops(nm, pr * src["n_ant"], src["n_f"], 0) / (t_ms * 1e-3) / 1e12
                    rec[nm] = {"ms": round(t_ms, 3), "tflops": tf, "frac": tf / fp32_peak}
                block = {"recurrence_per_call_ms": {k: round(src["per_call_rec"][k], 3) for k in PHASOR_CALLS},
                         "recurrence_roofline": rec,
                         "recurrence_terms_per_s": 2 * (src["n_pts"] + src["n_vox"]) * src["n_ant"] * src["n_f"]
                         / (sum(src["per_call_rec"][k] for k in PHASOR_CALLS) * 1e-3)}
                if src is m:
                    line["phasor_method"].update(block)
                else:
                    src["phasor_method_rec"] = block
        if "bank_step" in m:
            line["bank_step"] = m["bank_step"]
        if "c2" in extras:
            c = extras["c2"]
            ccalls, cdom, _, _, _ = roofline_of(c, peaks, sm_count)
            line["c2"] = {"workload": WORKLOADS["c2"], "dtype": DTYPES[c["precision"]], "steps": c["steps"],
                          "ms_per_step": c["ms"] / c["steps"], "value": c["value"], "unit": "terms/s",
                          "terms_per_step": c["terms"],
                          "per_call_ms": {k: round(v, 3) for k, v in c["per_call"].items()},
                          "roofline_calls": ccalls, "dominant": cdom,
                          "chebyshev_work": {nm: {"whole_set_order": w[0], "max_part_order": w[1],
                                                  "instance_orders": w[2], "orders_per_pair": round(w[3], 3)}
                                             for nm, w in c["cheb_work"].items()},
                          "phasor_method_recurrence": c.get("phasor_method_rec"),
                          "bank_step": c.get("bank_step")}
        if not args.no_extras and args.workload in ("c3", "c2"):
            torch.cuda.empty_cache()
            line["train_step"] = train_step_compare(dev)
            torch.cuda.empty_cache()
            line["paper_config"] = paper_config_step(dev)
            torch.cuda.empty_cache()
            line["paper_config_bf16"] = paper_config_step(dev, precision="bf16")
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
