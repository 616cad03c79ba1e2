#!/usr/bin/env python
"""Directional wavelet transforms per second on GB300.

Workload: 16 real maps per GPU at L = 256, N = 8, lambda = 2, J0 = 2, spin 0, McEwen-Wiaux
sampling; harmonic coefficients seeded complex Gaussian with variance (l+1)^-2 and the
reality condition (synth.py), synthesised to maps by the library's inverse SHT before
timing.  One step = analysis + synthesis (Algorithm 1) of the whole batch: the metric is
the round trip per map, the paper's protocol (Sec. 4.4).  Default precision "fp64_tc":
float64 accuracy with precomputed Wigner-d tables built at plan creation (outside the timed
region, like the paper's precomputed mode, Sec. 4.2) and the l-contractions on the tensor
cores by exact integer slicing; the other modes are timed on the same
inputs under "other_modes", and the same maps sampled on Driscoll-Healy grids under
"samplings".

value  device time (CUDA events on the launching stream) of K steps, inputs resident in
       HBM, L2 flushed (256 MB write) between steps; max over ranks.
e2e    same metric through the public API with host buffers: pinned host maps copied in,
       analysis + synthesis, reconstructed maps copied back, every step.
Multi-GPU: replicas only (each rank transforms its own maps; no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L, N, LAM, J0, B = 256, 8, 2.0, 2, 16
METRIC = "wavelet transforms/s (fwd+inv) at L=256,N=8"
UNIT = "transforms/s"
WORKLOAD = "sphere L=256 N=8 lambda=2 J0=2 spin0, 16 real maps/GPU, MW sampling, a_lm ~ CN(0,(l+1)^-2)"
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 2 FP64 FMA/clk x 2.07 GHz (derived)
# A compensated-float32 multiply-add (comp32.cuh acc_add) issues 12 FP32-pipe instructions for one
# float64-accurate real multiply-add (2 flop): 152 SMs x 128 lanes x 2.07 GHz x 2/12.
C32_PEAK_TFLOPS = 152 * 128 * 2.07e9 * 2 / 12 / 1e12
PEAKS = {
    "fp64": (C32_PEAK_TFLOPS, "derived: compensated-float32 multiply-add = 12 FP32 instructions; "
             "152 SMs x 128 FP32 lanes x 2.07 GHz x 2 flop / 12"),
    "fp64_native": (FP64_PEAK_TFLOPS, "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz (probe measured "
                    "1.196 TFLOP/s FP64 at 1987 MHz)"),
}
PEAKS["fp32_split"] = PEAKS["bf16"] = PEAKS["fp64_table"] = PEAKS["fp64_tc"] = PEAKS["fp64"]
# DRAM bytes (read + write) per launch of a kernel region, mean over one step's launches, from one
# ncu capture of the kernels as they are built now.  An entry is dropped whenever its kernel
# changes; a missing entry reports null.
TRAFFIC_BYTES = {("fp64", "wigner_forward"): 368.88e6 / 9 + 0.54e6 / 9,   # k_wig_fwd, on-the-fly mode
                 ("fp64_table", "wigner_forward"): 209.0e6}   # k_tab_fwd


def hbm_peak():
    """Measured copy bandwidth of the GB300s (driver-written), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs: torch copy, read+write bytes)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback: 6.8 TB/s, one earlier GB300 measurement"


def dft_bytes_per_step(plan):
    """Algorithmic HBM bytes of one direction of azimuthal DFTs in one step: the pixels of every
    transform (spin SHT, scaling function, each wavelet scale; real float64 samples,
    B (2N_j-1) L_j (2L_j-1)) moved once -- the map in and the wavelet coefficients back.  The
    m-columns between the DFTs and the l-contractions are an intermediate of this design, not
    algorithmic traffic, and are not counted."""
    def one(Lt, Nt):
        return B * (2 * Nt - 1) * Lt * (2 * Lt - 1) * 8
    tot = one(L, 1) + one(plan.L_phi, 1)
    for s in range(plan.nscales):
        tot += one(plan.Lj[s], plan.Nj[s])
    return tot


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_items(rank: int):
    """Map indices of one replica's batch: rank r transforms maps r*B .. r*B+B-1 of the seeded
    workload (replicas only: no rank reads another's data)."""
    return [b + B * rank for b in range(B)]


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's time (the job's time); identity on one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = f"/tmp/s2w_clocks_{os.getpid()}.csv"

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(torch, plan, rank):
    import numpy as np
    import synth
    flm = np.stack([synth.flm_random(L, synth.rng_for(2, item), reality=True)[:, L - 1:]
                    for item in replica_items(rank)])
    flm_d = torch.from_numpy(np.ascontiguousarray(flm)).cuda()
    f = plan.empty_map()
    plan.sht_inverse(flm_d, f)
    torch.cuda.synchronize()
    return flm, f


def cpu_baseline_sample():
    """The float64 oracle timed on this host's cores on one map round trip of the workload."""
    import numpy as np
    import synth
    from oracle import harmonic, wavelet
    flm = synth.flm_random(L, synth.rng_for(2, 0), reality=True)
    f = harmonic.sht_inverse(flm, L).real
    t0 = time.perf_counter()
    W, Wp = wavelet.analysis(f, L, N, LAM, J0, 0, True)
    f2 = wavelet.synthesis(W, Wp, L, N, LAM, J0, 0, True)
    dt = time.perf_counter() - t0
    err = float(np.abs(harmonic.sht_forward(f2, L) - flm).max() / np.abs(flm).max())
    return dt, err


PRECISIONS = {"fp64": 0, "fp64_table": 0, "fp64_native": 3, "fp32_split": 1, "bf16": 2, "fp64_tc": 4}


def contraction_kernels_per_step(precision, nscales):
    """Library kernels of the 2 (nscales + 2) contractions of one step (analysis + synthesis: the
    SHT, the scaling transform and every wavelet scale, each once per direction): exponent pass +
    slicing pass + GEMM on the sliced path (fp64_tc: every transform; the reduced modes: the SHT
    and the scaling transform), operand preparation + GEMM for the reduced modes' wavelet scales,
    one kernel in the float64 modes."""
    if precision == "fp64_tc":
        return 3 * 2 * (nscales + 2)
    if precision in ("fp32_split", "bf16"):
        return 3 * 2 * 2 + 2 * 2 * nscales
    return 2 * (nscales + 2)

# kernels of one azimuthal DFT by form (forward, inverse): 0 SIMT (one kernel); 1 direct tensor-core
# GEMM (slicing prologue + GEMM); 2 prime-factor (forward: gamma-DFT prologue + tensor-core kernel;
# inverse: column prologue + tensor-core kernel + gamma synthesis)
DFT_KERNELS = {0: (1, 1), 1: (2, 2), 2: (2, 3)}
PRECOMPUTE = {"fp64_table": 1}
PRECISION_DOC = {
    "fp64": "float64 accuracy: Wigner-d recursion in float64; l-contractions, DFTs and colatitude "
            "quadrature in compensated float32 pairs",
    "fp64_native": "plain float64: every step in native float64",
    "fp64_table": "float64 accuracy: precomputed Wigner-d tables (float64 recursion at plan time, "
                  "colatitude quadrature folded into the forward tables) in float pairs; "
                  "compensated-float32 table contractions and DFTs",
    "fp32_split": "reduced: tcgen05 contractions on precomputed Wigner-d tiles, fp16 hi/lo operands "
                  "(3 MMAs), float32 accumulation; plain float32 DFTs; spin SHT and scaling transform "
                  "float64-accurate (the fp64_tc kernels)",
    "bf16": "reduced: split-bf16, tcgen05 contractions on precomputed Wigner-d tiles, bf16 hi/lo tables "
            "and data (3 MMAs), float32 accumulation; plain float32 DFTs; spin SHT and scaling transform "
            "float64-accurate (the fp64_tc kernels)",
    "fp64_tc": "float64 accuracy on the tensor cores: precomputed Wigner-d tables and the data cut into "
               "seven 7-bit integer slices (bf16), 28 slice products per K step summed exactly in float32 "
               "TMEM accumulators (error-free splitting); azimuthal DFTs on the tensor cores by the same "
               "slicing or in compensated float32, whichever the autotuner measured faster per transform",
}
# Differentiation study: gradient of sum_j mean |W^j|^2 w.r.t. the pixels of 8 real maps at
# L = 512, N = 4, lambda = 2, J0 = 3 (analysis + its hand-written adjoint per step).
DIFF_L, DIFF_N, DIFF_J0, DIFF_B = 512, 4, 3, 8


# Ball study: one real field at L = P = 128, N = 4, lambda = nu = 2, J0 = J0' = 0.
BALL_L, BALL_P, BALL_N = 128, 128, 4


def run_ball(torch, s2w, stream, flush, steps, precision, autotune=True):
    """Ball wavelet round trips per second (analysis + synthesis of one field, device time,
    L2 flushed) and the round-trip error."""
    import numpy as np
    import synth
    plan = s2w.BallWavPlan(BALL_L, BALL_N, BALL_P, 2.0, 2.0, 0, 0, batch=1, precision=PRECISIONS[precision],
                           precompute=PRECOMPUTE.get(precision, 0))
    if autotune:
        plan.autotune()
    bp = s2w.BallPlan(BALL_L, BALL_P, reality=True, batch=1)
    flmp = synth.flmp_random(BALL_L, BALL_P, synth.rng_for(5, 0), reality=True)[None, :, :, BALL_L - 1:]
    f = plan.empty_field()
    bp.sl_inverse(torch.from_numpy(np.ascontiguousarray(flmp)).cuda(), f)
    wav, scal, f2 = plan.empty_wav(), plan.empty_field(), plan.empty_field()
    for _ in range(3):
        plan.forward(f, wav, scal)
        plan.inverse(wav, scal, f2)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.nvtx.range_push("ball_timed")   # lets a profiler select the ball's timed launches
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        plan.forward(f, wav, scal)
        plan.inverse(wav, scal, f2)
        e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    plan.check()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    err = float((f2 - f).abs().max() / f.abs().max())
    # algorithmic HBM bytes of one round trip: the wavelet coefficients written by the analysis and
    # read by the synthesis, the field read, the scaling coefficients written and read, the
    # reconstruction written (float64 samples; the intermediates between the steps are not counted)
    alg = 2 * plan.wav_elems * 8 + 4 * plan.field_elems * 8
    mean_ms = sum(ms) / len(ms)
    hbm, hbm_src = hbm_peak()
    achieved = alg / (mean_ms * 1e-3) / 1e9
    out = {"workload": f"ball L={BALL_L} P={BALL_P} N={BALL_N} lambda=nu=2 J0=J0'=0, 1 real field, "
                       "f_lmp ~ N(0, (l+1)^-2 (p+1)^-2)",
           "value": len(ms) / (sum(ms) * 1e-3), "unit": "ball transforms/s (fwd+inv)",
           "ms_per_step": mean_ms, "precision": precision, "max_rel_err": err,
           "wavelet_coefficients_bytes": int(plan.wav_elems * 8), "autotuned": bool(autotune),
           "roofline": {"bound": "hbm", "algorithmic_bytes_per_step": int(alg), "achieved": achieved,
                        "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "peak_source": hbm_src}}
    plan.close()
    bp.close()
    return out


def run_sampling(torch, s2w, stream, flush, steps, flm, precision, autotune):
    """The headline workload on Driscoll-Healy grids (2L rings): transforms per second of the
    same 16 band-limited maps sampled on the DH grid, and the round-trip error."""
    import numpy as np
    plan = s2w.Plan(L, N, LAM, J0, reality=True, batch=B, precision=PRECISIONS[precision],
                    precompute=PRECOMPUTE.get(precision, 0), sampling=s2w.S2W_SAMPLING_DH)
    if autotune:
        plan.autotune()
    f = plan.empty_map()
    plan.sht_inverse(torch.from_numpy(np.ascontiguousarray(flm)).cuda(), f)
    wav, scal, f2 = plan.empty_wav(), plan.empty_scal(), plan.empty_map()
    for _ in range(3):
        plan.forward(f, wav, scal)
        plan.inverse(wav, scal, f2)
    ms = time_steps(torch, plan, f, wav, scal, f2, flush, stream, steps)
    plan.check()
    flm2 = plan.empty_flm()
    plan.sht_forward(f2, flm2)
    err = float(np.abs(flm2.cpu().numpy() - flm).max() / np.abs(flm).max())
    out = {"dh": {"value": B * len(ms) / (sum(ms) * 1e-3), "unit": UNIT, "ms_per_step": sum(ms) / len(ms),
                  "rings": plan.R, "precision": precision, "max_rel_err": err,
                  "map_bytes": int(plan.map_elems * 8), "wavelet_coefficients_bytes": int(plan.wav_elems * 8)}}
    plan.close()
    return out


# Batching study: 64 complex maps, L in {64, 128, 256, 512} x 16 (spin 0 and 2 alternating),
# N = 4, lambda = 2, white coefficients; 8 plans of 8 maps.
def run_batching(torch, s2w, stream, flush, steps, autotune, precision="fp64_tc"):
    import numpy as np
    import synth
    plans, fd, wavs, scals, outs = [], [], [], [], []
    for L in (64, 128, 256, 512):
        for spin in (0, 2):
            p = s2w.Plan(L, 4, 2.0, 0, spin=spin, reality=False, batch=8, precision=PRECISIONS[precision])
            if autotune:
                p.autotune()
            flm = np.stack([synth.flm_random(L, synth.rng_for(3, 16 * L + 2 * b + spin // 2), spin=spin,
                                             variance=lambda l: np.ones_like(l)) for b in range(8)])
            x = p.empty_map()
            p.sht_inverse(torch.from_numpy(flm).cuda(), x)
            plans.append(p)
            fd.append(x)
            wavs.append(p.empty_wav())
            scals.append(p.empty_scal())
            outs.append(p.empty_map())

    def sequential():
        for p, x, w, sc, o in zip(plans, fd, wavs, scals, outs):
            p.forward(x, w, sc)
            p.inverse(w, sc, o)

    batch = s2w.Batch(plans, fd, wavs, scals, outs, what=2)
    res = {}
    for name, fn in (("sequential_one_stream", sequential), ("graph", batch.launch)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        res[name] = {"value": 64 * len(ms) / (sum(ms) * 1e-3), "ms_per_step": sum(ms) / len(ms)}
    for p in plans:
        p.check()
    err = max(float((o - x).abs().max() / x.abs().max()) for x, o in zip(fd, outs))
    batch.close()
    for p in plans:
        p.close()
    return {"workload": "64 complex maps, L in {64,128,256,512} x 16, spin 0/2 alternating, N=4, lambda=2, "
                        f"white a_lm; 8 plans x 8 maps, precision {precision}",
            "precision_detail": PRECISION_DOC[precision],
            "unit": "transforms/s (fwd+inv)", "autotuned": bool(autotune), "max_rel_err": err, **res}


def run_differentiation(torch, s2w, stream, flush, steps):
    """Loss-gradient evaluations per second (analysis + adjoint, device time, L2 flushed) and
    a central finite-difference check of one directional derivative."""
    import numpy as np
    import synth
    plan = s2w.Plan(DIFF_L, DIFF_N, LAM, DIFF_J0, reality=True, batch=DIFF_B, precision=PRECISIONS["fp64"])
    flm = np.stack([synth.flm_random(DIFF_L, synth.rng_for(4, b), reality=True)[:, DIFF_L - 1:]
                    for b in range(DIFF_B)])
    f = plan.empty_map()
    plan.sht_inverse(torch.from_numpy(flm).cuda(), f)
    wav, scal, gf = plan.empty_wav(), plan.empty_scal(), plan.empty_map()
    gscal = torch.zeros_like(scal)
    norm = torch.empty_like(wav)
    for s in range(plan.nscales):
        a, b = plan.wav_offsets[s], plan.wav_offsets[s + 1]
        norm[:, a:b] = 2.0 / (b - a)

    def step(x):
        plan.forward(x, wav, scal)
        torch.mul(wav, norm, out=wav)          # dLoss/dW^j = 2 W^j / n_j
        plan.forward_adjoint(wav, gscal, gf)

    for _ in range(3):
        step(f)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        step(f)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    plan.check()
    # the gradient against central differences of the library's own loss.  The loss is quadratic
    # in f, so (L(f + h v) - L(f - h v)) / 2h is the directional derivative for every h; h of the
    # size of the map itself keeps the loss's rounding small against the difference
    step(f)
    g = gf.clone()

    def loss(x):
        plan.forward(x, wav, scal)
        return sum(float((plan.scale_view(wav, s) ** 2).mean(dim=(1, 2, 3)).sum()) for s in range(plan.nscales))
    fd_rel = 0.0
    for k in range(4):   # seeded band-limited directions
        vl = np.stack([synth.flm_random(DIFF_L, synth.rng_for(4, 100 + 8 * k + b), reality=True)[:, DIFF_L - 1:]
                       for b in range(DIFF_B)])
        v = plan.empty_map()
        plan.sht_inverse(torch.from_numpy(vl).cuda(), v)
        an = float((g * v).sum())
        fd = (loss(f + 0.5 * v) - loss(f - 0.5 * v)) / 1.0
        fd_rel = max(fd_rel, abs(fd - an) / abs(an))
    # 32 seeded single pixels: h = 1e3 balances the loss's rounding (which grows with h^2) against
    # the size of the difference; error relative to the largest of the 32 gradient entries
    rng = synth.rng_for(4, 200)
    pix = [(int(rng.integers(DIFF_B)), int(rng.integers(DIFF_L)), int(rng.integers(2 * DIFF_L - 1)))
           for _ in range(32)]
    gp, fdp = [], []
    for (b, t, p) in pix:
        e = torch.zeros_like(f)
        e[b, t, p] = 1e3
        fdp.append((loss(f + e) - loss(f - e)) / 2e3)
        gp.append(float(g[b, t, p]))
    fd_pix_rel = max(abs(a - c) for a, c in zip(fdp, gp)) / max(abs(c) for c in gp)
    # inner-product identity <A^H u, v> = <u, A v> for seeded random u (wavelet and scaling
    # coefficients) and v (pixels)
    u = torch.from_numpy(synth.pixels_random(tuple(wav.shape), synth.rng_for(4, 300))).cuda()
    us = torch.from_numpy(synth.pixels_random(tuple(scal.shape), synth.rng_for(4, 301))).cuda()
    v = torch.from_numpy(synth.pixels_random(tuple(f.shape), synth.rng_for(4, 302))).cuda()
    plan.forward_adjoint(u, us, gf)
    plan.forward(v, wav, scal)
    lhs, rhs = float((gf * v).sum()), float((u * wav).sum() + (us * scal).sum())
    plan.check()
    plan.close()
    return {"workload": f"L={DIFF_L} N={DIFF_N} lambda=2 J0={DIFF_J0}, {DIFF_B} real maps, "
                        "loss sum_j mean |W^j|^2, gradient w.r.t. pixels by the adjoint",
            "value": DIFF_B * len(ms) / (sum(ms) * 1e-3), "unit": "gradients/s (per map)",
            "ms_per_step": sum(ms) / len(ms),
            "fd_check_rel": fd_rel, "fd_check": "4 seeded band-limited directions, h = 0.5, max rel err",
            "fd_pixels_rel": fd_pix_rel, "fd_pixels": "32 seeded single pixels, h = 1e3, err / max |grad|",
            "inner_product_rel": abs(lhs - rhs) / abs(rhs)}


def time_steps(torch, plan, f, wav, scal, f2, flush, stream, steps):
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        plan.forward(f, wav, scal)
        plan.inverse(wav, scal, f2)
        ends[k].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2402_01282_gb300 as s2w

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = s2w.Plan(L, N, LAM, J0, reality=True, batch=B, precision=PRECISIONS[args.precision],
                    precompute=PRECOMPUTE.get(args.precision, 0))
    plan_create_s = time.perf_counter() - t0
    table_bytes, workspace_bytes = plan.device_bytes()
    t0 = time.perf_counter()
    if not args.no_autotune:
        plan.autotune()
    autotune_s = time.perf_counter() - t0
    flm, f = make_inputs(torch, plan, rank)
    wav, scal, f2 = plan.empty_wav(), plan.empty_scal(), plan.empty_map()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.forward(f, wav, scal)
        plan.inverse(wav, scal, f2)
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(local)
    gpu_id = getattr(props, "uuid", None)
    gpu_id = f"GPU-{gpu_id}" if gpu_id is not None and not str(gpu_id).startswith("GPU-") else str(local)
    sampler = ClockSampler(str(gpu_id)) if rank == 0 else None
    plan.trace(True, capacity=64 * (args.steps + 1))
    plan.trace_reset()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    torch.cuda.nvtx.range_push("timed")   # lets a profiler select the timed launches
    step_ms = time_steps(torch, plan, f, wav, scal, f2, flush, stream, args.steps)
    torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    plan.check()
    total_ms = sum(step_ms)
    trace = plan.trace_read()
    plan.trace(False)
    total_ms = max_over_ranks(total_ms, dist, "cuda")

    # accuracy of the round trip (Sec. 4.4 protocol): f_lm' = Y f' against the seeded f_lm
    flm2 = plan.empty_flm()
    plan.sht_forward(f2, flm2)
    err = float(np.abs(flm2.cpu().numpy() - flm).max() / np.abs(flm).max())

    # end to end through the public API with host buffers
    f_host = f.cpu().pin_memory()
    out_host = torch.empty_like(f_host).pin_memory()
    f_dev = torch.empty_like(f)
    for _ in range(2):
        f_dev.copy_(f_host, non_blocking=True)
        plan.forward(f_dev, wav, scal)
        plan.inverse(wav, scal, f2)
        out_host.copy_(f2, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        f_dev.copy_(f_host, non_blocking=True)
        plan.forward(f_dev, wav, scal)
        plan.inverse(wav, scal, f2)
        out_host.copy_(f2, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")
    e2e_err = float(np.abs(out_host.numpy() - f_host.numpy()).max() / np.abs(f_host.numpy()).max())

    # the other precision modes on the same inputs, for comparison (not the headline)
    other = {}
    if not args.no_compare:
        for name in ("fp64", "fp64_table", "fp64_tc", "fp64_native", "fp32_split", "bf16"):
            if name == args.precision:
                continue
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            alt = s2w.Plan(L, N, LAM, J0, reality=True, batch=B, precision=PRECISIONS[name],
                           precompute=PRECOMPUTE.get(name, 0))
            alt_create_s = time.perf_counter() - t0
            alt_tab, alt_ws = alt.device_bytes()
            for _ in range(2):
                alt.forward(f, wav, scal)
                alt.inverse(wav, scal, f2)
            ms = time_steps(torch, alt, f, wav, scal, f2, flush, stream, max(2, args.steps // 2))
            alt.check()
            flm3 = plan.empty_flm()
            plan.sht_forward(f2, flm3)
            other[name] = {"value": B * len(ms) / (sum(ms) * 1e-3), "ms_per_step": sum(ms) / len(ms),
                           "max_rel_err": float(np.abs(flm3.cpu().numpy() - flm).max() / np.abs(flm).max()),
                           "plan_create_s": alt_create_s, "table_bytes": alt_tab, "workspace_bytes": alt_ws,
                           "precision": PRECISION_DOC[name]}
            alt.close()
    diff = None
    if not args.no_diff:
        diff = run_differentiation(torch, s2w, stream, flush, max(3, args.steps // 2))
    batching = None
    if not args.no_batching:
        batching = run_batching(torch, s2w, stream, flush, max(3, args.steps // 2), not args.no_autotune)
        # the study's "FP32 contractions with FP64 recursion" arm: split-precision tensor-core
        # contractions against tables computed by the float64 recursion
        batching["fp32_split"] = {k: v for k, v in run_batching(torch, s2w, stream, flush, max(3, args.steps // 2),
                                                                not args.no_autotune, "fp32_split").items()
                                  if k in ("max_rel_err", "sequential_one_stream", "graph")}
    samplings = None
    if not args.no_sampling:
        samplings = run_sampling(torch, s2w, stream, flush, max(3, args.steps // 2), flm, args.precision,
                                 not args.no_autotune)
    ball = None
    if not args.no_ball:
        ball = run_ball(torch, s2w, stream, flush, max(3, args.steps // 2), args.precision, not args.no_autotune)
        # the ball study's split-precision arm: reduced sphere contractions, radial maps on the
        # tensor cores
        ball["fp32_split"] = {k: v for k, v in run_ball(torch, s2w, stream, flush, max(3, args.steps // 2),
                                                        "fp32_split", not args.no_autotune).items()
                              if k in ("value", "ms_per_step", "max_rel_err")}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    maps = B * world * args.steps
    dft_forms = [plan.dft_forms(k) for k in range(plan.nscales + 2)]
    dom = max(trace.items(), key=lambda kv: kv[1][1])
    name, (launches, ms, flops) = dom
    per_kernel = {k: {"launches": v[0], "ms": v[1], "tflops": (v[2] / (v[1] * 1e-3) / 1e12) if v[1] else 0.0}
                  for k, v in trace.items()}
    if args.precision == "fp64_tc" and name.startswith("dft"):
        # tensor-core DFTs: the speed of light is HBM, the DFT's own input and output read and
        # written once (dft_bytes_per_step), against the measured copy bandwidth
        hbm, hbm_src = hbm_peak()
        achieved = dft_bytes_per_step(plan) * args.steps / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "traffic": TRAFFIC_BYTES.get((args.precision, name)),
                    "traffic_unit": "bytes/launch", "peak_source": hbm_src,
                    "algorithmic_bytes_per_launch": dft_bytes_per_step(plan) / (launches / args.steps),
                    "per_kernel": per_kernel}
    else:
        achieved = flops / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
        peak, peak_src = PEAKS[args.precision]
        roofline = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": TRAFFIC_BYTES.get((args.precision, name)), "traffic_unit": "bytes/launch",
                    "peak_source": peak_src, "per_kernel": per_kernel}
    line = {
        "metric": METRIC, "value": maps / (total_ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded band-limited maps, the paper's random-signal protocol)",
        "config": {"workload": WORKLOAD, "L": L, "N": N, "lambda": LAM, "J0": J0, "spin": 0,
                   "maps_per_gpu": B, "precision": args.precision, "precompute": PRECOMPUTE.get(args.precision, 0),
                   "launch_shapes": None if args.no_autotune else [plan.launch_shapes(k) for k in range(plan.nscales + 2)],
                   "dft_forms": dft_forms,
                   "dft_forms_key": "per transform (SHT, scaling, scales) forward/inverse: 2 tensor-core "
                                    "prime-factor, 1 tensor-core direct, 0 SIMT",
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps (256 MB write)"},
        "precision_detail": PRECISION_DOC[args.precision],
        "max_rel_err": err,
        # precompute cost (outside the timed region, like the paper's precompute mode): plan
        # creation builds and slices the Wigner-d tables; the autotuner times launch shapes
        "plan": {"create_s": plan_create_s, "autotune_s": autotune_s, "table_bytes": table_bytes,
                 "workspace_bytes": workspace_bytes},
        "other_modes": other,
        "differentiation": diff,
        "ball": ball,
        "batching": batching,
        "samplings": samplings,
        "roofline": roofline,
        "clocks": clocks,
        "e2e": {"value": maps / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(f.numel() * 8),
                "d2h_bytes_per_step": int(f.numel() * 8), "max_rel_err": e2e_err},
        # per step: the contractions' kernels (contraction_kernels_per_step) and every
        # transform's forward and inverse DFT, with DFT_KERNELS[form] (forward, inverse) kernels
        "gpu_launches": int(args.steps * (contraction_kernels_per_step(args.precision, plan.nscales)
                                          + sum(DFT_KERNELS[fw][0] + DFT_KERNELS[iv][1] for fw, iv in dft_forms))),
    }
    if world == 1 and not args.no_cpu_baseline:
        dt, cerr = cpu_baseline_sample()
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": "1 map round trip (analysis + synthesis) of the same workload",
                                "seconds": dt, "max_rel_err": cerr}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_reference(args, world, rank):
    """The oracle (plain float64 CPU code) on this host's cores, same metric and workload;
    each step is a bounded sample of one map's round trip, within a ~150 s budget."""
    if rank != 0:
        return
    for _ in range(min(args.warmup, 1)):
        cpu_baseline_sample()
    times, errs = [], []
    t_start = time.perf_counter()
    for _ in range(args.steps):
        dt, e = cpu_baseline_sample()
        times.append(dt)
        errs.append(e)
        if time.perf_counter() - t_start > 150.0:
            break
    total = sum(times)
    value = len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": len(times), "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded band-limited maps)",
        "config": {"workload": WORKLOAD, "L": L, "N": N, "lambda": LAM, "J0": J0, "spin": 0,
                   "maps_per_step": 1, "precision": "fp64"},
        "max_rel_err": max(errs),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "1 map round trip per step (time-budgeted to ~150 s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_footprint():
    """Precompute cost of the float64-accurate tensor-core mode (the paper's precompute mode,
    Sec. 4.2): plan creation time and the device bytes of the sliced tables and workspaces for
    one real map at L in {64, 128, 256, 512} with N = 4 and N = 8 (lambda = 2, J0 = 2).  One JSON
    line; nothing is timed on the transforms."""
    import time

    import torch
    import paper_2402_01282_gb300 as s2w
    s2w.load()
    rows = []
    for n_dir in (4, 8):
        for Lf in (64, 128, 256, 512):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan = s2w.Plan(Lf, n_dir, 2.0, 2, reality=True, batch=1, precision=PRECISIONS["fp64_tc"])
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            tab, ws = plan.device_bytes()
            rows.append({"L": Lf, "N": n_dir, "create_s": dt, "table_bytes": tab, "workspace_bytes_1map": ws})
            plan.close()
    print(json.dumps({"footprint": "fp64_tc plans, one real map, lambda=2, J0=2", "plans": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the plain float64 path")
    ap.add_argument("--precision", default="fp64_tc", choices=sorted(PRECISIONS))
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiation-study timing")
    ap.add_argument("--no-ball", action="store_true", help="skip the ball-study timing")
    ap.add_argument("--no-batching", action="store_true", help="skip the batching-study timing")
    ap.add_argument("--no-sampling", action="store_true", help="skip the Driscoll-Healy timing")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--maps", type=int, default=B,
                    help="maps per GPU (default 16, the headline workload; smaller batches are for "
                         "profiler captures of single kernels, not bench lines)")
    ap.add_argument("--footprint", action="store_true",
                    help="only report plan creation time and table bytes of fp64_tc plans at L = 64..512")
    ap.add_argument("--ball-only", type=int, default=0, metavar="LP",
                    help="only run the ball study, at L = P = LP (128 is the study's size; smaller sizes are "
                         "for profiler captures of single kernels, not bench lines)")
    args = ap.parse_args()
    if args.footprint:
        run_footprint()
        return
    if args.ball_only:
        import torch
        import paper_2402_01282_gb300 as s2w
        s2w.load()
        globals().update(BALL_L=args.ball_only, BALL_P=args.ball_only)
        stream = torch.cuda.current_stream()
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        print(json.dumps(run_ball(torch, s2w, stream, flush, max(3, args.steps // 2), args.precision,
                                  not args.no_autotune)), flush=True)
        return
    if args.maps != B:
        globals()["B"] = args.maps
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
