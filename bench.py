#!/usr/bin/env python
"""Throughput of the seismic saliency hot path on GB300.

One step = one pass of the whole path over one synthetic volume resident in HBM: the forward
(K1 local spectra + projection + features, K2 directional center-surround, K3 normalisation and
combination) and the backward of L = sum gS * S for a fixed seeded upstream gradient gS (the
combination adjoint, K4 center-surround adjoint, K5 spectral adjoint with brick recompute).

Prints one JSON line.  Multi-GPU (torchrun): every rank processes its own volume (the path
shards into independent volumes, no collective on the data path), the timed region is
bracketed by barriers and the max over ranks is taken; value = all voxels / that time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload full462x951x651] [--impl ours|reference]

The default workload is the full-scale volume (462 x 951 x 651, 286 M voxels, window 16^3, BF16
tensor-core local DFT): the largest configuration of the method that fits one GPU.
"""
import argparse
import json
import re
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mvoxel/s full saliency map (fwd, fwd+bwd), BF16-TC vs FP32 at stated error vs FP64"
WORKLOADS = {
    "salt128": dict(spec="salt128", n=16, desc="128x128x128 synthetic seismic volume (layered reflectivity, "
                    "30 Hz Ricker, 3 faults of random strike/dip with throw 2-8, salt ellipsoid 30/30/45 with "
                    "boundary reflector, folds amp 5 / wavelength 64, noise 0.1 rms), window 16^3",
                    cpu_sample=40, ref_sample=20),
    "fault48": dict(spec="fault48", n=8, desc="48^3 synthetic seismic volume (layers, one 60 deg normal fault "
                    "with throw 4, noise 0.1 rms), window 8^3", cpu_sample=48, ref_sample=32),
    "fault128": dict(spec="fault128", n=8, desc="128x128x128 synthetic seismic volume (layers, one 60 deg "
                     "normal fault with throw 4, noise 0.1 rms), window 8^3", cpu_sample=48, ref_sample=32),
    "precision256x384x192": dict(spec="precision256x384x192", n=16, desc="256x384x192 synthetic seismic volume "
                                 "(6 faults, 2 salt bodies, SNR 5 dB, folds), window 16^3", cpu_sample=40,
                                 ref_sample=20),
    "section462x951": dict(spec="section462x951", n=16, section=True, weights=(0.0, 0.5, 0.5),
                           directions=((0, 1, 0), (0, 0, 1), (0, 1, 1)),
                           desc="2-D vertical section 462 (t) x 951 (x) of a synthetic seismic slab (6 faults, 1 salt "
                           "body, folds, noise 0.1 rms), passed as a volume [1][462][951] (one plane), window 16^2, "
                           "the in-plane t, x, t-x window, weights (0, 1/2, 1/2)",
                           cpu_sample=256, ref_sample=80),   # one plane: sample x sample voxels
    "full462x951x651": dict(spec="full462x951x651", n=16, desc="config 5: 462x951x651 synthetic seismic volume "
                            "(20 faults, 3 salt bodies, 4 sinuous channels, folds, noise 0.1 rms), window 16^3",
                            cpu_sample=40, ref_sample=20, e2e_steps=10, side_steps=3),
}
DEFAULT_WORKLOAD = "full462x951x651"   # the largest configuration that fits one GPU
# Peaks of the ALU pipes, set by set_alu_peaks() from the device: the FP32 FMA pipe from its unit count
# (128 lanes per SM), the SM count of the device and its maximum SM clock; the MUFU pipe measured live
# (sal_measure_mufu_rate).  The values below are the nominal GB300 figures, used only until then.
PEAKS = {"sms": 152, "sm_ghz": 2.070, "fp32_tflops": 152 * 128 * 2 * 2.070e9 / 1e12,
         "fma_tops": 152 * 128 * 2.070e9 / 1e12, "mufu": {}, "mufu_note": "nominal 16/clk/SM (not measured)"}


def set_alu_peaks(sal, sms: int, sm_max_mhz):
    """FP32 FMA peak = SMs x 128 lanes x 2 flop x max SM clock (unit counts and clocks); MUFU peak =
    the measured issue rate of sqrt.approx / rsqrt.approx over the whole device."""
    ghz = (sm_max_mhz or 2070.0) / 1e3
    PEAKS.update(sms=sms, sm_ghz=ghz, fp32_tflops=sms * 128 * 2 * ghz * 1e9 / 1e12,
                 fma_tops=sms * 128 * ghz * 1e9 / 1e12)
    for op in ("sqrt", "rsqrt"):
        rate, _ = sal.sal_measure_mufu_rate(op)
        PEAKS["mufu"][op] = rate / 1e12
    # the tensor pipe's cost per MMA (M = 128, K = 16) at the widths the local-spectrum kernels issue
    PEAKS["mma_cycles"] = {nc: sal.sal_measure_mma_rate(nc)[0] for nc in (16, 32, 64)}
    PEAKS["mufu_note"] = (f"measured in this run: {op_rates()} (sal_measure_mufu_rate: 8 CTAs x 256 threads per SM, "
                          f"16 independent chains per thread); {sms} SMs")


def op_rates():
    return ", ".join(f"{k} {v:.3f} T/s ({v * 1e12 / (PEAKS['sms'] * PEAKS['sm_ghz'] * 1e9):.1f}/clk/SM at the max clock)"
                     for k, v in PEAKS["mufu"].items())
# K1 DRAM traffic per launch (bytes) from an ncu capture of the same kernel and workload;
# None until captured for the current kernel.
K1_TRAFFIC = {("salt128", 16, "fp32"): 8711168,   # sliding, 32-output form; profiles/salt128_n16_fp32_fwd_bwd.md
              ("salt128", 16, "bf16"): 8546816,   # profiles/salt128_n16_bf16_fwd_bwd.md (per launch)
              # one-pass capture of the full-scale launch (1.56 GB read + 3.39 GB written: ncu's 3-digit
              # figures); profiles/full462x951x651_n16_bf16_fwd_bwd.md
              ("full462x951x651", 16, "bf16"): 4950000000}
# K5 alone (the brick blocks it writes dominate): 34.7 MB read + 689.5 MB written per 128^3 launch of 16,384
# bricks (profiles/salt128_n16_bf16_fwd_bwd.md); a brick's traffic does not depend on the volume, so the
# full-scale call (2,254,098 bricks over its t-slab launches) is that per-brick figure times its bricks.
K5_TRAFFIC = {("salt128", 16, "bf16"): 724247040,
              ("full462x951x651", 16, "bf16"): 99641345482}


def measured_peaks():
    """Measured peaks of the GB300s, if present."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}



def bins_per_voxel(n: int) -> int:
    """abs(F) bins per voxel of the half spectrum (k_t in [0, n/2]): h n^2, one sqrt each."""
    return (n // 2 + 1) * n * n


def mma_per_brick(kind: str, n: int):
    """(MMAs per brick, N) of the tensor-core kernels at window n (8, 16), from their geometry: a brick is
    one t0, 128/n positions x0 and 16 outputs y0; stage 1 one MMA per 128 halo positions (24 x YP),
    per k_t tile stage 2 three K steps, stage 3 two per output; the adjoint adds per tile two adjoint-y
    MMAs per output, 16 adjoint-x MMAs and one t-adjoint MMA per 128 halo positions."""
    h = n // 2 + 1
    yp = 8 * -(-(16 + n - 1) // 8)
    nb1 = -(-(24 * yp) // 128)
    fwd = [(nb1, 16), (3 * h, 2 * yp), (32 * h, 2 * n)]
    return fwd if kind == "k1" else fwd + [(32 * h, 32), (16 * h, 64), (nb1 * h, 16)]


def tensor_issue(kind: str, n: int, shape, ms: float):
    """The tensor pipe's instruction floor of a tensor-core kernel: its MMAs per brick at the measured cost per
    MMA of each width (sal_measure_mma_rate; a width above 64 taken at the 64-column cost), the bricks spread
    evenly over the SMs at the max SM clock; frac = floor / measured time."""
    cyc = PEAKS.get("mma_cycles")
    if not cyc or n not in (8, 16):
        return None
    T, X, Y = shape
    bricks = -(-Y // 16) * -(-X // (128 // n)) * T
    per_brick = sum(c * cyc[min((w for w in cyc if w >= nc), default=64)] for c, nc in mma_per_brick(kind, n))
    floor_ms = bricks / PEAKS["sms"] * per_brick / (PEAKS["sm_ghz"] * 1e6)
    return {"mma_per_brick": sum(c for c, _ in mma_per_brick(kind, n)), "cycles_per_brick": per_brick,
            "cycles_per_mma": {str(k): round(v, 1) for k, v in cyc.items()}, "floor_ms": floor_ms,
            "frac": floor_ms / ms,
            "note": "tensor-pipe instruction rate measured in this run (sal_measure_mma_rate), bricks over the SMs"}


def roofline(kernel, prec, n, nvox, ms, flops_mult, traffic, mufu_op="sqrt", feature="abs", flops_per_voxel=None):
    """Roofline of a spectral kernel.  FP32 form: its contraction flops (the per-voxel figure
    4hn + 8hn^2 + 8hn^3, x2 for the adjoint; the sliding form's own count where it runs) on the FP32
    FMA pipe.  BF16/FP16 form: the
    contraction runs on the tensor cores (reported as `tensor`), and the binding pipe is the
    abs(F) epilogue, h n^2 square roots per voxel on the MUFU pipe; with the energy reading of the
    feature there is no root, and the epilogue's FP32 arithmetic (about 4 FMA-pipe operations per
    bin: |F|^2 and its share of the weighted sums) on the FMA pipe binds."""
    fpv = k1_flops_per_voxel(n) if flops_per_voxel is None else flops_per_voxel
    flops = flops_mult * fpv * nvox / (ms / 1e3) / 1e12
    fp32_note = (f"FP32 FMA peak {PEAKS['sms']} SM x 128 lanes x 2 x {PEAKS['sm_ghz']:.2f} GHz (unit counts and "
                 "the max SM clock)")
    if prec == "fp32":
        pk = PEAKS["fp32_tflops"]
        return {"kernel": kernel, "bound": "alu", "pipe": "fp32 fma", "achieved": flops, "peak": pk,
                "unit": "TFLOP/s", "frac": flops / pk, "traffic": traffic, "peak_note": fp32_note}
    bins = bins_per_voxel(n) * nvox / (ms / 1e3) / 1e12
    tpk = measured_peaks().get("bf16_tflops", 1900.0)
    tensor = {"achieved_tflops": flops, "peak_tflops": tpk, "frac": flops / tpk,
              "peak_note": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json); fp16 dense rate is equal"}
    if feature == "energy":
        ops = 4.0 * bins
        pk = PEAKS["fma_tops"]
        return {"kernel": kernel, "bound": "alu", "pipe": "FP32 FMA (energy epilogue: ~4 operations per bin)",
                "achieved": ops, "peak": pk, "unit": "Tops/s", "frac": ops / pk, "traffic": traffic,
                "peak_note": fp32_note.replace("x 2 x", "x"), "tensor": tensor}
    what = "abs(F) epilogue: one sqrt per bin" if mufu_op == "sqrt" else "Gamma epilogue: one rsqrt per bin"
    pk = PEAKS["mufu"].get(mufu_op, 16 * PEAKS["sms"] * PEAKS["sm_ghz"] * 1e9 / 1e12)
    return {"kernel": kernel, "bound": "alu", "pipe": f"MUFU ({what})", "achieved": bins,
            "peak": pk, "unit": f"T{mufu_op}/s", "frac": bins / pk, "traffic": traffic,
            "peak_note": PEAKS["mufu_note"], "tensor": tensor}


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise max of per-rank timings (the slowest rank bounds the job)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def job_throughput(world: int, voxels_per_rank: int, steps: int, max_ms: float) -> float:
    """Whole-job Mvoxel/s: every rank processes its own volume per step (weak scaling)."""
    return world * voxels_per_rank * steps / (max_ms / 1e3) / 1e6


def k1_flops_per_voxel(n: int) -> int:
    """Algorithmic flops per voxel of the separable sliding local DFT (stages along t, x, y with
    h = n/2+1 retained t-bins): 4hn + 8hn^2 + 8hn^3."""
    h = n // 2 + 1
    return 4 * h * n + 8 * h * n * n + 8 * h * n ** 3


def k1_flops_per_voxel_spatial(n: int, adjoint: bool = False) -> int:
    """Flops per voxel of the spatial reading's kernels: per window 9 n^2 line FFTs (forward: three passes
    of the forward transform, three of the two inverse transforms) or 18 n^2 (adjoint), each a radix-2 FFT
    of n points at 5 n log2 n flops."""
    lines = (18 if adjoint else 9) * n * n
    return lines * 5 * n * (n.bit_length() - 1)


# Outputs per thread of the FP32 K1's sliding form (rect taper, stride 1): the first of each run by the
# direct stage-3 sum, the others by the recursion.
K1_F32_SLIDING_RUN = {8: 8, 16: 16, 32: 8}


def k1_flops_per_voxel_sliding(n: int) -> int:
    """Algorithmic flops per voxel of the FP32 K1's sliding form: stages along t and x as in the direct
    form (4hn + 8hn^2); along y one complex add and one complex rotation per bin and output (8hn^2),
    and the direct sum (8hn^3) for one output of each run."""
    h = n // 2 + 1
    return 4 * h * n + 8 * h * n * n + 8 * h * n * n + 8 * h * n ** 3 // K1_F32_SLIDING_RUN[n]


K5_F32_SLIDING_RUN = {8: 4, 16: 8}   # outputs per thread run of the FP32 adjoint (its YC)


def k5_flops_per_voxel_sliding(n: int) -> int:
    """Algorithmic flops per voxel of the FP32 adjoint with both y-passes sliding (rect taper, n = 8, 16), run
    of r outputs per (k_t, k_x) row: the forward recompute (stages t, x; along y the direct sum for the
    run's first output and one complex multiply-add per bin for the others), then the adjoints of the three
    stages: along y per output one complex add per bin (the prefix sums) and, per run, r - 1 + n point
    evaluations of n bins (8n flops each); along x 8hn^2, along t 4hn."""
    h, r = n // 2 + 1, K5_F32_SLIDING_RUN[n]
    fwd = 4 * h * n + 8 * h * n * n + 8 * h * n * n + 8 * h * n ** 3 // r
    inv_y = h * n * (2 * n + 8 * n * (r - 1 + n) // r)
    return fwd + inv_y + 8 * h * n * n + 4 * h * n


def max_sm_clock_mhz(gpu_id):
    """The device's maximum SM clock (nvidia-smi clocks.max.sm), or None."""
    cmd = ["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"]
    if gpu_id:
        cmd += ["-i", gpu_id]
    try:
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=30).stdout.strip().splitlines()
        return float(out[0]) if out else None
    except (OSError, ValueError, subprocess.SubprocessError):
        return None


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_oracle_rate(V, n, sample, backward=True, feature="abs", stride=1, wl=None):  # noqa: C901
    """The FP64 oracle, as it stands, on a corner sub-volume of the workload, sample voxels per axis (a
    one-plane section: sample x sample), all host cores: forward, and the backward with the same fixed
    upstream gradient as the GPU step, with the workload's window and weights."""
    import numpy as np

    import oracle
    sub = np.ascontiguousarray(V[:sample, :sample, :sample])
    gS = _upstream(sub.shape)
    wl = wl or {}
    st = oracle.dcs_stencil(wl["directions"]) if "directions" in wl else None
    W = np.asarray(wl["weights"], np.float64) if "weights" in wl else np.full(3, 1.0 / 3.0)
    t0 = time.perf_counter()
    fwd = oracle.saliency(sub, n, stencil=st, weights=W if "weights" in wl else "equal", feature=feature,
                          stride=stride)
    if backward:
        oracle.saliency_backward(sub, n, W, gS, stencil=st, fwd=fwd, feature=feature, stride=stride)
    dt = time.perf_counter() - t0
    return sub.size / dt / 1e6, dt, sub.shape


def sampled_error(V, n, params, E, S3, count=48, seed=7):
    """Relative L2 error of the GPU's raw maps E_m and S_m against the FP64 oracle at seeded voxels
    (the oracle computes them one voxel at a time)."""
    import numpy as np

    import oracle
    import synth
    st = oracle.dcs_stencil(params.directions, params.R, params.sigma)
    pts = synth.sample_points(V.shape, count, seed=seed)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    if params.stride > 1:
        # stride s: the sampled voxels moved to the lattice, where E is the cube's own feature
        pts = (pts // params.stride) * params.stride
        Ec = oracle.features_at(V, pts, n, feature=params.feature)
        Eg = E.cpu().numpy()[:, pts[:, 0], pts[:, 1], pts[:, 2]].T.astype(np.float64)
        return {"voxels": count, "lattice": True, "E_rel_l2": [rel(Eg[:, m], Ec[:, m]) for m in range(3)]}
    Ec, Sc = oracle.center_surround_at(V, pts, n, st[0], st[3], feature=params.feature)
    Eg = E.cpu().numpy()[:, pts[:, 0], pts[:, 1], pts[:, 2]].T.astype(np.float64)
    Sg = S3.cpu().numpy()[:, pts[:, 0], pts[:, 1], pts[:, 2]].T.astype(np.float64)
    return {"voxels": count, "E_rel_l2": [rel(Eg[:, m], Ec[:, m]) for m in range(3)],
            "S_m_rel_l2": [rel(Sg[:, m], Sc[:, m]) for m in range(3)]}


def _workload_volume(wl):
    """The workload's volume; a section workload is the middle plane along y of its slab (t x x), passed
    as one plane [1][T][X] (its bricks and rows then run along the section's x)."""
    import numpy as np

    import synth
    # X slabs made in spawned processes (the generator is slab-invariant: same volume bit for bit)
    V, _ = synth.volume(wl["spec"], with_mask=False, workers=min(16, os.cpu_count() or 1))
    if wl.get("section"):
        V = np.ascontiguousarray(V[:, :, V.shape[2] // 2])[None]
    return V


def _upstream(shape):
    """Fixed seeded upstream gradient dL/dS of the backward half of a step."""
    import numpy as np
    return np.random.default_rng(12345).standard_normal(shape).astype(np.float32)


def run_reference(args, wl):
    """Reference arm: the FP64 oracle timed on the host cores (a deliberately slow baseline)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    V = _workload_volume(wl)
    s = wl["ref_sample"]
    bwd = getattr(args, "form", "fwdbwd") == "fwdbwd"
    for _ in range(args.warmup):
        cpu_oracle_rate(V, wl["n"], s, backward=bwd, feature=args.feature, stride=args.stride, wl=wl)
    times = []
    for _ in range(args.steps):
        _, dt, shape = cpu_oracle_rate(V, wl["n"], s, backward=bwd, feature=args.feature, stride=args.stride,
                                       wl=wl)
        times.append(dt)
    vox = int(np.prod(shape))
    value = vox * args.steps / sum(times) / 1e6
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mvoxel/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "n": wl["n"], "shape": list(V.shape), "precision": "fp64 oracle",
                       "form": "forward+backward" if bwd else "forward", "feature": args.feature,
                       "stride": args.stride},
            "cpu_baseline": {"value": value, "unit": "Mvoxel/s", "cores": cores, "kind": "oracle",
                             "sample": f"{'x'.join(map(str, shape))} corner sub-volume of the workload per step, "
                                       f"FP64 {'forward+backward' if bwd else 'forward'}"},
            "e2e": {"value": value, "unit": "Mvoxel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp16", "fp32"],
                    help="arithmetic of the local-DFT contraction (bf16/fp16: tensor cores)")
    ap.add_argument("--n", type=int, default=None, help="window side (overrides the workload's)")
    ap.add_argument("--form", default="fwdbwd", choices=["fwdbwd", "fwd"],
                    help="fwdbwd: forward + backward step (default); fwd: forward only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--feature", default="abs", choices=["abs", "energy", "spatial"],
                    help="E_m: mean of |F_m| (the paper's step 3), of |F_m|^2 (energy reading), or over the "
                         "cube of |IDFT(F_m)| (spatial reading: FP32, n <= 16)")
    ap.add_argument("--stride", type=int, default=1,
                    help="cubes at voxels whose indices are multiples of the stride (1 < stride < n/2)")
    ap.add_argument("--measure-peaks", action="store_true",
                    help="print the measured MUFU issue rates (the roofline denominators of the |F| epilogues) "
                         "and the tensor pipe's cost per MMA by width, and exit")
    args = ap.parse_args()
    if args.measure_peaks:
        import torch

        import paper_2201_06174_gb300 as sal
        props = torch.cuda.get_device_properties(0)
        set_alu_peaks(sal, props.multi_processor_count, max_sm_clock_mhz(""))
        mma = {str(nc): sal.sal_measure_mma_rate(nc)[0] for nc in (16, 32, 64, 128, 256)}
        print(json.dumps({"mufu_tops": PEAKS["mufu"], "sms": PEAKS["sms"], "sm_ghz": PEAKS["sm_ghz"],
                          "fp32_tflops": PEAKS["fp32_tflops"], "note": PEAKS["mufu_note"],
                          "mma_cycles_per_mma": mma,
                          "mma_note": "tcgen05.mma kind::f16, M = 128, K = 16, by N; back-to-back issue on every SM"}),
              flush=True)
        return
    wl = dict(WORKLOADS[args.workload])
    if args.n is not None:
        wl["n"] = args.n
        wl["desc"] = re.sub(r"window \d+\^3", f"window {args.n}^3", wl["desc"])
    if wl["n"] >= 32:  # the FP64 oracle costs 12 n^4 flop per voxel: keep its sample to ~30 s
        wl["cpu_sample"], wl["ref_sample"] = 16, 12
    if args.feature == "spatial":
        if args.prec != "fp32" or wl["n"] > 16 or args.stride != 1:
            ap.error("--feature spatial runs in FP32 with n <= 16 and stride 1")
        # the oracle's spatial reading goes one voxel at a time through numpy's FFTs
        wl["cpu_sample"], wl["ref_sample"] = min(wl["cpu_sample"], 16), min(wl["ref_sample"], 12)
    if args.impl == "reference":
        run_reference(args, wl)
        return

    import numpy as np
    import torch

    import paper_2201_06174_gb300 as sal
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    V = _workload_volume(wl)
    nvox = V.size
    params = sal.Params(n=wl["n"], prec=args.prec, feature=args.feature, stride=args.stride,
                        **({"directions": wl["directions"]} if "directions" in wl else {}))
    eng = sal.Saliency(V.shape, params)
    dev = torch.device("cuda", local_rank)
    Vd = torch.from_numpy(V).to(dev)
    gSd = torch.from_numpy(_upstream(V.shape)).to(dev)
    Wd = torch.tensor(wl.get("weights", (1.0 / 3.0,) * 3), dtype=torch.float32, device=dev)
    E = torch.empty((3,) + V.shape, dtype=torch.float32, device=dev)
    S3 = torch.empty_like(E)
    gS3 = torch.empty_like(E)
    gE = torch.empty_like(E)
    S = torch.empty(V.shape, dtype=torch.float32, device=dev)
    gV = torch.empty_like(S)
    W = torch.empty(3, dtype=torch.float32, device=dev)
    gW = torch.empty(3, dtype=torch.float32, device=dev)
    galpha = torch.empty(3, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    # one step: the forward (K1, K2, K3) and the backward of L = sum gS * S through the
    # stepwise public calls (combine adjoint, center-surround adjoint K4, spectral adjoint K5)
    calls = [
        ("k1_local_spectra_project", lambda: sal.sal_local_spectra_project(eng.h, Vd, E)),
        ("k2_center_surround", lambda: sal.sal_center_surround(eng.h, E, S3)),
        ("k3_combine", lambda: sal.sal_combine(eng.h, S3, None, Wd, W, S)),
        ("combine_backward", lambda: sal.sal_combine_backward(eng.h, S3, Wd, gSd, gS3, gW)),
        ("k4_center_surround_backward", lambda: sal.sal_center_surround_backward(eng.h, E, gS3, gE, galpha)),
        ("k5_local_spectra_project_backward", lambda: sal.sal_local_spectra_project_backward(eng.h, Vd, gE, gV)),
    ]

    if args.form == "fwd":
        calls = calls[:3]

    def step():
        for _, c in calls:
            c()

    dev_props = torch.cuda.get_device_properties(local_rank)
    gpu_id = str(getattr(dev_props, "uuid", "") or "")
    if gpu_id and not gpu_id.startswith("GPU-"):
        gpu_id = "GPU-" + gpu_id
    set_alu_peaks(sal, dev_props.multi_processor_count, max_sm_clock_mhz(gpu_id))
    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)] for _ in range(args.steps)]
    clocks = ClockSampler(gpu_id)
    clocks.start()
    barrier()
    launches0 = sal.sal_launch_count()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev = evs[i]
        ev[0].record()
        for j, (_, c) in enumerate(calls):
            c()
            ev[j + 1].record()
    barrier()
    wall = time.perf_counter() - wall0
    launches = sal.sal_launch_count() - launches0
    clk = clocks.stop()
    per_call = [sum(ev[j].elapsed_time(ev[j + 1]) for ev in evs) for j in range(len(calls))]
    total_ms = sum(per_call)
    red = max_over_ranks([total_ms] + per_call, dist, dev)
    total_ms, per_call = red[0], red[1:]
    fwd_ms = sum(per_call[:3])
    value = job_throughput(world, nvox, args.steps, total_ms)

    # end to end through the fused public calls, host buffers, copies inside the timed region
    Vh = torch.from_numpy(V).pin_memory()
    gSh = torch.from_numpy(_upstream(V.shape)).pin_memory()
    Sh = torch.empty(V.shape, dtype=torch.float32).pin_memory()
    gVh = torch.empty(V.shape, dtype=torch.float32).pin_memory()

    # (a) the forward as one call that also returns its intermediates, the backward through the
    # per-step adjoint calls that take them (each step computed once); (b) the fused backward call,
    # which recomputes the forward from V by itself
    def e2e_step(fused_backward=False):
        Vd.copy_(Vh, non_blocking=True)
        if args.form == "fwdbwd":
            gSd.copy_(gSh, non_blocking=True)
        sal.sal_saliency(eng.h, Vd, None, Wd, S, S3, E, W)
        if args.form == "fwdbwd":
            if fused_backward:
                sal.sal_saliency_backward(eng.h, Vd, Wd, gSd, gV, gW, galpha)
            else:
                sal.sal_combine_backward(eng.h, S3, Wd, gSd, gS3, gW)
                sal.sal_center_surround_backward(eng.h, E, gS3, gE, galpha)
                sal.sal_local_spectra_project_backward(eng.h, Vd, gE, gV)
        Sh.copy_(S, non_blocking=True)
        if args.form == "fwdbwd":
            gVh.copy_(gV, non_blocking=True)

    # the end-to-end and side measurements of a large workload take fewer steps than the headline
    e2e_steps = min(args.steps, wl.get("e2e_steps", args.steps))
    side_steps = min(args.steps, wl.get("side_steps", args.steps))

    def e2e_rate(fused_backward, steps):
        for _ in range(3):
            e2e_step(fused_backward)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            e2e_step(fused_backward)
        e1.record()
        barrier()
        ms = max_over_ranks([e0.elapsed_time(e1)], dist, dev)[0]
        return job_throughput(world, nvox, steps, ms)

    # (c) the calls of (a) with the copies overlapped: inputs and results double-buffered on the device; step
    # i + 1's inputs are copied in (one copy stream) and step i's results read back (another) while step i
    # computes.  Every step still copies its V (and gS) in and its S (and gV) out inside the timed region.
    def e2e_overlapped_rate(steps):
        comp = torch.cuda.current_stream()
        h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
        Vb, gSb = [Vd, torch.empty_like(Vd)], [gSd, torch.empty_like(gSd)]
        Sb, gVb = [S, torch.empty_like(S)], [gV, torch.empty_like(gV)]

        def compute(b):
            sal.sal_saliency(eng.h, Vb[b], None, Wd, Sb[b], S3, E, W)
            if args.form == "fwdbwd":
                sal.sal_combine_backward(eng.h, S3, Wd, gSb[b], gS3, gW)
                sal.sal_center_surround_backward(eng.h, E, gS3, gE, galpha)
                sal.sal_local_spectra_project_backward(eng.h, Vb[b], gE, gVb[b])

        def run(nsteps):
            loaded = [torch.cuda.Event() for _ in range(2)]   # the buffer's inputs are on the device
            done = [torch.cuda.Event() for _ in range(2)]     # the buffer's step has computed
            read = [torch.cuda.Event() for _ in range(2)]     # the buffer's results are read back
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

            def load(b):
                with torch.cuda.stream(h2d):
                    Vb[b].copy_(Vh, non_blocking=True)
                    if args.form == "fwdbwd":
                        gSb[b].copy_(gSh, non_blocking=True)
                    loaded[b].record(h2d)

            e0.record(comp)
            h2d.wait_event(e0)
            for b in range(min(2, nsteps)):
                load(b)
            for i in range(nsteps):
                b = i & 1
                comp.wait_event(loaded[b])
                if i >= 2:
                    comp.wait_event(read[b])     # step i - 2's results left this buffer
                compute(b)
                done[b].record(comp)
                with torch.cuda.stream(d2h):
                    d2h.wait_event(done[b])
                    Sh.copy_(Sb[b], non_blocking=True)
                    if args.form == "fwdbwd":
                        gVh.copy_(gVb[b], non_blocking=True)
                    read[b].record(d2h)
                if i + 2 < nsteps:
                    h2d.wait_event(done[b])      # step i no longer reads this buffer's inputs
                    load(b)
            comp.wait_stream(d2h)
            e1.record(comp)
            return e0, e1

        run(min(3, steps))
        barrier()
        e0, e1 = run(steps)
        barrier()
        ms = max_over_ranks([e0.elapsed_time(e1)], dist, dev)[0]
        del Vb[1], gSb[1], Sb[1], gVb[1]
        return job_throughput(world, nvox, steps, ms)

    e2e_serial_value = e2e_rate(False, e2e_steps)
    e2e_value = e2e_overlapped_rate(e2e_steps)
    e2e_fused_value = e2e_rate(True, side_steps) if args.form == "fwdbwd" else None
    S_prec = S.clone()   # the map of this precision form, weights Wd (from the last e2e step's forward)

    # the plain FP32 form of K1 on the same volume (forward comparison of the precision forms)
    k1_fp32_ms = None
    s_vs_fp32 = None
    if args.prec != "fp32":
        eng32 = sal.Saliency(V.shape, sal.Params(n=wl["n"], prec="fp32", feature=args.feature, stride=args.stride,
                                                 **({"directions": wl["directions"]} if "directions" in wl else {})))
        E32 = torch.empty_like(E)
        for _ in range(3):
            sal.sal_local_spectra_project(eng32.h, Vd, E32)
        barrier()
        tot = 0.0
        for i in range(side_steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            sal.sal_local_spectra_project(eng32.h, Vd, E32)
            b.record()
            b.synchronize()
            tot += a.elapsed_time(b)
        k1_fp32_ms = tot / side_steps
        # the map of the FP32 form (oracle-pinned) with the same weights, against this form's map
        S32 = torch.empty_like(S)
        sal.sal_saliency(eng32.h, Vd, None, Wd, S32, None, None, W)
        torch.cuda.synchronize()
        dS = (S_prec.double() - S32.double())
        s_vs_fp32 = {"max_abs": float(dS.abs().max()), "rel_l2": float(dS.norm() / S32.double().norm()),
                     "voxels": nvox, "what": "normalised [0,1] map S of this form against the FP32 form's S, "
                                              "every voxel, same weights"}
        del E32, S32, dS
        eng32.close()

    n = wl["n"]
    names = [c[0] for c in calls]
    # dominant kernel: K5 (spectral adjoint with brick recompute, incl. its overlap-add gather);
    # K1 in the forward-only form
    k1_ms = per_call[names.index("k1_local_spectra_project")] / args.steps
    tag = "tc" if args.prec != "fp32" else "f32"
    trk = (args.workload, n, args.prec) if args.feature == "abs" and args.stride == 1 else None
    # cubes the K1 launch computes: every voxel at stride 1; with stride s the tensor-core form computes
    # the whole lattice planes t = k s, the FP32 form only the lattice
    sc = args.stride
    T_, X_, Y_ = V.shape
    ncubes = nvox if sc == 1 else (-(-T_ // sc) * X_ * Y_ if args.prec != "fp32" else
                                   -(-T_ // sc) * -(-X_ // sc) * -(-Y_ // sc))
    spatial = args.feature == "spatial"
    sliding = args.prec == "fp32" and sc == 1 and n in K1_F32_SLIDING_RUN and not spatial
    k1_rl = roofline("k1_spatial_f32" if spatial else f"k1_spectra_{tag}", args.prec, n, ncubes, k1_ms, 1,
                     K1_TRAFFIC.get(trk), feature=args.feature,
                     flops_per_voxel=(k1_flops_per_voxel_spatial(n) if spatial else
                                      k1_flops_per_voxel_sliding(n) if sliding else None))
    if sliding:
        k1_rl["form"] = "sliding DFT along y (flops of that form)"
    if spatial:
        k1_rl["form"] = "spatial reading: per-window separable radix-2 FFTs in shared memory (flops of that form)"
    if sc > 1:
        k1_rl["cubes_per_launch"] = ncubes
    if args.prec != "fp32" and sc == 1 and not spatial and n in (8, 16):
        k1_rl["tensor_issue"] = tensor_issue("k1", n, V.shape, k1_ms)
    if args.form == "fwdbwd":
        k5_ms = per_call[names.index("k5_local_spectra_project_backward")] / args.steps
        # the timed call is memset + K5 + the overlap-add gather; the traffic entry is K5's own
        # the FP32 adjoint at n = 8, 16 runs both y-passes as sliding recursions (k5_flops_per_voxel_sliding);
        # otherwise its flops are twice the direct forward's
        k5_sliding = args.prec == "fp32" and n in K5_F32_SLIDING_RUN and not spatial
        k5_name = "k5_spatial_adjoint_f32" if spatial else f"k5_spectra_adjoint_{tag}"
        rl = roofline(f"{k5_name} (call incl. memset and the two overlap-add passes)", args.prec, n, nvox, k5_ms,
                      1 if k5_sliding or spatial else 2, K5_TRAFFIC.get(trk),
                      mufu_op="rsqrt" if args.prec != "fp32" else "sqrt", feature=args.feature,
                      flops_per_voxel=(k1_flops_per_voxel_spatial(n, adjoint=True) if spatial else
                                       k5_flops_per_voxel_sliding(n) if k5_sliding else None))
        if spatial:
            rl["form"] = "spatial reading's adjoint: forward recompute, signs, combined inverse (flops of that form)"
        if k5_sliding:
            rl["form"] = "forward recompute and inverse along y by sliding recursions (flops of that form)"
        if args.prec != "fp32" and sc == 1 and n in (8, 16) and not spatial:
            rl["tensor_issue"] = tensor_issue("k5", n, V.shape, k5_ms)
        rl["k1"] = k1_rl
    else:
        rl = k1_rl
    line = {
        "metric": METRIC, "value": value, "unit": "Mvoxel/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"bf16": "bf16", "fp16": "f16", "fp32": "f32"}[args.prec], "data": "synthetic",
        "config": {"workload": wl["desc"], "n": n, "shape": list(V.shape),
                   "precision": args.prec + (" tensor-core local DFT (FP32 accumulate); the adjoint's "
                                             "tensor-core operands are FP16" if args.prec != "fp32" else " SIMT"),
                   "form": "forward+backward (upstream gradient fixed, seeded)" if args.form == "fwdbwd"
                   else "forward",
                   "feature": {"abs": "mean of |F_m| (step 3)", "energy": "mean of |F_m|^2 (energy reading)",
                               "spatial": "mean over the cube of |IDFT(F_m)| (spatial reading)"}[args.feature],
                   "stride": args.stride,
                   "l2": "flushed between steps (256 MiB device write outside the events)",
                   "parallelism": f"replicas x{world}"},
        "forward": {"value": world * nvox * args.steps / (fwd_ms / 1e3) / 1e6, "unit": "Mvoxel/s",
                    "ms_per_step": fwd_ms / args.steps},
        "ms_per_call": {nm: v / args.steps for nm, v in zip(names, per_call)},
        "k1_vs_fp32": None if k1_fp32_ms is None else {
            "k1_ms": k1_ms, "k1_fp32_ms": k1_fp32_ms, "speedup": k1_fp32_ms / k1_ms, "fp32_steps": side_steps,
            "forward_fp32_Mvoxel_s": world * nvox / ((k1_fp32_ms + sum(per_call[1:3]) / args.steps) / 1e3) / 1e6},
        "roofline": rl,
        "max_abs_S": None if s_vs_fp32 is None else s_vs_fp32["max_abs"],
        "S_vs_fp32": s_vs_fp32,
        "e2e": {"value": e2e_value, "unit": "Mvoxel/s", "steps": e2e_steps,
                "h2d_bytes_per_step": (2 if args.form == "fwdbwd" else 1) * V.nbytes,
                "d2h_bytes_per_step": (2 if args.form == "fwdbwd" else 1) * V.nbytes,
                "calls": "sal_saliency (with E, S3 out)" + (" + sal_combine_backward + sal_center_surround_backward + "
                                                            "sal_local_spectra_project_backward"
                                                            if args.form == "fwdbwd" else ""),
                "copies": "overlapped with compute: inputs and results double-buffered on the device, the next "
                          "step's inputs copied in and this step's results read back on two copy streams",
                "serial_value": e2e_serial_value,
                "fused_backward_value": e2e_fused_value, "fused_backward_steps": side_steps},
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s_timed": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = wl["cpu_sample"]
        rate, dt, shape = cpu_oracle_rate(V, n, s, backward=args.form == "fwdbwd", feature=args.feature,
                                          stride=args.stride, wl=wl)
        line["cpu_baseline"] = {"value": rate, "unit": "Mvoxel/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{'x'.join(map(str, shape))} corner sub-volume of the workload, FP64 "
                                          f"{'forward+backward' if args.form == 'fwdbwd' else 'forward'}, {dt:.1f} s",
                                "sampled_error_vs_fp64": sampled_error(V, n, params, E, S3)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    eng.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
