#!/usr/bin/env python
"""Throughput of the seismic saliency hot path on GB300.

One step = one pass of the whole path over one synthetic volume resident in HBM:
K1 local spectra + projection + features, K2 directional center-surround, K3 normalisation
and combination (sal_local_spectra_project, sal_center_surround, sal_combine).

Prints one JSON line.  Multi-GPU (torchrun): every rank processes its own volume (the path
shards into independent volumes, no collective on the data path), the timed region is
bracketed by barriers and the max over ranks is taken; value = all voxels / that time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload salt128] [--impl ours|reference]
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

METRIC = "Mvoxel/s full saliency map (fwd, fwd+bwd), BF16-TC vs FP32 at stated error vs FP64"
WORKLOADS = {
    "salt128": dict(spec="salt128", n=16, desc="128x128x128 synthetic seismic volume (layered reflectivity, "
                    "30 Hz Ricker, 3 faults of random strike/dip with throw 2-8, salt ellipsoid 30/30/45 with "
                    "boundary reflector, folds amp 5 / wavelength 64, noise 0.1 rms), window 16^3, FP32",
                    cpu_sample=80, ref_sample=24),
    "fault48": dict(spec="fault48", n=8, desc="48^3 synthetic seismic volume (layers, one 60 deg normal fault "
                    "with throw 4, noise 0.1 rms), window 8^3, FP32", cpu_sample=48, ref_sample=32),
    "precision256x384x192": dict(spec="precision256x384x192", n=16, desc="256x384x192 synthetic seismic volume "
                                 "(6 faults, 2 salt bodies, SNR 5 dB), window 16^3, FP32", cpu_sample=48,
                                 ref_sample=24),
}
# Peak of the binding pipe of K1 (FP32 SIMT form): 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# K1 DRAM traffic per launch (bytes) from an ncu capture of the same kernel and workload;
# None until captured for the current kernel.
K1_TRAFFIC = {}


def k1_flops_per_voxel(n: int) -> int:
    """Algorithmic flops per voxel of the separable sliding local DFT (stages along t, x, y with
    h = n/2+1 retained t-bins): 4hn + 8hn^2 + 8hn^3."""
    h = n // 2 + 1
    return 4 * h * n + 8 * h * n * n + 8 * h * n ** 3


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


def cpu_oracle_rate(V, n, sample):
    """The FP64 oracle, as it stands, on a sample^3 corner sub-volume of the workload (all host cores)."""
    import numpy as np

    import oracle
    sub = np.ascontiguousarray(V[:sample, :sample, :sample])
    t0 = time.perf_counter()
    oracle.saliency(sub, n)
    dt = time.perf_counter() - t0
    return sub.size / dt / 1e6, dt, sub.shape


def run_reference(args, wl):
    """Reference arm: the FP64 oracle timed on the host cores (a deliberately slow baseline)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    V, _ = synth.volume(wl["spec"], with_mask=False)
    s = wl["ref_sample"]
    for _ in range(args.warmup):
        cpu_oracle_rate(V, wl["n"], s)
    times = []
    for _ in range(args.steps):
        _, dt, shape = cpu_oracle_rate(V, wl["n"], s)
        times.append(dt)
    vox = s ** 3
    value = vox * args.steps / sum(times) / 1e6
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mvoxel/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "n": wl["n"], "shape": list(V.shape), "precision": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": "Mvoxel/s", "cores": cores, "kind": "oracle",
                             "sample": f"{s}^3 corner sub-volume of the workload per step, full forward"},
            "e2e": {"value": value, "unit": "Mvoxel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="salt128", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
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

    V, _ = synth.volume(wl["spec"], with_mask=False)
    nvox = V.size
    params = sal.Params(n=wl["n"])
    eng = sal.Saliency(V.shape, params)
    dev = torch.device("cuda", local_rank)
    Vd = torch.from_numpy(V).to(dev)
    E = torch.empty((3,) + V.shape, dtype=torch.float32, device=dev)
    S3 = torch.empty_like(E)
    S = torch.empty(V.shape, dtype=torch.float32, device=dev)
    W = torch.empty(3, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    launches_per_step = 8  # K1, K2, K3: minmax3, minmax_finalize x2, weights, combine, normalize

    def step():
        sal.sal_local_spectra_project(eng.h, Vd, E)
        sal.sal_center_surround(eng.h, E, S3)
        sal.sal_combine(eng.h, S3, None, None, W, S)

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    dev_props = torch.cuda.get_device_properties(local_rank)
    gpu_id = str(getattr(dev_props, "uuid", "") or "")
    if gpu_id and not gpu_id.startswith("GPU-"):
        gpu_id = "GPU-" + gpu_id
    clocks = ClockSampler(gpu_id)
    clocks.start()
    barrier()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        a, b, c = evs[i]
        a.record()
        sal.sal_local_spectra_project(eng.h, Vd, E)
        b.record()
        sal.sal_center_surround(eng.h, E, S3)
        sal.sal_combine(eng.h, S3, None, None, W, S)
        c.record()
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(c) for a, b, c in evs)
    k1_ms = sum(a.elapsed_time(b) for a, b, c in evs)
    t = torch.tensor([total_ms, k1_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms, k1_ms = float(t[0]), float(t[1])
    value = world * nvox * args.steps / (total_ms / 1e3) / 1e6

    # end to end through the public fused call, host buffers, copies inside the timed region
    Vh = torch.from_numpy(V).pin_memory()
    Sh = torch.empty(V.shape, dtype=torch.float32).pin_memory()

    def e2e_step():
        Vd.copy_(Vh, non_blocking=True)
        sal.sal_saliency(eng.h, Vd, None, None, S, None, None, W)
        Sh.copy_(S, non_blocking=True)

    for _ in range(max(args.warmup, 3)):
        e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        e2e_step()
    e1.record()
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = world * nvox * args.steps / (float(t[0]) / 1e3) / 1e6

    n = wl["n"]
    k1_launch_s = k1_ms / 1e3 / args.steps
    achieved = k1_flops_per_voxel(n) * nvox / k1_launch_s / 1e12
    traffic = K1_TRAFFIC.get((args.workload, n, "fp32"))
    line = {
        "metric": METRIC, "value": value, "unit": "Mvoxel/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"], "n": n, "shape": list(V.shape), "precision": "fp32",
                   "form": "forward", "l2": "flushed between steps (256 MiB device write outside the events)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"kernel": "k1_spectra_f32", "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                     "peak_note": "FP32 FMA peak 152 SM x 128 lanes x 2 x 2.07 GHz (derived, not measured)",
                     "k1_ms_per_launch": k1_ms / args.steps, "k1_share_of_step": k1_ms / total_ms},
        "e2e": {"value": e2e_value, "unit": "Mvoxel/s", "h2d_bytes_per_step": V.nbytes,
                "d2h_bytes_per_step": V.nbytes},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "wall_s_timed": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = wl["cpu_sample"]
        rate, dt, shape = cpu_oracle_rate(V, n, s)
        line["cpu_baseline"] = {"value": rate, "unit": "Mvoxel/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{s}^3 corner sub-volume of the workload, full FP64 forward, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    eng.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
