"""Host arithmetic of the benchmark's roofline: the algorithmic work per voxel of each form of the local
DFT and the fractions reported against the peaks (no GPU)."""
import pytest

import bench


@pytest.mark.parametrize("n,flops", [(8, 23_200), (16, 313_920), (32, 4_597_888)])
def test_direct_dft_flops_per_voxel(n, flops):
    """4hn + 8hn^2 + 8hn^3 (h = n/2 + 1 retained t-bins): real input along t, complex along x and y."""
    assert bench.k1_flops_per_voxel(n) == flops


@pytest.mark.parametrize("n", [8, 16, 32])
def test_sliding_form_flops_per_voxel(n):
    """Stages along t and x as in the direct form, 8 flops per bin and output along y, and the direct
    stage-3 sum once per run of outputs: below the direct count, above the stages along t and x."""
    h = n // 2 + 1
    run = bench.K1_F32_SLIDING_RUN[n]
    tx = 4 * h * n + 8 * h * n * n
    assert bench.k1_flops_per_voxel_sliding(n) == tx + 8 * h * n * n + 8 * h * n ** 3 // run
    assert tx < bench.k1_flops_per_voxel_sliding(n) < bench.k1_flops_per_voxel(n)


@pytest.mark.parametrize("n,flops", [(8, 20_800), (16, 150_912)])
def test_sliding_adjoint_flops_per_voxel(n, flops):
    """The FP32 adjoint with both y-passes sliding, counted by hand at n = 16 (h = 9, runs of 8 outputs):
    forward 576 + 18432 + 18432 + 36864; inverse along y 144 (32 + 8 16 23 / 8); along x 18432, along t 576.
    Below the cost of two direct forward passes, which it replaces."""
    assert bench.k5_flops_per_voxel_sliding(n) == flops
    assert bench.k5_flops_per_voxel_sliding(n) < 2 * bench.k1_flops_per_voxel(n)


def test_bins_per_voxel():
    assert [bench.bins_per_voxel(n) for n in (8, 16, 32)] == [320, 2304, 17408]


def test_fp32_roofline_fraction():
    n, nvox, ms = 16, 128 ** 3, 8.0
    rl = bench.roofline("k", "fp32", n, nvox, ms, 1, 123)
    achieved = bench.k1_flops_per_voxel(n) * nvox / (ms / 1e3) / 1e12
    assert rl["achieved"] == pytest.approx(achieved)
    assert rl["frac"] == pytest.approx(achieved / bench.PEAKS["fp32_tflops"])
    assert rl["unit"] == "TFLOP/s" and rl["traffic"] == 123 and rl["bound"] == "alu"
    sl = bench.roofline("k", "fp32", n, nvox, ms, 1, None, flops_per_voxel=bench.k1_flops_per_voxel_sliding(n))
    assert sl["achieved"] == pytest.approx(achieved * bench.k1_flops_per_voxel_sliding(n) / bench.k1_flops_per_voxel(n))


def test_tensor_form_roofline_is_the_mufu_epilogue():
    n, nvox, ms = 16, 128 ** 3, 2.7
    rl = bench.roofline("k", "bf16", n, nvox, ms, 1, None)
    bins = bench.bins_per_voxel(n) * nvox / (ms / 1e3) / 1e12
    nominal = 16 * bench.PEAKS["sms"] * bench.PEAKS["sm_ghz"] * 1e9 / 1e12   # before a measured rate is set
    assert rl["achieved"] == pytest.approx(bins) and rl["peak"] == pytest.approx(nominal)
    assert rl["frac"] == pytest.approx(bins / nominal)
    assert "tensor" in rl and rl["tensor"]["frac"] == pytest.approx(rl["tensor"]["achieved_tflops"] /
                                                                     rl["tensor"]["peak_tflops"])
    en = bench.roofline("k", "bf16", n, nvox, ms, 1, None, feature="energy")
    assert en["peak"] == bench.PEAKS["fma_tops"] and en["achieved"] == pytest.approx(4 * bins)


def test_peaks_derived_from_unit_counts_and_the_measured_mufu_rate(monkeypatch):
    """The FP32 peak follows the device's SM count and max clock; the MUFU peak is the measured rate."""
    monkeypatch.setattr(bench, "PEAKS", dict(bench.PEAKS, mufu={}))

    class FakeSal:
        @staticmethod
        def sal_measure_mufu_rate(op):
            return (5.5e12 if op == "sqrt" else 6.0e12), 150

        @staticmethod
        def sal_measure_mma_rate(nc):
            return {16: 44.0, 32: 44.0, 64: 48.0}[nc], 150
    bench.set_alu_peaks(FakeSal, 150, 2000.0)
    assert bench.PEAKS["fp32_tflops"] == pytest.approx(150 * 128 * 2 * 2.0e9 / 1e12)
    assert bench.PEAKS["fma_tops"] == pytest.approx(bench.PEAKS["fp32_tflops"] / 2)
    assert bench.PEAKS["mufu"] == {"sqrt": pytest.approx(5.5), "rsqrt": pytest.approx(6.0)}
    rl = bench.roofline("k", "bf16", 16, 128 ** 3, 2.0, 1, None, mufu_op="rsqrt")
    assert rl["peak"] == pytest.approx(6.0) and "measured" in rl["peak_note"]


def test_reference_arm_on_a_section_counts_its_plane_and_uses_its_window(monkeypatch, capsys):
    """The oracle is timed on the workload's own configuration: a one-plane section sample has
    sample^2 voxels, and runs with the section's in-plane window and weights."""
    import json

    import numpy as np

    import oracle
    calls = []
    real_saliency, real_backward = oracle.saliency, oracle.saliency_backward

    def saliency(V, n, **kw):
        calls.append(("fwd", V.shape, kw.get("stencil"), kw.get("weights")))
        return real_saliency(V, n, **kw)

    def saliency_backward(V, n, W, gS, **kw):
        calls.append(("bwd", V.shape, kw.get("stencil"), W))
        return real_backward(V, n, W, gS, **kw)
    monkeypatch.setattr(oracle, "saliency", saliency)
    monkeypatch.setattr(oracle, "saliency_backward", saliency_backward)
    monkeypatch.setenv("RANK", "0")
    wl = dict(bench.WORKLOADS["section462x951"], ref_sample=20)
    monkeypatch.setattr(bench, "_workload_volume", lambda w: np.random.default_rng(0).standard_normal(
        (1, 40, 50)).astype(np.float32))

    class A:
        steps, warmup, gpus, feature, stride, form = 1, 0, 1, "abs", 1, "fwdbwd"
    bench.run_reference(A(), wl)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["cpu_baseline"]["sample"].startswith("1x20x20 ")
    assert line["value"] * line["ms_per_step"] / 1e3 * 1e6 == pytest.approx(400)
    expect = oracle.dcs_stencil(wl["directions"])
    for kind, shape, st, W in calls:
        assert shape == (1, 20, 20)
        assert np.array_equal(st[0], expect[0]) and np.allclose(st[3], expect[3])
        assert np.allclose(W, [0.0, 0.5, 0.5])
    assert [c[0] for c in calls] == ["fwd", "bwd"]


def test_spatial_reading_flops_and_guard():
    """The spatial reading's kernels: 9 n^2 (forward) or 18 n^2 (adjoint) radix-2 line FFTs of 5 n log2 n
    flops per window; the bench runs them only in the form the library provides."""
    import subprocess
    import sys
    assert [bench.k1_flops_per_voxel_spatial(n) for n in (2, 4, 8, 16)] == [360, 5760, 69120, 737280]
    assert bench.k1_flops_per_voxel_spatial(16, adjoint=True) == 2 * 737280
    r = subprocess.run([sys.executable, bench.__file__, "--feature", "spatial", "--prec", "bf16", "--form", "fwd",
                        "--workload", "fault48"], capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "--feature spatial runs in FP32" in r.stderr


def test_tensor_issue_floor_counts_the_kernels_mmas(monkeypatch):
    """The MMA counts per brick follow the kernels' geometry (n = 16: 6 stage-1 MMAs, per k_t tile 3 stage-2
    and 32 stage-3 MMAs, the adjoint 32 + 16 + 6 more), and the floor spreads the bricks over the SMs."""
    monkeypatch.setattr(bench, "PEAKS", dict(bench.PEAKS, sms=100, sm_ghz=2.0, mma_cycles={16: 40.0, 32: 40.0, 64: 50.0}))
    assert sum(c for c, _ in bench.mma_per_brick("k1", 16)) == 6 + 9 * 35
    assert sum(c for c, _ in bench.mma_per_brick("k5", 16)) == 6 + 9 * 89
    ti = bench.tensor_issue("k5", 16, (100, 80, 160), 10.0)
    bricks = 10 * 10 * 100
    cyc = 6 * 40 + 9 * (3 * 50 + 32 * 40 + 32 * 40 + 16 * 50 + 6 * 40)
    assert ti["cycles_per_brick"] == cyc
    assert ti["floor_ms"] == pytest.approx(bricks / 100 * cyc / 2.0e6)
    assert ti["frac"] == pytest.approx(ti["floor_ms"] / 10.0)
