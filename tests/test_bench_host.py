"""Host-side logic of bench.py that needs no GPU: the roofline's choice of
bound per kernel group and workload, and the traffic lookup."""
import bench
from synth import config_c2, config_c3

PEAKS = {"hbm_gbs": 7000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1700.0}


def stats(name, ms=10.0, launches=10, work=1e12, is_bytes=False):
    return {name: {"total_ms": ms, "launches": launches, "work": work, "is_bytes": is_bytes}}


def test_tensor_core_taylor_is_rated_against_tf32():
    r = bench.roofline_for(stats("propagate"), "tf32x3", PEAKS, "measured", config_c2(), "c2")
    assert r["bound"] == "tensor"
    assert r["peak"] == 850.0
    # 1e12 flops per 1 ms launch
    assert r["achieved"] == 1000.0
    assert r["traffic"] is not None       # the committed C2 capture


def test_cuda_core_taylor_is_rated_against_fp32():
    r = bench.roofline_for(stats("propagate"), "tf32x3", PEAKS, "measured", config_c3(), "c3",
                           taylor_fused=0)
    assert r["bound"] == "alu"
    assert r["peak"] == round(bench.FP32_SIMT_TFLOPS, 3)


def test_streamed_tensor_core_taylor_above_m64_is_rated_against_tf32():
    r = bench.roofline_for(stats("propagate"), "tf32x3", PEAKS, "measured", config_c3(), "c3",
                           taylor_fused=3)
    assert config_c3().M > 64
    assert r["bound"] == "tensor" and r["peak"] == 850.0


def test_bf16x3_propagation_is_rated_against_bf16():
    r = bench.roofline_for(stats("propagate"), "bf16x3", PEAKS, "measured", config_c2(), "c2",
                           taylor_fused=1)
    assert r["bound"] == "tensor" and r["peak"] == 1700.0
    r = bench.roofline_for(stats("one_body"), "bf16x3", PEAKS, "measured", config_c2(), "c2",
                           taylor_fused=1)
    assert r["peak"] == 850.0             # TF32X3 contractions


def test_small_matrix_kernels_are_rated_against_fp32():
    r = bench.roofline_for(stats("overlap"), "tf32x3", PEAKS, "measured", config_c2(), "c2")
    assert r["bound"] == "alu"
    assert r["traffic"] == bench.lookup_traffic("overlap", "tf32x3", "c2")


def test_block_diagonal_series_is_rated_against_fp32():
    r = bench.roofline_for(stats("propagate"), "bf16x3", PEAKS, "measured", config_c3(), "c3",
                           taylor_fused=4)
    assert r["bound"] == "alu"
