"""The arithmetic-pipe microbenchmark that supplies the solve's roofline
denominators returns plausible GB300 figures: the FP32 FMA rate near the
152 SM x 128 lanes x 2 flops x clock of the part, FP64 far below it, and the
special-function unit's exp2 and reciprocal rates well below FP32 FMA."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_peaks_plausible():
    import paper_2011_14998_gb300 as mgx

    mgx.build()
    ctx = mgx.Context(0)
    try:
        p = mgx.mgx_alu_peaks(ctx.ptr, 2)
        with pytest.raises(mgx.MgxError):
            mgx.mgx_alu_peaks(ctx.ptr, 0)
    finally:
        ctx.close()
    print(p)
    assert 20.0 < p["fp32_fma_tflops"] < 100.0
    assert 0.1 < p["fp64_fma_tflops"] < 0.25 * p["fp32_fma_tflops"]
    for k in ("ex2_gops", "rcp_gops"):
        assert 100.0 < p[k] < 1e3 * p["fp32_fma_tflops"] / 2
