"""The FMA throughput probe that the rooflines' FP64 and FP32 pipe peaks come from: it runs,
computes what it says, and rejects what it does not support."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
F = pytest.importorskip("paper_1702_03818_gb300.frkc2")


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32x2"])
def test_fma_probe_values_and_rejections(prec):
    """The throughput probe writes one finite value per thread: the sum of its 8 chains after
    `iters` rounds x <- a x + b with a = 1 - 2^-20, b = 2^-10 (checked in FP64 on the host for
    the first thread); unknown precisions are rejected."""
    import math

    dt = torch.float64 if prec == "fp64" else torch.float32
    buf = torch.zeros(2 * 256, dtype=dt, device="cuda")
    iters = 64
    F.frkc2_fma_probe(prec, 2, iters, buf)
    torch.cuda.synchronize()
    a, b = 1.0 - 2.0 ** -20, 2.0 ** -10
    want = 0.0
    for i in range(8):
        x = i * 1e-3
        for _ in range(iters):
            x = x * a + b
        want += x
    got = buf.cpu().double()
    assert torch.isfinite(got).all()
    assert math.isclose(float(got[0]), want, rel_tol=1e-5 if dt == torch.float32 else 1e-12)
    with pytest.raises(F.Frkc2Error):
        F.frkc2_fma_probe("mixed", 2, iters, buf)
