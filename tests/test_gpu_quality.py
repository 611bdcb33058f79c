"""Reconstruction quality through the stream API (free-running recursion, 8-bit output against
the generator's ground truth, the paper's border rule).

Only properties that follow from the method are asserted: on translating content the past
frames' measured pixels, projected by motion compensation (Sec. 2.2) and checked (Sec. 3.1),
add samples that single-frame FSR does not have.  With a dynamic mask every pixel is measured
once in four frames (Sec. 1): under a (2, 1) pixel translation the source of a missing pixel is
measured in a given past frame with probability 1/4, so about 1 - (3/4)^3 = 58 % of the missing
pixels receive a projection from three past frames.  With a fixed mask the odd column shift
moves the sampling grid against the content.  The margins asserted are conservative bounds.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
from paper_2203_09200_gb300 import rfsr  # noqa: E402


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def mean_psnr(seq, first, **kw):
    import bench
    q = bench.quality_run(rfsr, seq, kw, with_ssim=False)
    return float(np.mean([p for p, _ in q[first:]]))


@pytest.mark.gpu
@pytest.mark.parametrize("mask_type,min_gain", [(synth.MASK_DYNAMIC, 1.0), (synth.MASK_FIXED, 0.5)])
def test_projection_beats_single_frame_fsr_on_translation(built, mask_type, min_gain):
    seq = synth.sinusoid_translation(96, 128, 12, seed=4, velocity=(2, 1), mask_type=mask_type)
    single = mean_psnr(seq, 4, num_refs=0, cc_mode="none")
    recursive = mean_psnr(seq, 4, cc_mode="nnc_frmc")
    assert recursive > single + min_gain, (single, recursive)


def test_quality_metrics_against_known_values():
    """PSNR and SSIM of the harness on closed-form cases (no GPU needed by the metrics)."""
    import bench
    a = np.full((64, 64), 100, np.uint8)
    b = a.copy()
    b[10, 10] = 110                      # one pixel off by 10 inside the border
    assert bench.psnr(a, a, 2) == 99.0
    mse = 100.0 / (60 * 60)
    assert abs(bench.psnr(b, a, 2) - 10 * np.log10(255.0 ** 2 / mse)) < 1e-9
    assert abs(bench.ssim(a, a, 2) - 1.0) < 1e-12
    rng = np.random.default_rng(0)
    x = rng.integers(0, 256, (64, 64)).astype(np.uint8)
    assert bench.ssim(x, 255 - x, 5) < 0.0   # anti-correlated content
