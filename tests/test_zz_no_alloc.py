"""The allocation-free entry point, rfsr_me_cc_project_noalloc.

It serves callers that cannot allocate device memory while they run (real-time loops, plugins in
applications that own all of the GPU's memory, code that may not allocate after start-up): all
its intermediate planes live in one fixed array of the library's static device memory, and the
caller passes only inputs and outputs.  This test calls it through the C ABI twice in a row --
the second call runs on the scratch contents the first left behind -- and checks that both
calls give exactly the projection sums, counts and decision labels of the regular stream path
for the same inputs (integer results, so the tolerance is zero).  It also checks one call against
the CPU oracle directly, and that a frame with a bad mask leaves every output but the status word
as it was.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2203_09200_gb300 import rfsr  # noqa: E402


@pytest.fixture(autouse=True, scope="module")
def built():
    """The library (and the oracle) built in-tree, also when this file runs alone."""
    if torch.cuda.is_available():
        import __graft_entry__
        __graft_entry__.build()


def stream_path(eng, smp, msk, hist, **cfg):
    H, W = smp.shape
    st = eng.create_stream(height=H, width=W, **cfg)
    try:
        st.set_history(hist)
        st.push_frame(smp, msk)
        st.get_frame(timeout_ms=120000)
        dec = [st.debug_get(rfsr.DBG_DECISION, k) for k in range(1, len(hist) + 1)]
        return st.debug_get(rfsr.DBG_PSUM), st.debug_get(rfsr.DBG_PCNT), dec
    finally:
        st.destroy()


def test_noalloc_matches_stream_path_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    H, W = 480, 640                       # the largest frame that fits with three past frames
    seq = synth.config2(seed=77, H=H, W=W, F=6)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    cfg = dict(cc_mode="nnc_frmc", template_size=9, search_radius=8)
    eng = rfsr.Engine(device=0)
    try:
        for t in (4, 5):                  # two calls in a row on the same scratch
            smp, msk = seq.samples[t], seq.masks[t]
            hist = [(seq.frames[t - k], seq.samples[t - k], seq.masks[t - k]) for k in (1, 2, 3)]
            ref_psum, ref_pcnt, ref_dec = stream_path(eng, smp, msk, hist, **cfg)
            refs = [(dev(r), dev(s), dev(m)) for r, s, m in hist]
            d_psum = torch.full((H, W), -1, dtype=torch.int16, device="cuda")
            d_pcnt = torch.full((H, W), 255, dtype=torch.uint8, device="cuda")
            d_dec = torch.full((3, H, W), 255, dtype=torch.uint8, device="cuda")
            d_status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            stream = torch.cuda.current_stream()
            rfsr.me_cc_project_noalloc(dev(smp), dev(msk), refs, d_psum, d_pcnt, H, W,
                                       d_dec=d_dec, d_status=d_status,
                                       cuda_stream=stream.cuda_stream, **cfg)
            stream.synchronize()
            assert int(d_status.item()) == 0
            np.testing.assert_array_equal(d_psum.cpu().numpy().view(np.uint16), ref_psum)
            np.testing.assert_array_equal(d_pcnt.cpu().numpy(), ref_pcnt)
            got_dec = d_dec.cpu().numpy()
            for k in range(3):
                np.testing.assert_array_equal(got_dec[k], ref_dec[k])
            assert ref_pcnt.any()         # the frames do project something
    finally:
        eng.destroy()


def test_noalloc_rejects_frames_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    H, W = 1080, 1920
    z8 = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    z16 = torch.zeros((H, W), dtype=torch.int16, device="cuda")
    with pytest.raises(rfsr.RfsrError) as e:
        rfsr.me_cc_project_noalloc(z8, z8, [(z8, z8, z8)] * 3, z16, z8, H, W)
    assert e.value.code == rfsr.RFSR_EINVAL
    assert "bytes of scratch" in str(e.value)


def run_noalloc(smp, msk, hist, H, W, fill=None, **cfg):
    """One call on device copies of the inputs; returns (status, psum, pcnt, dec) on the host."""
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    refs = [(dev(r), dev(s), dev(m)) for r, s, m in hist]
    K = len(hist)
    outs = fill if fill is not None else (
        torch.full((H, W), -1, dtype=torch.int16, device="cuda"),
        torch.full((H, W), 255, dtype=torch.uint8, device="cuda"),
        torch.full((max(1, K), H, W), 255, dtype=torch.uint8, device="cuda"))
    d_psum, d_pcnt, d_dec = outs
    d_status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rfsr.me_cc_project_noalloc(dev(smp), dev(msk), refs, d_psum, d_pcnt, H, W, d_dec=d_dec,
                               d_status=d_status, cuda_stream=stream.cuda_stream, **cfg)
    stream.synchronize()
    return (int(d_status.item()), d_psum.cpu().numpy().view(np.uint16), d_pcnt.cpu().numpy(),
            d_dec.cpu().numpy(), outs)


def test_noalloc_matches_oracle():
    """One ragged 96 x 136 frame with three past frames in the RMC and NNC+FRMC modes against
    the oracle's ME + checks + projection."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    H, W = 96, 136
    seq = synth.config2(seed=78, H=H, W=W, F=4)
    t = 3
    smp, msk = seq.samples[t], seq.masks[t]
    hist = [(seq.frames[t - k], seq.samples[t - k], seq.masks[t - k]) for k in (1, 2, 3)]
    for mode in ("rmc", "nnc_frmc"):
        status, psum, pcnt, dec, _ = run_noalloc(smp, msk, hist, H, W, cc_mode=mode,
                                                 template_size=9, search_radius=8)
        ref = oracle.frame_step(smp, msk, hist, cc_mode=oracle.CC_NAMES[mode], T=9, R=8,
                                run_fsr=False)
        assert status == 0
        np.testing.assert_array_equal(psum, ref.psum)
        np.testing.assert_array_equal(pcnt, ref.pcnt)
        for k in range(3):
            np.testing.assert_array_equal(dec[k], ref.dec[k], err_msg=f"{mode} k={k + 1}")


def test_noalloc_bad_mask_leaves_outputs_unwritten():
    """A good call, then a call whose mask has two measured pixels in one 2x2 block: the second
    reports status 1 and leaves the projection sums, counts and decisions of the first as they
    were (the scratch still holds the first call's planes, which must not leak out)."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    H, W = 64, 96
    seq = synth.config2(seed=79, H=H, W=W, F=4)
    t = 3
    smp, msk = seq.samples[t], seq.masks[t]
    hist = [(seq.frames[t - k], seq.samples[t - k], seq.masks[t - k]) for k in (1, 2, 3)]
    cfg = dict(cc_mode="nnc_frmc", template_size=9, search_radius=8)
    status, psum, pcnt, dec, outs = run_noalloc(smp, msk, hist, H, W, **cfg)
    assert status == 0 and pcnt.any()
    bad = msk.copy()
    y, x = np.argwhere(bad[:2, :2] == 0)[0]
    bad[y, x] = 1                         # two measured pixels in the first 2x2 block
    status2, psum2, pcnt2, dec2, _ = run_noalloc(seq.samples[t - 1], bad, hist, H, W, fill=outs,
                                                 **cfg)
    assert status2 == 1
    np.testing.assert_array_equal(psum2, psum)
    np.testing.assert_array_equal(pcnt2, pcnt)
    np.testing.assert_array_equal(dec2, dec)
