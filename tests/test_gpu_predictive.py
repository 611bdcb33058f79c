"""GPU parity of the predictive-centre ME variant (opt-in, not in the paper): past frames t-2 and
later are searched within radius Rp of k * v1(p).  The GPU's motion fields, filtered fields,
decisions and projections must equal the oracle's bit for bit, and its FSR output must pass the
replay rule of tests/fsr_parity.py.  Past frames come from the generator (rfsr_set_history), so no
oracle input comes from the GPU.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from fsr_parity import check_replay

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2203_09200_gb300 import rfsr  # noqa: E402


@pytest.fixture(scope="module")
def engine():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    eng = rfsr.Engine(device=0, max_inflight=4)
    yield eng
    eng.destroy()


def _step(eng, smp, msk, hist, **cfg):
    H, W = smp.shape
    st = eng.create_stream(height=H, width=W, keep_f32=True, fsr_trace=True, **cfg)
    try:
        st.set_history(hist)
        st.push_frame(smp, msk)
        rec, f32 = st.get_frame(timeout_ms=120000, f32=True)
        K = len(hist)
        return dict(rec=rec, fsr=f32, sel=st.debug_get(rfsr.DBG_FSR_SEL),
                    mv=[st.debug_get(rfsr.DBG_MV, k) for k in range(1, K + 1)],
                    fmv=[st.debug_get(rfsr.DBG_FMV, k) for k in range(1, K + 1)],
                    dec=[st.debug_get(rfsr.DBG_DECISION, k) for k in range(1, K + 1)],
                    psum=st.debug_get(rfsr.DBG_PSUM), pcnt=st.debug_get(rfsr.DBG_PCNT))
    finally:
        st.destroy()


def _history(seq, t, K):
    return [(seq.frames[t - k], seq.samples[t - k], seq.masks[t - k]) for k in range(1, K + 1)]


# ragged sizes over several 32x32 tiles, both search radii, windows from 1 to the full 2R
@pytest.mark.parametrize("H,W,R,Rp,mode,seed", [
    (72, 104, 8, 2, "nnc_frmc", 1),
    (130, 158, 9, 1, "rmc", 2),
    (66, 98, 4, 3, "frmc", 3),
    (96, 128, 3, 6, "nnc", 4),
])
def test_predictive_step_against_oracle(engine, H, W, R, Rp, mode, seed):
    seq = synth.config2(seed=400 + seed, H=H, W=W, F=5)
    t = 4
    smp, msk = seq.samples[t], seq.masks[t]
    hist = _history(seq, t, 3)
    got = _step(engine, smp, msk, hist, cc_mode=mode, search_radius=R, check_radius=R,
                me_predict_radius=Rp)
    ref = oracle.frame_step(smp, msk, hist, cc_mode=oracle.CC_NAMES[mode], T=9, R=R, Rc=R,
                            me_predict_radius=Rp)
    for k in range(3):
        np.testing.assert_array_equal(got["mv"][k], ref.mv[k], err_msg=f"mv k={k + 1}")
        np.testing.assert_array_equal(got["fmv"][k], ref.fmv[k], err_msg=f"fmv k={k + 1}")
        np.testing.assert_array_equal(got["dec"][k], ref.dec[k], err_msg=f"dec k={k + 1}")
    np.testing.assert_array_equal(got["psum"], ref.psum)
    np.testing.assert_array_equal(got["pcnt"], ref.pcnt)
    check_replay(got["fsr"], got["sel"], smp, msk, ref.psum, ref.pcnt)


def test_predictive_fields_720p_every_pixel(engine):
    """Whole 1280x720 frame, three past frames, Rp = 2: every pixel of every field."""
    seq = synth.config2(F=4)
    t = 3
    smp, msk = seq.samples[t], seq.masks[t]
    hist = _history(seq, t, 3)
    H, W = smp.shape
    st = engine.create_stream(height=H, width=W, cc_mode="nnc_frmc", me_predict_radius=2)
    try:
        st.set_history(hist)
        st.push_frame(smp, msk)
        st.get_frame(timeout_ms=120000)
        mv = [st.debug_get(rfsr.DBG_MV, k) for k in (1, 2, 3)]
    finally:
        st.destroy()
    oracle.set_threads(max(1, min(16, os.cpu_count() or 1)))
    try:
        mv1 = oracle.me_field(smp, msk, hist[0][0], 9, 8)
        np.testing.assert_array_equal(mv[0], mv1)
        for k in (2, 3):
            want = oracle.me_field_predictive(smp, msk, hist[k - 1][0], 9, 8, 2, k, mv1)
            np.testing.assert_array_equal(mv[k - 1], want, err_msg=f"k={k}")
    finally:
        oracle.set_threads(1)


def test_full_window_equals_full_search(engine):
    """Rp = 2R covers [-R, R]^2: the fields equal those of the default (full-search) stream."""
    seq = synth.config2(seed=410, H=120, W=200, F=4)
    t = 3
    smp, msk = seq.samples[t], seq.masks[t]
    hist = _history(seq, t, 3)
    a = _step(engine, smp, msk, hist, cc_mode="nnc_frmc", search_radius=5, check_radius=5)
    b = _step(engine, smp, msk, hist, cc_mode="nnc_frmc", search_radius=5, check_radius=5,
              me_predict_radius=10)
    for k in range(3):
        np.testing.assert_array_equal(a["mv"][k], b["mv"][k])
        np.testing.assert_array_equal(a["dec"][k], b["dec"][k])


def test_predictive_config_errors(engine):
    with pytest.raises(rfsr.RfsrError, match="EINVAL"):
        engine.create_stream(height=64, width=64, me_predict_radius=19)
    with pytest.raises(rfsr.RfsrError, match="EINVAL"):
        engine.create_stream(height=64, width=64, template_size=7, me_predict_radius=2)
    batched = rfsr.Engine(device=0, batched=True)
    try:
        with pytest.raises(rfsr.RfsrError, match="EINVAL"):
            batched.create_stream(height=64, width=64, me_predict_radius=2)
    finally:
        batched.destroy()


def test_predictive_stream_resumes_from_export(engine):
    """The option travels with the stream state: a stream imported from an export made after
    frame 3 continues bit-identically to the uninterrupted stream."""
    seq = synth.config2(seed=420, H=96, W=160, F=6)
    H, W = seq.shape
    a = engine.create_stream(height=H, width=W, cc_mode="nnc_frmc", me_predict_radius=2)
    try:
        for f in range(4):
            a.push_frame(seq.samples[f], seq.masks[f])
            a.get_frame(timeout_ms=120000)
        b = engine.import_stream(a.export_state())
        try:
            for f in (4, 5):
                a.push_frame(seq.samples[f], seq.masks[f])
                b.push_frame(seq.samples[f], seq.masks[f])
                np.testing.assert_array_equal(a.get_frame(timeout_ms=120000),
                                              b.get_frame(timeout_ms=120000))
                for k in (1, 2, 3):
                    np.testing.assert_array_equal(a.debug_get(rfsr.DBG_MV, k),
                                                  b.debug_get(rfsr.DBG_MV, k))
        finally:
            b.destroy()
    finally:
        a.destroy()


def test_predictive_noalloc_matches_stream(engine):
    """The allocation-free ME + checks + projection call honours the option like a stream."""
    seq = synth.config2(seed=430, H=80, W=120, F=5)
    t = 4
    H, W = seq.shape
    smp, msk = seq.samples[t], seq.masks[t]
    hist = _history(seq, t, 3)
    got = _step(engine, smp, msk, hist, cc_mode="nnc_frmc", me_predict_radius=2)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    refs = [(dev(r), dev(s), dev(m)) for r, s, m in hist]
    d_psum = torch.zeros((H, W), dtype=torch.int16, device="cuda")
    d_pcnt = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    d_dec = torch.zeros((3, H, W), dtype=torch.uint8, device="cuda")
    rfsr.me_cc_project_noalloc(dev(smp), dev(msk), refs, d_psum, d_pcnt, H, W, d_dec=d_dec,
                               cc_mode="nnc_frmc", me_predict_radius=2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d_psum.cpu().numpy().view(np.uint16), got["psum"])
    np.testing.assert_array_equal(d_pcnt.cpu().numpy(), got["pcnt"])
    for k in range(3):
        np.testing.assert_array_equal(d_dec[k].cpu().numpy(), got["dec"][k])
