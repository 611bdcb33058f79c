"""GPU parity of FSR with concealed weighting delta > 0 (the original FSR; the paper sets delta to
zero in Sec. 4 so that blocks are independent).

With delta > 0 block (i, j) reads the reconstruction of the blocks before it in raster order, so
the oracle runs in the same order, each block replaying the selection sequence the GPU recorded
for it and reading the oracle's own earlier outputs as concealed values.  Every block is then
compared under the replay rule of tests/fsr_parity.py: within 1e-4 of the replay, and every
iteration that leaves the FP64 argmax a tie within FP32 rounding.  The output buffer is filled
with a value far outside [0, 1] before the call, so a block that read a concealed pixel before
its block was written would show.
"""
import numpy as np
import pytest

import oracle
import synth
from fsr_parity import BOUND, check_against

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2203_09200_gb300 import rfsr  # noqa: E402

B = 4


@pytest.fixture(scope="module")
def engine():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    eng = rfsr.Engine(device=0, max_inflight=4)
    yield eng
    eng.destroy()


def projections(seq, msk, seed, frac=0.4):
    H, W = msk.shape
    rng = np.random.default_rng(seed)
    pcnt = np.where((msk == 0) & (rng.random((H, W)) < frac), rng.integers(1, 4, (H, W)), 0)
    pcnt = pcnt.astype(np.uint8)
    psum = (pcnt.astype(np.uint16) * seq.frames[0]).astype(np.uint16)
    return psum, pcnt


def check_raster(got, sel, P, delta, smp, msk, psum, pcnt):
    """Raster-order replay of every block against the GPU's output; returns the stats dict."""
    assert np.isfinite(got).all()
    out, _, rep = oracle.fsr_frame_concealed(P, delta, smp, msk, psum, pcnt, sel=sel, bound=BOUND)
    return check_against(got, out, rep, B=B)


def run_fsr_device(smp, msk, psum, pcnt, delta, iters):
    H, W = smp.shape
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out32 = torch.full((H, W), 7.0, dtype=torch.float32, device="cuda")
    out8 = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    sel = torch.empty(((-(-H // B)) * (-(-W // B)), iters), dtype=torch.int16, device="cuda")
    rfsr.fsr_device_trace(dev(smp), dev(msk), None if psum is None else dev(psum),
                          None if pcnt is None else dev(pcnt), out32, out8, sel, H, W,
                          cuda_stream=torch.cuda.current_stream().cuda_stream,
                          fsr_iterations=iters, fsr_concealed_weight=delta)
    torch.cuda.synchronize()
    return out32.cpu().numpy(), out8.cpu().numpy(), sel.cpu().numpy().view(np.uint16)


@pytest.mark.parametrize("H,W,delta,iters,proj", [
    (64, 96, 0.5, 100, True),      # the paper's iteration count, with projected pixels
    (50, 70, 0.2, 30, False),      # ragged edges in both directions
    (24, 200, 1.0, 60, True),      # wide frame: many blocks per wavefront
    (120, 16, 0.5, 60, True),      # four block columns: one block per wavefront
])
def test_concealed_fsr_device_matches_oracle(engine, H, W, delta, iters, proj):
    seq = synth.config2(seed=H + W, H=H, W=W, F=1)
    smp, msk = seq.samples[0], seq.masks[0]
    psum, pcnt = projections(seq, msk, seed=H) if proj else (None, None)
    got, got8, sel = run_fsr_device(smp, msk, psum, pcnt, delta, iters)
    P = oracle.FsrParams(iterations=iters)
    stats = check_raster(got, sel, P, delta, smp, msk, psum, pcnt)
    print(f"{H}x{W} delta {delta} iters {iters}: {stats}")
    m = msk == 1
    np.testing.assert_array_equal(got8[m], smp[m])
    # delta really changes the result (the wavefront path is not the independent-block one)
    indep, _ = oracle.fsr_frame(P, smp, msk, psum, pcnt)
    assert np.abs(got.astype(np.float64) - indep).max() > 1e-3


def test_concealed_stream_step(engine):
    """A stream with delta > 0: ME, checks and projection bit-exact, FSR in raster order."""
    H, W, delta = 64, 80, 0.5
    seq = synth.config2(seed=31, H=H, W=W, F=4)
    t = 3
    smp, msk = seq.samples[t], seq.masks[t]
    hist = [(seq.frames[t - k], seq.samples[t - k], seq.masks[t - k]) for k in (1, 2, 3)]
    st = engine.create_stream(height=H, width=W, keep_f32=True, fsr_concealed_weight=delta,
                              fsr_trace=True)
    try:
        st.set_history(hist)
        st.push_frame(smp, msk)
        rec, got = st.get_frame(timeout_ms=120000, f32=True)
        psum, pcnt = st.debug_get(rfsr.DBG_PSUM), st.debug_get(rfsr.DBG_PCNT)
        sel = st.debug_get(rfsr.DBG_FSR_SEL)
    finally:
        st.destroy()
    P = oracle.FsrParams()
    ref = oracle.frame_step(smp, msk, hist, cc_mode=oracle.CC_NNC_FRMC, T=9, R=8, run_fsr=False)
    np.testing.assert_array_equal(psum, ref.psum)
    np.testing.assert_array_equal(pcnt, ref.pcnt)
    check_raster(got, sel, P, delta, smp, msk, ref.psum, ref.pcnt)
    np.testing.assert_array_equal(rec[msk == 1], smp[msk == 1])


def test_concealed_first_frame_of_a_stream(engine):
    """Frame 0 has no references (no projections): FSR alone with delta > 0."""
    H, W, delta = 40, 48, 0.5
    seq = synth.config2(seed=32, H=H, W=W, F=1)
    smp, msk = seq.samples[0], seq.masks[0]
    st = engine.create_stream(height=H, width=W, keep_f32=True, fsr_concealed_weight=delta,
                              fsr_trace=True)
    try:
        st.push_frame(smp, msk)
        _, got = st.get_frame(timeout_ms=60000, f32=True)
        sel = st.debug_get(rfsr.DBG_FSR_SEL)
    finally:
        st.destroy()
    P = oracle.FsrParams()
    check_raster(got, sel, P, delta, smp, msk, None, None)


@pytest.mark.parametrize("serve", [False, True])
def test_concealed_streams_in_batched_steps_equal_alone(engine, serve):
    """Batched and serving engines: streams with delta > 0 (their FSR runs as wavefront launches
    after each batched step) next to delta = 0 streams give the same bits as each stream alone on
    an unbatched engine, frame after frame (the recursion included)."""
    specs = [(64, 80, 0.5, 41), (48, 96, 0.0, 42), (40, 64, 1.0, 43)]
    F = 4
    seqs = [synth.config2(seed=sd, H=H, W=W, F=F) for H, W, _, sd in specs]
    alone = []
    for (H, W, d, _), seq in zip(specs, seqs):
        st = engine.create_stream(height=H, width=W, keep_f32=True, fsr_concealed_weight=d)
        res = []
        for t in range(F):
            st.push_frame(seq.samples[t], seq.masks[t])
            res.append(st.get_frame(timeout_ms=60000, f32=True))
        st.destroy()
        alone.append(res)
    with rfsr.Engine(device=0, batched=not serve, serve=serve) as beng:
        sts = [beng.create_stream(height=H, width=W, keep_f32=True, fsr_concealed_weight=d)
               for H, W, d, _ in specs]
        for t in range(F):
            for st, seq in zip(sts, seqs):
                st.push_frame(seq.samples[t], seq.masks[t])
            if not serve:
                beng.step()
            for i, st in enumerate(sts):
                rec, f32 = st.get_frame(timeout_ms=60000, f32=True)
                np.testing.assert_array_equal(rec, alone[i][t][0], err_msg=f"stream {i} t {t}")
                np.testing.assert_array_equal(f32, alone[i][t][1], err_msg=f"stream {i} t {t}")


def test_concealed_errors(engine):
    with pytest.raises(rfsr.RfsrError, match="fsr_concealed_weight"):
        engine.create_stream(height=32, width=32, fsr_concealed_weight=-1.0)
    d = torch.zeros((32, 32), dtype=torch.uint8, device="cuda")
    with pytest.raises(rfsr.RfsrError, match="d_out_f32"):
        rfsr.fsr_device(d, d, None, None, None, d, 32, 32, fsr_concealed_weight=0.5)
