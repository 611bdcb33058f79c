"""Stream state export / import (checkpoint, resume, migration between engines) and the router.

The recursion state of a stream is its configuration and the reconstructed frame, sample plane
and mask of its last K frames (the past frames that ME and projection read, Sec. 2.2).  A stream
resumed from an exported state must give bit-identical results to the stream it came from.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2203_09200_gb300 import rfsr  # noqa: E402


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def run(st, seq, frames):
    out = []
    for t in frames:
        st.push_frame(seq.samples[t], seq.masks[t])
        out.append(st.get_frame(timeout_ms=60000, f32=True))
    return out


@pytest.mark.parametrize("mode,batched", [("nnc_frmc", False), ("rme", True), ("rmc", False)])
def test_export_import_resumes_bit_exact(built, mode, batched):
    seq = synth.config2(seed=31, H=120, W=176, F=9)
    kw = dict(height=120, width=176, cc_mode=mode, keep_f32=True)
    with rfsr.Engine(device=0) as a, rfsr.Engine(device=0, batched=batched, serve=batched) as b:
        st = a.create_stream(**kw)
        run(st, seq, range(5))
        state = st.export_state()
        assert len(state) > 3 * 3 * 120 * 176            # three past frames of three planes
        moved = b.import_stream(state)
        assert moved.info().history_frames == 3
        ref = run(st, seq, range(5, 9))                  # the original continues on engine a
        got = run(moved, seq, range(5, 9))               # the imported copy on engine b
        for (r8, r32), (g8, g32) in zip(ref, got):
            np.testing.assert_array_equal(g8, r8)
            np.testing.assert_array_equal(g32, r32)


def test_export_import_errors(built):
    seq = synth.config2(seed=32, H=64, W=64, F=2)
    with rfsr.Engine(device=0) as eng:
        st = eng.create_stream(height=64, width=64)
        st.push_frame(seq.samples[0], seq.masks[0])
        with pytest.raises(rfsr.RfsrError) as e:         # a frame not yet collected
            st.export_state()
        assert e.value.code == rfsr.RFSR_ESTATE
        st.get_frame(timeout_ms=60000)
        state = bytearray(st.export_state())
        with pytest.raises(rfsr.RfsrError) as e:         # not a state buffer
            eng.import_stream(b"\0" * len(state))
        assert e.value.code == rfsr.RFSR_EINVAL
        with pytest.raises(rfsr.RfsrError) as e:         # truncated
            eng.import_stream(bytes(state[:-1]))
        assert e.value.code == rfsr.RFSR_EINVAL
        need = st.info().device_bytes
    with rfsr.Engine(device=0, memory_budget=int(need * 1.5)) as small:
        small.create_stream(height=64, width=64)
        with pytest.raises(rfsr.RfsrError) as e:         # budget full: nothing is created
            small.import_stream(bytes(state))
        assert e.value.code == rfsr.RFSR_EAGAIN
        assert small.info()["streams_queued"] == 0


def test_router_places_and_migrates(built):
    seqs = [synth.config2(seed=40 + i, H=96, W=128, F=6) for i in range(4)]
    with rfsr.Engine(device=0) as alone:
        ref = []
        for q in seqs:
            st = alone.create_stream(height=96, width=128, keep_f32=True)
            ref.append([o for o, _ in run(st, q, range(6))])
            st.destroy()
    with rfsr.Engine(device=0, memory_budget=400 << 20) as e0, \
            rfsr.Engine(device=0, memory_budget=400 << 20) as e1:
        router = rfsr.Router([e0, e1])
        sts = [router.create_stream(height=96, width=128, keep_f32=True) for _ in seqs]
        assert {s.engine for s in sts} == {e0, e1}           # spread over both replicas
        got = [[run(s, q, [t])[0][0] for t in range(3)] for s, q in zip(sts, seqs)]
        sts[0] = router.migrate(sts[0], e1 if sts[0].engine is e0 else e0)
        for i, (s, q) in enumerate(zip(sts, seqs)):
            got[i] += [run(s, q, [t])[0][0] for t in range(3, 6)]
    for g, r in zip(got, ref):
        for a, b in zip(g, r):
            np.testing.assert_array_equal(a, b)
