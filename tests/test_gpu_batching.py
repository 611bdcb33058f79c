"""Batched steps and serving on the GPU.

A batched engine runs one step over all streams that have a staged frame (one persistent launch
per phase, replayed from a CUDA graph).  The kernels compute each (stream, tile) exactly as the
per-stream launches do, so every result -- reconstruction, FSR output, motion fields, decisions,
projections -- must be bit-identical to the same stream run alone on an unbatched engine, for
uneven frame sizes, mixed masks and check modes, and streams that join and leave.  The serving
engine (its own thread, continuous batching) must give the same results while client threads
push and collect concurrently.  Memory admission queues streams that do not fit and admits them
when memory frees.  Waits are bounded: a frame that is never stepped times out.
"""
import threading

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


SPECS = [  # (H, W, mask type, cc mode, seed)
    (96, 128, synth.MASK_DYNAMIC, "nnc_frmc", 1),
    (64, 64, synth.MASK_FIXED, "rmc", 2),
    (200, 136, synth.MASK_DYNAMIC, "frmc", 3),
    (48, 80, synth.MASK_FIXED, "nnc", 4),
    (120, 160, synth.MASK_DYNAMIC, "none", 5),
    (66, 98, synth.MASK_DYNAMIC, "rme", 6),
]


def sequences(F):
    return [synth.config2(seed=sd, H=H, W=W, F=F, mask_type=mt) for H, W, mt, _, sd in SPECS]


def run_alone(seqs, F, planes=True):
    """Each stream on its own unbatched engine: per frame the outputs (and debug planes)."""
    out = []
    with rfsr.Engine(device=0) as eng:
        for (H, W, _, mode, _), seq in zip(SPECS, seqs):
            st = eng.create_stream(height=H, width=W, cc_mode=mode, keep_f32=True)
            res = []
            for t in range(F):
                st.push_frame(seq.samples[t], seq.masks[t])
                rec, f32 = st.get_frame(timeout_ms=60000, f32=True)
                dbg = None
                if planes and t >= 1:
                    dbg = (st.debug_get(rfsr.DBG_MV, 1), st.debug_get(rfsr.DBG_DECISION, 1),
                           st.debug_get(rfsr.DBG_PSUM), st.debug_get(rfsr.DBG_PCNT))
                res.append((rec, f32, dbg))
            st.destroy()
            out.append(res)
    return out


def test_batched_steps_equal_streams_alone(built):
    F = 6
    seqs = sequences(F)
    alone = run_alone(seqs, F)
    with rfsr.Engine(device=0, batched=True, profile=True) as eng:
        sts = [eng.create_stream(height=H, width=W, cc_mode=mode, keep_f32=True)
               for H, W, _, mode, _ in SPECS]
        for t in range(F):
            for st, seq in zip(sts, seqs):
                st.push_frame(seq.samples[t], seq.masks[t])
            assert eng.step() == len(SPECS)
            ms, n = eng.last_step_ms()
            assert n == len(SPECS) and ms > 0
            for i, st in enumerate(sts):
                rec, f32 = st.get_frame(timeout_ms=60000, f32=True)
                np.testing.assert_array_equal(rec, alone[i][t][0], err_msg=f"stream {i} t {t}")
                np.testing.assert_array_equal(f32, alone[i][t][1], err_msg=f"stream {i} t {t}")
                if t >= 1:
                    mv, dec, psum, pcnt = alone[i][t][2]
                    np.testing.assert_array_equal(st.debug_get(rfsr.DBG_MV, 1), mv)
                    np.testing.assert_array_equal(st.debug_get(rfsr.DBG_DECISION, 1), dec)
                    np.testing.assert_array_equal(st.debug_get(rfsr.DBG_PSUM), psum)
                    np.testing.assert_array_equal(st.debug_get(rfsr.DBG_PCNT), pcnt)


@pytest.mark.parametrize("rows,blocks,variant", [(64, 4, 0), (32, 4, 0), (64, 2, 0), (32, 2, 0),
                                                 (64, 8, 0), (32, 8, 0), (64, 4, 1)])
def test_every_batch_shape_equals_streams_alone(built, rows, blocks, variant):
    """Each tile shape the autotuner can choose gives the same bits as the streams run alone."""
    F = 4
    seqs = sequences(F)
    alone = run_alone(seqs, F, planes=False)
    with rfsr.Engine(device=0, batched=True, autotune=False) as eng:
        eng.set_shape(me_tile_rows=rows, fsr_blocks=blocks, me_variant=variant)
        assert eng.tuning()["shape"] == {"me_tile_rows": rows, "fsr_blocks": blocks,
                                         "me_variant": variant}
        sts = [eng.create_stream(height=H, width=W, cc_mode=mode, keep_f32=True)
               for H, W, _, mode, _ in SPECS]
        for t in range(F):
            for st, seq in zip(sts, seqs):
                st.push_frame(seq.samples[t], seq.masks[t])
            eng.step()
            for i, st in enumerate(sts):
                rec, f32 = st.get_frame(timeout_ms=60000, f32=True)
                np.testing.assert_array_equal(rec, alone[i][t][0], err_msg=f"stream {i} t {t}")
                np.testing.assert_array_equal(f32, alone[i][t][1], err_msg=f"stream {i} t {t}")


def test_autotuner_measures_every_candidate_and_settles(built):
    F = 12
    seqs = sequences(F)
    alone = run_alone(seqs, F, planes=False)
    with rfsr.Engine(device=0, batched=True) as eng:
        assert not eng.tuning()["tuned"]
        sts = [eng.create_stream(height=H, width=W, cc_mode=mode, keep_f32=True)
               for H, W, _, mode, _ in SPECS]
        for t in range(F):
            for st, seq in zip(sts, seqs):
                st.push_frame(seq.samples[t], seq.masks[t])
            eng.step()
            for i, st in enumerate(sts):
                rec, f32 = st.get_frame(timeout_ms=60000, f32=True)
                np.testing.assert_array_equal(rec, alone[i][t][0])
                np.testing.assert_array_equal(f32, alone[i][t][1])
        tu = eng.tuning()
        assert tu["tuned"] and tu["steps"] >= 6
        assert all(v > 0 for v in tu["fsr_ns_per_block"].values())
        assert all(v > 0 for v in tu["me_ns_per_pixel_ref"].values())
        assert tu["shape"]["me_tile_rows"] in (32, 64) and tu["shape"]["fsr_blocks"] in (2, 4, 8)
        with pytest.raises(rfsr.RfsrError) as e:
            eng.set_shape(me_tile_rows=48)
        assert e.value.code == rfsr.RFSR_EINVAL


def test_batched_streams_join_and_leave(built):
    """Streams start at different steps and leave early; device and host pushes mixed."""
    F = 6
    seqs = sequences(F)
    alone = run_alone(seqs, F, planes=False)
    start = [0, 2, 1, 3, 0, 1]
    stop = [6, 6, 4, 6, 3, 5]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    keep = []
    with rfsr.Engine(device=0, batched=True) as eng:
        sts = [None] * len(SPECS)
        for step in range(F + 3):
            for i, (H, W, _, mode, _) in enumerate(SPECS):
                if step == start[i]:
                    sts[i] = eng.create_stream(height=H, width=W, cc_mode=mode, keep_f32=True)
                t = step - start[i]
                if sts[i] is not None and 0 <= t < stop[i] - start[i] and t < F:
                    if i % 2:
                        a, b = dev(seqs[i].samples[t]), dev(seqs[i].masks[t])
                        keep.append((a, b))
                        sts[i].push_frame_device(a, b)
                    else:
                        sts[i].push_frame(seqs[i].samples[t], seqs[i].masks[t])
            eng.step()
            for i in range(len(SPECS)):
                t = step - start[i]
                if sts[i] is not None and 0 <= t < stop[i] - start[i] and t < F:
                    rec, f32 = sts[i].get_frame(timeout_ms=60000, f32=True)
                    np.testing.assert_array_equal(rec, alone[i][t][0])
                    np.testing.assert_array_equal(f32, alone[i][t][1])
                if sts[i] is not None and step == stop[i] - 1 + start[i] and i % 3 == 0:
                    sts[i].destroy()
                    sts[i] = None


def test_serving_engine_equals_streams_alone(built):
    """Client threads push and collect concurrently on a serving engine (continuous batching);
    every frame equals the stream run alone."""
    F = 8
    seqs = sequences(F)
    alone = run_alone(seqs, F, planes=False)
    results = {}
    errors = []
    with rfsr.Engine(device=0, serve=True, max_inflight=2) as eng:
        sts = [eng.create_stream(height=H, width=W, cc_mode=mode, keep_f32=True)
               for H, W, _, mode, _ in SPECS]

        def client(i):
            try:
                got = []
                pending = 0
                t = 0
                while len(got) < F:
                    if t < F and pending < 2:
                        sts[i].push_frame(seqs[i].samples[t], seqs[i].masks[t])
                        t += 1
                        pending += 1
                    else:
                        got.append(sts[i].get_frame(timeout_ms=60000, f32=True))
                        pending -= 1
                results[i] = got
            except Exception as e:   # reported below
                errors.append(e)

        th = [threading.Thread(target=client, args=(i,)) for i in range(len(SPECS))]
        for x in th:
            x.start()
        for x in th:
            x.join()
    assert not errors, errors
    for i in range(len(SPECS)):
        for t in range(F):
            np.testing.assert_array_equal(results[i][t][0], alone[i][t][0])
            np.testing.assert_array_equal(results[i][t][1], alone[i][t][1])


def test_memory_admission_queues_and_admits(built):
    seq = synth.config2(seed=7, H=128, W=160, F=3)
    probe = rfsr.Engine(device=0, batched=True)
    st0 = probe.create_stream(height=128, width=160)
    need = st0.info().device_bytes
    probe.destroy()
    with rfsr.Engine(device=0, batched=True, memory_budget=int(need * 1.5)) as eng:
        a = eng.create_stream(height=128, width=160)
        b = eng.create_stream(height=128, width=160, allow_queued=True)
        assert a.live and not b.live
        with pytest.raises(rfsr.RfsrError) as e:
            b.push_frame(seq.samples[0], seq.masks[0])
        assert e.value.code == rfsr.RFSR_EAGAIN
        with pytest.raises(rfsr.RfsrError) as e:
            eng.create_stream(height=1024, width=1024)          # alone exceeds the budget
        assert e.value.code == rfsr.RFSR_ENOMEM
        a.push_frame(seq.samples[0], seq.masks[0])
        eng.step()
        a.get_frame(timeout_ms=60000)
        a.destroy()
        assert b.live
        for t in range(3):
            b.push_frame(seq.samples[t], seq.masks[t])
            eng.step()
            b.get_frame(timeout_ms=60000)


def test_bounded_waits(built):
    """A staged frame that is never stepped times out instead of hanging."""
    seq = synth.config2(seed=8, H=64, W=64, F=1)
    with rfsr.Engine(device=0, batched=True) as eng:
        st = eng.create_stream(height=64, width=64)
        st.push_frame(seq.samples[0], seq.masks[0])
        with pytest.raises(rfsr.RfsrError) as e:
            st.get_frame(timeout_ms=50)
        assert e.value.code == rfsr.RFSR_ETIMEDOUT
        with pytest.raises(rfsr.RfsrError) as e:
            eng.sync(timeout_ms=10)
        assert e.value.code == rfsr.RFSR_ESTATE
        eng.step()
        st.get_frame(timeout_ms=60000)


# --------------------------------------------------------------------------------------------
# a batched step of several streams against the oracle (not only against the streams alone)
# --------------------------------------------------------------------------------------------
ORACLE_SPECS = [  # (H, W, mask type, cc mode, seed): T = 9, three past frames each
    (240, 320, synth.MASK_DYNAMIC, "nnc_frmc", 11),
    (130, 250, synth.MASK_FIXED, "frmc", 12),
    (96, 128, synth.MASK_DYNAMIC, "rmc", 13),
    (66, 98, synth.MASK_DYNAMIC, "rme", 14),
    (64, 64, synth.MASK_FIXED, "nnc", 15),
]


@pytest.mark.parametrize("rows,blocks,variant", [(64, 4, 0), (32, 2, 1)])
def test_batched_step_against_oracle(built, rows, blocks, variant):
    """One batched step over streams of uneven sizes, masks and check modes, with injected
    generator-made past frames: every stream's motion fields, filtered fields, decisions and
    projections equal the oracle's bit for bit, and its FSR output passes the replay rule.
    variant 1 runs the T = 9 motion estimation as sliding-window box sums (me_variant = 1), so its
    vectors are compared with the oracle's directly."""
    import oracle
    from fsr_parity import check_replay
    t = 3
    seqs = [synth.config2(seed=sd, H=H, W=W, F=t + 1, mask_type=mt)
            for H, W, mt, _, sd in ORACLE_SPECS]
    with rfsr.Engine(device=0, batched=True, autotune=False) as eng:
        eng.set_shape(me_tile_rows=rows, fsr_blocks=blocks, me_variant=variant)
        sts = [eng.create_stream(height=H, width=W, cc_mode=mode, keep_f32=True, fsr_trace=True)
               for H, W, _, mode, _ in ORACLE_SPECS]
        hists = []
        for st, seq in zip(sts, seqs):
            hist = [(seq.frames[t - k], seq.samples[t - k], seq.masks[t - k]) for k in (1, 2, 3)]
            hists.append(hist)
            st.set_history(hist)
            st.push_frame(seq.samples[t], seq.masks[t])
        assert eng.step() == len(ORACLE_SPECS)
        for st, seq, hist, (H, W, _, mode, _) in zip(sts, seqs, hists, ORACLE_SPECS):
            rec, f32 = st.get_frame(timeout_ms=60000, f32=True)
            ref = oracle.frame_step(seq.samples[t], seq.masks[t], hist,
                                    cc_mode=oracle.CC_NAMES[mode], T=9, R=8)
            for k in range(3):
                np.testing.assert_array_equal(st.debug_get(rfsr.DBG_MV, k + 1), ref.mv[k],
                                              err_msg=f"{H}x{W} {mode} mv k={k + 1}")
                np.testing.assert_array_equal(st.debug_get(rfsr.DBG_FMV, k + 1), ref.fmv[k])
                np.testing.assert_array_equal(st.debug_get(rfsr.DBG_DECISION, k + 1), ref.dec[k],
                                              err_msg=f"{H}x{W} {mode} dec k={k + 1}")
            np.testing.assert_array_equal(st.debug_get(rfsr.DBG_PSUM), ref.psum)
            np.testing.assert_array_equal(st.debug_get(rfsr.DBG_PCNT), ref.pcnt)
            check_replay(f32, st.debug_get(rfsr.DBG_FSR_SEL), seq.samples[t], seq.masks[t],
                         ref.psum, ref.pcnt)
            m = seq.masks[t] == 1
            np.testing.assert_array_equal(rec[m], seq.samples[t][m])
