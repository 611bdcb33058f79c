"""The fused ME + checks + projection launch of unbatched streams (engine option fuse_me_cc;
T = 9, full ME search, no RME): one persistent launch per frame in which the check tiles wait
for the ME bands they read.

* Its results equal those of the separate ME and checks launches (the default, which
  test_gpu_parity.py compares with the oracle) bit for bit, over several frames of a
  free-running stream.
* Its waits are bounded: an engine with wait_test set makes every wait run out (a count that no
  ME tile reaches).  The frame then ends with EDEVICE, the stream must be reset, and the context
  stays usable for the next frame and for other engines.  No GPU is faulted or hung.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2203_09200_gb300 import rfsr  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _run(seq, frames, **eng_kw):
    H, W = seq.shape
    out = []
    with rfsr.Engine(device=0, **eng_kw) as eng:
        st = eng.create_stream(height=H, width=W, cc_mode="nnc_frmc", keep_f32=True)
        for f in range(frames):
            st.push_frame(seq.samples[f], seq.masks[f])
            rec, f32 = st.get_frame(timeout_ms=120000, f32=True)
            K = min(f, 3)
            out.append((rec, f32, [st.debug_get(rfsr.DBG_MV, k) for k in range(1, K + 1)],
                        [st.debug_get(rfsr.DBG_DECISION, k) for k in range(1, K + 1)],
                        st.debug_get(rfsr.DBG_PSUM), st.debug_get(rfsr.DBG_PCNT)))
    return out


@pytest.mark.parametrize("H,W,seed", [(200, 248, 1), (130, 96, 2), (64, 64, 3)])
def test_fused_equals_separate_launches(H, W, seed):
    seq = synth.config2(seed=500 + seed, H=H, W=W, F=6)
    a = _run(seq, 6, fuse_me_cc=True)
    b = _run(seq, 6)
    for f, (x, y) in enumerate(zip(a, b)):
        np.testing.assert_array_equal(x[0], y[0], err_msg=f"rec frame {f}")
        np.testing.assert_array_equal(x[1], y[1], err_msg=f"fsr frame {f}")
        for k in range(len(x[2])):
            np.testing.assert_array_equal(x[2][k], y[2][k], err_msg=f"mv frame {f} k={k + 1}")
            np.testing.assert_array_equal(x[3][k], y[3][k], err_msg=f"dec frame {f} k={k + 1}")
        np.testing.assert_array_equal(x[4], y[4], err_msg=f"psum frame {f}")
        np.testing.assert_array_equal(x[5], y[5], err_msg=f"pcnt frame {f}")


def test_fused_full_hd_equals_separate_launches():
    seq = synth.config3(seed=7, F=4)
    a = _run(seq, 4, fuse_me_cc=True)
    b = _run(seq, 4)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x[0], y[0])
        for k in range(len(x[2])):
            np.testing.assert_array_equal(x[2][k], y[2][k])
            np.testing.assert_array_equal(x[3][k], y[3][k])


def test_waits_that_run_out_end_the_frame_with_edevice():
    seq = synth.config2(seed=520, H=128, W=192, F=4)
    H, W = seq.shape
    with rfsr.Engine(device=0, fuse_me_cc=True, wait_test=True) as eng:
        st = eng.create_stream(height=H, width=W, cc_mode="nnc_frmc")
        st.push_frame(seq.samples[0], seq.masks[0])       # no past frame: no fused launch
        st.get_frame(timeout_ms=120000)
        st.push_frame(seq.samples[1], seq.masks[1])
        with pytest.raises(rfsr.RfsrError, match="EDEVICE"):
            st.get_frame(timeout_ms=120000)
        with pytest.raises(rfsr.RfsrError, match="ESTATE"):   # the stream must be reset
            st.push_frame(seq.samples[2], seq.masks[2])
    # the context is intact: a fused engine runs the same frames and matches the separate path
    a = _run(seq, 4, fuse_me_cc=True)
    b = _run(seq, 4)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x[0], y[0])
