"""Boundary details of the C ABI on the GPU: the producer stream of device pushes, the caller's
device allocator, and the default engine behind NULL engine arguments."""
import ctypes as C

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


def host_run(seq, frames, **kw):
    H, W = seq.shape
    with rfsr.Engine(device=0) as eng:
        st = eng.create_stream(height=H, width=W, keep_f32=True, **kw)
        out = []
        for t in frames:
            st.push_frame(seq.samples[t], seq.masks[t])
            out.append(st.get_frame(timeout_ms=60000, f32=True))
    return out


@pytest.mark.parametrize("batched", [False, True])
def test_device_push_waits_for_the_producer_stream(built, batched):
    """The frame is written on another stream behind a ~25 ms GPU spin; the push returns at once
    and the engine's work must still see the new data (an event dependency, no host wait)."""
    seq = synth.config2(seed=51, H=96, W=128, F=3)
    ref = host_run(seq, range(3))
    prod = torch.cuda.Stream()
    d_s = torch.zeros((96, 128), dtype=torch.uint8, device="cuda")
    d_m = torch.zeros((96, 128), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    with rfsr.Engine(device=0, batched=batched) as eng:
        st = eng.create_stream(height=96, width=128, keep_f32=True)
        for t in range(3):
            src_s = torch.from_numpy(seq.samples[t]).pin_memory()
            src_m = torch.from_numpy(seq.masks[t]).pin_memory()
            with torch.cuda.stream(prod):
                torch.cuda._sleep(50_000_000)
                d_s.copy_(src_s, non_blocking=True)
                d_m.copy_(src_m, non_blocking=True)
            st.push_frame_device(d_s, d_m, stream=prod)
            if batched:
                eng.step()
            rec, f32 = st.get_frame(timeout_ms=60000, f32=True)
            np.testing.assert_array_equal(rec, ref[t][0])
            np.testing.assert_array_equal(f32, ref[t][1])
            prod.synchronize()


def test_torch_caching_allocator(built):
    seq = synth.config2(seed=52, H=96, W=128, F=3)
    ref = host_run(seq, range(3))
    before = torch.cuda.memory_allocated(0)
    with rfsr.Engine(device=0, allocator="torch") as eng:
        st = eng.create_stream(height=96, width=128, keep_f32=True)
        held = torch.cuda.memory_allocated(0) - before
        assert held >= st.info().device_bytes > 0          # stream state came from torch
        for t in range(3):
            st.push_frame(seq.samples[t], seq.masks[t])
            rec, f32 = st.get_frame(timeout_ms=60000, f32=True)
            np.testing.assert_array_equal(rec, ref[t][0])
            np.testing.assert_array_equal(f32, ref[t][1])
        st.destroy()
    assert torch.cuda.memory_allocated(0) == before         # and went back to it


def test_allocator_callbacks_come_in_pairs(built):
    lib = rfsr.load()
    cfg = rfsr.rfsr_engine_config()
    lib.rfsr_engine_config_default(C.byref(cfg))
    cfg.dev_alloc = rfsr.ALLOC_FN(lambda n, ctx: None)
    h = C.c_void_p()
    assert lib.rfsr_engine_create(C.byref(cfg), C.byref(h)) == rfsr.RFSR_EINVAL


def test_null_engine_uses_the_default_engine(built):
    seq = synth.config2(seed=53, H=64, W=96, F=2)
    ref = host_run(seq, range(2))
    lib = rfsr.load()
    cfg = rfsr.stream_config(64, 96, keep_f32=True)
    h = C.c_void_p()
    assert lib.rfsr_create_stream(None, C.byref(cfg), C.byref(h)) == 0
    out = np.empty((64, 96), np.uint8)
    o32 = np.empty((64, 96), np.float32)
    for t in range(2):
        s = np.ascontiguousarray(seq.samples[t])
        m = np.ascontiguousarray(seq.masks[t])
        assert lib.rfsr_push_frame(h, s.ctypes.data, m.ctypes.data) == 0
        assert lib.rfsr_get_frame(h, out.ctypes.data, o32.ctypes.data, 60000) == 0
        np.testing.assert_array_equal(out, ref[t][0])
        np.testing.assert_array_equal(o32, ref[t][1])
    assert lib.rfsr_destroy(h) == 0
