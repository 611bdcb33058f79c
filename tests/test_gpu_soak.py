"""Lifecycle soak: engines (plain, batched, serving), streams of several sizes and check modes,
device pushes, state export / import, the stand-alone FSR and the allocation-free entry point,
created and destroyed over and over.  Every cycle must give the same reconstructions as the first
one, and the device memory in use must come back to where it started (no leak per cycle)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2203_09200_gb300 import rfsr  # noqa: E402

MB = 1 << 20


def used_bytes():
    torch.cuda.synchronize()
    free, total = torch.cuda.mem_get_info()
    return total - free


def one_cycle(seqs):
    """Everything the library allocates, once; returns the reconstructions it produced."""
    out = []
    with rfsr.Engine(device=0) as eng:
        for i, (seq, mode) in enumerate(seqs):
            st = eng.create_stream(height=seq.shape[0], width=seq.shape[1], cc_mode=mode)
            for t in range(4):
                if i % 2:
                    d_s = torch.from_numpy(np.ascontiguousarray(seq.samples[t])).cuda()
                    d_m = torch.from_numpy(np.ascontiguousarray(seq.masks[t])).cuda()
                    st.push_frame_device(d_s, d_m)
                else:
                    st.push_frame(seq.samples[t], seq.masks[t])
                out.append(st.get_frame(timeout_ms=60000))
            state = st.export_state()
            st.destroy()
            st2 = eng.import_stream(state)
            st2.push_frame(seq.samples[4], seq.masks[4])
            out.append(st2.get_frame(timeout_ms=60000))
            st2.destroy()
    for kw in (dict(batched=True), dict(batched=True, serve=True)):
        with rfsr.Engine(device=0, **kw) as eng:
            sts = [eng.create_stream(height=s.shape[0], width=s.shape[1], cc_mode=m)
                   for s, m in seqs]
            for t in range(4):
                for st, (seq, _) in zip(sts, seqs):
                    st.push_frame(seq.samples[t], seq.masks[t])
                if not kw.get("serve"):
                    eng.step()
                for st in sts:
                    out.append(st.get_frame(timeout_ms=60000))
            for st in sts:
                st.destroy()
    seq = seqs[0][0]
    H, W = seq.shape
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_s, d_m = dev(seq.samples[3]), dev(seq.masks[3])
    o32 = torch.empty((H, W), dtype=torch.float32, device="cuda")
    o8 = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    rfsr.fsr_device(d_s, d_m, None, None, o32, o8, H, W)
    psum = torch.empty((H, W), dtype=torch.int16, device="cuda")
    pcnt = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    refs = [(dev(seq.frames[2 - k]), dev(seq.samples[2 - k]), dev(seq.masks[2 - k]))
            for k in range(3)]
    rfsr.me_cc_project_noalloc(d_s, d_m, refs, psum, pcnt, H, W)
    torch.cuda.synchronize()
    out.append(o8.cpu().numpy())
    out.append(pcnt.cpu().numpy())
    return out


def test_lifecycle_soak_no_leak_same_results():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    seqs = [(synth.config2(seed=41, H=96, W=128, F=5), "nnc_frmc"),
            (synth.config2(seed=42, H=64, W=160, F=5), "rme"),
            (synth.config2(seed=43, H=120, W=96, F=5, mask_type=synth.MASK_FIXED), "rmc")]
    first = one_cycle(seqs)                     # warms up every one-time allocation
    base = used_bytes()
    for c in range(8):
        got = one_cycle(seqs)
        assert len(got) == len(first)
        for a, b in zip(first, got):
            np.testing.assert_array_equal(a, b, err_msg=f"cycle {c}")
        grown = used_bytes() - base
        assert grown <= 8 * MB, f"cycle {c}: {grown / MB:.1f} MB more device memory in use"
