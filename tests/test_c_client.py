"""The C ABI from a plain C program (tests/c/rfsr_c_client.c): it compiles and links against
include/rfsr.h and librfsr.so with a C compiler (CPU), and on a GPU its reconstructions equal the
Python binding's for the same frames."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "rfsr_c_client.c")
LIBDIR = os.path.join(ROOT, "paper_2203_09200_gb300")


def build_client(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    if not os.path.exists(os.path.join(LIBDIR, "librfsr.so")):
        pytest.skip("librfsr.so not built")
    exe = str(tmp_path / "rfsr_c_client")
    subprocess.run([cc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    SRC, "-L", LIBDIR, "-lrfsr", f"-Wl,-rpath,{LIBDIR}", "-o", exe], check=True)
    return exe


def test_c_client_compiles_and_links(tmp_path):
    assert os.path.exists(build_client(tmp_path))


@pytest.mark.gpu
def test_c_client_matches_the_binding(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    exe = build_client(tmp_path)
    H, W, F = 96, 160, 6
    seq = synth.config2(seed=61, H=H, W=W, F=F)
    inp = np.stack([np.stack([seq.samples[t], seq.masks[t]]) for t in range(F)]).astype(np.uint8)
    (tmp_path / "in.bin").write_bytes(inp.tobytes())
    subprocess.run([exe, str(H), str(W), str(F), str(tmp_path / "in.bin"), str(tmp_path / "out.bin")],
                   check=True, timeout=300)
    got = np.frombuffer((tmp_path / "out.bin").read_bytes(), np.uint8).reshape(F, H, W)
    from paper_2203_09200_gb300 import rfsr
    with rfsr.Engine(device=0) as eng:
        st = eng.create_stream(height=H, width=W)
        for t in range(F):
            st.push_frame(seq.samples[t], seq.masks[t])
            np.testing.assert_array_equal(got[t], st.get_frame(timeout_ms=60000), err_msg=f"t={t}")
