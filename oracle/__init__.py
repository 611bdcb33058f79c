"""CPU oracle for the R-FSR frame step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of ``bench.py``
may import this package.  The product path (``paper_2203_09200_gb300``) never imports it, and it
never imports the product path: the two share only the seeded input generators in ``synth``.

The arithmetic lives in ``rfsr_oracle.c`` (plain single-threaded C, FP64 for FSR); this module
compiles it with gcc on first use and wraps it with ctypes.  ``frame_step`` composes the per-frame
chain in the order of Fig. 1: motion estimation against each of the K previous reconstructed
frames (Sec. 2.2), the consistency checks (Sec. 2.2, 3.1), projection with averaging (Sec. 2.2),
FSR with the D-FSR overwrite rule (Sec. 2.1, 3.2) and 8-bit quantisation of the result.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rfsr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "librfsr_oracle.so")
_OMP_PATH = os.path.join(_HERE, "librfsr_oracle_omp.so")
_lock = threading.Lock()
_libs = {}
_threads = 1

# decision labels and consistency-check modes (same numbering as the C file)
DEC_MEASURED, DEC_NOT_PROJECTABLE, DEC_NNC_REJECT, DEC_CHECK_REJECT, DEC_ACCEPT = range(5)
CC_NONE, CC_RME, CC_RMC, CC_FRMC, CC_NNC, CC_NNC_FRMC = range(6)
CC_NAMES = {"none": CC_NONE, "rme": CC_RME, "rmc": CC_RMC, "frmc": CC_FRMC, "nnc": CC_NNC,
            "nnc_frmc": CC_NNC_FRMC}


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle shared library: plain C, -O2, single-threaded; with omp, the same source
    with -fopenmp (frame-level loops over independent pixels and blocks on several threads)."""
    path = _OMP_PATH if omp else _LIB_PATH
    with _lock:
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            tmp = path + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared"]
            cmd += ["-fopenmp"] if omp else []
            subprocess.run(cmd + ["-o", tmp, _SRC, "-lm"], check=True)
            os.replace(tmp, path)
    return path


def set_threads(n: int) -> None:
    """Run the frame-level oracle calls on n threads (n > 1: the OpenMP build; same results)."""
    global _threads
    _threads = max(1, int(n))
    if _threads > 1:
        _load().orc_set_threads(_threads)


def threads() -> int:
    return _threads


class _FsrParams(C.Structure):
    _fields_ = [("B", C.c_int), ("N", C.c_int), ("iterations", C.c_int), ("rho", C.c_double),
                ("gamma", C.c_double), ("proj_weight", C.c_double),
                ("overwrite_projected", C.c_int)]


@dataclasses.dataclass
class FsrParams:
    """FSR configuration.  The paper takes its FSR parameters from its reference [Jonscher 2016]
    without stating them (Sec. 4); these defaults are the reading used throughout."""
    B: int = 4
    N: int = 32
    iterations: int = 100
    rho: float = 0.7
    gamma: float = 0.5
    proj_weight: float = 1.0
    overwrite_projected: bool = False   # False: D-FSR (Sec. 3.2); True: R-FSR

    def _c(self) -> _FsrParams:
        return _FsrParams(self.B, self.N, self.iterations, self.rho, self.gamma, self.proj_weight,
                          int(self.overwrite_projected))


class _Replay(C.Structure):
    _fields_ = [("iterations_run", C.c_int), ("divergences", C.c_int), ("first_div", C.c_int),
                ("invalid", C.c_int), ("first_gap", C.c_double), ("max_gap", C.c_double),
                ("max_scale", C.c_double), ("max_excess", C.c_double)]


def _load():
    omp = _threads > 1
    lib = _libs.get(omp)
    if lib is None:
        lib = C.CDLL(build(omp=omp))
        u8p, i8p, u16p = C.POINTER(C.c_uint8), C.POINTER(C.c_int8), C.POINTER(C.c_uint16)
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        I = C.c_int
        lib.orc_cost.argtypes = [u8p, u8p, u8p, I, I, I, I, I, I, I, ip, ip]
        lib.orc_better.argtypes = [I] * 8
        lib.orc_me_pixel.argtypes = [u8p, u8p, u8p, I, I, I, I, I, I, i8p, i8p]
        lib.orc_me_field.argtypes = [u8p, u8p, u8p, I, I, I, I, i8p]
        lib.orc_me_pixel_predictive.argtypes = [u8p, u8p, u8p, I, I, I, I, I, I, I, I, I, I, i8p,
                                                i8p]
        lib.orc_me_field_predictive.argtypes = [u8p, u8p, u8p, I, I, I, I, I, I, i8p, i8p]
        lib.orc_nnc_field.argtypes = [i8p, I, I, i8p, u8p]
        lib.orc_check_frmc.argtypes = [u8p, u8p, u8p, I, I, I, I, I, I, I]
        lib.orc_check_rmc.argtypes = [u8p, u8p, u8p, I, I, I, I, I, I, I, I]
        lib.orc_check_rme.argtypes = [u8p, u8p, u8p, I, I, I, I, I, I, I, I]
        lib.orc_rme_vector.argtypes = [u8p, u8p, u8p, I, I, I, I, I, I, i8p, i8p]
        lib.orc_cc_project.argtypes = [I, I, I, I, u8p, u8p, u8p, u8p, u8p, I, I, i8p, i8p, u8p,
                                       u16p, u8p]
        lib.orc_cc_pixel.argtypes = [I, I, I, I, u8p, u8p, u8p, u8p, u8p, I, I, I, I, i8p, i8p,
                                     ip]
        lib.orc_cc_pixel.restype = I
        rp = C.POINTER(_Replay)
        lib.orc_fsr_block_ex.argtypes = [C.POINTER(_FsrParams), u8p, u8p, u16p, u8p, I, I, I, I,
                                         dp, dp, dp, dp, dp, dp, ip, dp, dp]
        lib.orc_fsr_block_replay.argtypes = [C.POINTER(_FsrParams), C.c_double, dp, u8p, u8p,
                                             u16p, u8p, I, I, I, I, u16p, dp, dp, ip, dp, dp, rp]
        lib.orc_fsr_frame.argtypes = [C.POINTER(_FsrParams), u8p, u8p, u16p, u8p, I, I, dp, dp]
        lib.orc_fsr_frame_replay.argtypes = [C.POINTER(_FsrParams), u8p, u8p, u16p, u8p, I, I,
                                             u16p, dp, dp, dp, rp]
        lib.orc_fsr_frame_concealed.argtypes = [C.POINTER(_FsrParams), C.c_double, u8p, u8p, u16p,
                                                u8p, I, I, u16p, dp, dp, dp, rp]
        lib.orc_fsr_support.argtypes = [C.POINTER(_FsrParams), C.c_double, dp, u8p, u8p, u16p, u8p,
                                        I, I, I, I, dp, dp]
        lib.orc_quantize.argtypes = [dp, u8p, u8p, I, I, u8p]
        lib.orc_set_threads.argtypes = [I]
        if omp:
            lib.orc_set_threads(_threads)
        _libs[omp] = lib
    return lib


def _p(a: Optional[np.ndarray], ct):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(ct))


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


# ----------------------------------------------------------------------------------------------
# motion estimation and checks
# ----------------------------------------------------------------------------------------------
def cost(smp, msk, ref, T, py, px, vy, vx) -> Tuple[int, int]:
    """(SAD, n) of the template at p against the past frame displaced by v (Sec. 2.2)."""
    lib = _load()
    smp, msk, ref = _u8(smp), _u8(msk), _u8(ref)
    H, W = smp.shape
    s, n = C.c_int(), C.c_int()
    lib.orc_cost(_p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(ref, C.c_uint8), H, W, T, py, px,
                 vy, vx, C.byref(s), C.byref(n))
    return s.value, n.value


def better(a: Tuple[int, int, int, int], b: Tuple[int, int, int, int]) -> bool:
    """(sad, n, vy, vx) a strictly before b in the cost order with the stated tie order."""
    return bool(_load().orc_better(*a, *b))


def me_pixel(smp, msk, ref, T, R, py, px) -> Tuple[int, int]:
    lib = _load()
    smp, msk, ref = _u8(smp), _u8(msk), _u8(ref)
    H, W = smp.shape
    a, b = C.c_int8(), C.c_int8()
    lib.orc_me_pixel(_p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(ref, C.c_uint8), H, W, T, R, py,
                     px, C.byref(a), C.byref(b))
    return a.value, b.value


def me_field(smp, msk, ref, T, R) -> np.ndarray:
    """Dense motion field (H, W, 2) int8: [..., 0] vertical, [..., 1] horizontal."""
    lib = _load()
    smp, msk, ref = _u8(smp), _u8(msk), _u8(ref)
    H, W = smp.shape
    mv = np.zeros((H, W, 2), dtype=np.int8)
    lib.orc_me_field(_p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(ref, C.c_uint8), H, W, T, R,
                     _p(mv, C.c_int8))
    return mv


def me_pixel_predictive(smp, msk, ref, T, R, Rp, k, v1, py, px) -> Tuple[int, int]:
    """Predictive-centre search of pixel (py, px) in past frame t-k (k >= 2) around k * v1, v1 the
    full-search vector to t-1 (an opt-in variant outside the paper)."""
    lib = _load()
    smp, msk, ref = _u8(smp), _u8(msk), _u8(ref)
    H, W = smp.shape
    a, b = C.c_int8(), C.c_int8()
    lib.orc_me_pixel_predictive(_p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(ref, C.c_uint8), H, W,
                                T, R, Rp, k, int(v1[0]), int(v1[1]), py, px, C.byref(a),
                                C.byref(b))
    return a.value, b.value


def me_field_predictive(smp, msk, ref, T, R, Rp, k, mv1) -> np.ndarray:
    """Predictive-centre field of past frame t-k from mv1, the full-search field of t-1."""
    lib = _load()
    smp, msk, ref = _u8(smp), _u8(msk), _u8(ref)
    H, W = smp.shape
    mv1 = np.ascontiguousarray(mv1, dtype=np.int8)
    mv = np.zeros((H, W, 2), dtype=np.int8)
    lib.orc_me_field_predictive(_p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(ref, C.c_uint8), H, W,
                                T, R, Rp, k, _p(mv1, C.c_int8), _p(mv, C.c_int8))
    return mv


def nnc_field(mv) -> Tuple[np.ndarray, np.ndarray]:
    """Eq. (1) median-filtered field and the NNC pass map."""
    lib = _load()
    mv = np.ascontiguousarray(mv, dtype=np.int8)
    H, W = mv.shape[:2]
    fmv = np.zeros_like(mv)
    ok = np.zeros((H, W), dtype=np.uint8)
    lib.orc_nnc_field(_p(mv, C.c_int8), H, W, _p(fmv, C.c_int8), _p(ok, C.c_uint8))
    return fmv, ok


def check_frmc(smp, msk, ref, T, py, px, vy, vx) -> bool:
    lib = _load()
    smp, msk, ref = _u8(smp), _u8(msk), _u8(ref)
    H, W = smp.shape
    return bool(lib.orc_check_frmc(_p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(ref, C.c_uint8),
                                   H, W, T, py, px, vy, vx))


def check_rmc(smp, msk, ref, T, Rc, py, px, vy, vx) -> bool:
    lib = _load()
    smp, msk, ref = _u8(smp), _u8(msk), _u8(ref)
    H, W = smp.shape
    return bool(lib.orc_check_rmc(_p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(ref, C.c_uint8),
                                  H, W, T, Rc, py, px, vy, vx))


def check_rme(smp, msk, ref, T, R, py, px, vy, vx) -> bool:
    lib = _load()
    smp, msk, ref = _u8(smp), _u8(msk), _u8(ref)
    H, W = smp.shape
    return bool(lib.orc_check_rme(_p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(ref, C.c_uint8),
                                  H, W, T, R, py, px, vy, vx))


def rme_vector(smp, msk, ref, T, R, qy, qx) -> Tuple[int, int]:
    lib = _load()
    smp, msk, ref = _u8(smp), _u8(msk), _u8(ref)
    H, W = smp.shape
    a, b = C.c_int8(), C.c_int8()
    lib.orc_rme_vector(_p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(ref, C.c_uint8), H, W, T, R,
                       qy, qx, C.byref(a), C.byref(b))
    return a.value, b.value


def cc_project(cc_mode, T, R, Rc, smp, msk, ref_rec, ref_smp, ref_msk, mv, psum=None,
               pcnt=None):
    """Checks + projection for one past frame.  Returns (fmv, dec, psum, pcnt); psum / pcnt
    accumulate into the arrays passed in (new zero arrays if None)."""
    lib = _load()
    smp, msk = _u8(smp), _u8(msk)
    ref_rec, ref_smp, ref_msk = _u8(ref_rec), _u8(ref_smp), _u8(ref_msk)
    H, W = smp.shape
    mv = np.ascontiguousarray(mv, dtype=np.int8)
    fmv = np.zeros_like(mv)
    dec = np.zeros((H, W), dtype=np.uint8)
    psum = np.zeros((H, W), np.uint16) if psum is None else psum
    pcnt = np.zeros((H, W), np.uint8) if pcnt is None else pcnt
    lib.orc_cc_project(cc_mode, T, R, Rc, _p(smp, C.c_uint8), _p(msk, C.c_uint8),
                       _p(ref_rec, C.c_uint8), _p(ref_smp, C.c_uint8), _p(ref_msk, C.c_uint8),
                       H, W, _p(mv, C.c_int8), _p(fmv, C.c_int8), _p(dec, C.c_uint8),
                       _p(psum, C.c_uint16), _p(pcnt, C.c_uint8))
    return fmv, dec, psum, pcnt


def cc_pixel(cc_mode, T, R, Rc, smp, msk, ref_rec, ref_smp, ref_msk, y, x):
    """Decision of a single pixel against one past frame.  Returns (dec, mv, fmv, projected
    sample or -1)."""
    lib = _load()
    H, W = smp.shape
    mv = np.zeros(2, np.int8)
    fmv = np.zeros(2, np.int8)
    pv = C.c_int()
    d = lib.orc_cc_pixel(cc_mode, T, R, Rc, _p(smp, C.c_uint8), _p(msk, C.c_uint8),
                         _p(ref_rec, C.c_uint8), _p(ref_smp, C.c_uint8), _p(ref_msk, C.c_uint8),
                         H, W, y, x, _p(mv, C.c_int8), _p(fmv, C.c_int8), C.byref(pv))
    return d, (int(mv[0]), int(mv[1])), (int(fmv[0]), int(fmv[1])), pv.value


# ----------------------------------------------------------------------------------------------
# FSR and quantisation
# ----------------------------------------------------------------------------------------------
@dataclasses.dataclass
class FsrTrace:
    out: np.ndarray          # (B, B) block output
    w: np.ndarray            # (N, N) support weights
    f: np.ndarray            # (N, N) support values
    g: np.ndarray            # (N, N) model over the support
    R: np.ndarray            # (N, N) complex final residual spectrum
    selected: np.ndarray     # (iterations,) linear bin index per iteration
    min_gap: float
    gaps: np.ndarray         # (iterations,) relative best / second-best gap per iteration


def fsr_block(params: FsrParams, smp, msk, psum, pcnt, by, bx) -> FsrTrace:
    """FSR of block (by, bx) along its own argmax, with every trace."""
    lib = _load()
    smp, msk = _u8(smp), _u8(msk)
    H, W = smp.shape
    psum = None if psum is None else np.ascontiguousarray(psum, np.uint16)
    pcnt = None if pcnt is None else np.ascontiguousarray(pcnt, np.uint8)
    N, B = params.N, params.B
    out = np.zeros((B, B))
    w, f, g = np.zeros((N, N)), np.zeros((N, N)), np.zeros((N, N))
    rre, rim = np.zeros((N, N)), np.zeros((N, N))
    sel = np.zeros(max(1, params.iterations), np.int32)
    gaps = np.zeros(max(1, params.iterations))
    gap = C.c_double()
    cp = params._c()
    lib.orc_fsr_block_ex(C.byref(cp), _p(smp, C.c_uint8), _p(msk, C.c_uint8),
                         _p(psum, C.c_uint16), _p(pcnt, C.c_uint8), H, W, by, bx,
                         _p(out, C.c_double), _p(w, C.c_double), _p(f, C.c_double),
                         _p(g, C.c_double), _p(rre, C.c_double), _p(rim, C.c_double),
                         sel.ctypes.data_as(C.POINTER(C.c_int)), C.byref(gap),
                         _p(gaps, C.c_double))
    return FsrTrace(out, w, f, g, rre + 1j * rim, sel[:params.iterations], gap.value,
                    gaps[:params.iterations])


@dataclasses.dataclass
class Replay:
    """Where a followed selection sequence left this evaluation's own argmax (Sec. 2.1 selects
    one basis pair per iteration): counts, first iteration, and the criterion's relative shortfall
    (best - followed) / best there and at worst; invalid: a followed index is no canonical bin;
    max_scale: 2 S / |R(best)| at the worst divergence, S the magnitude the rounding of the
    residual's arithmetic scales with (largest initial |R| plus the updates made so far);
    max_excess: the largest gap / (bound_q + bound_u * 2 S / |R(best)|) over all divergences, for
    the bound (bound_q, bound_u) given to the replay (0 without one)."""
    iterations_run: int
    divergences: int
    first_div: int
    invalid: bool
    first_gap: float
    max_gap: float
    max_scale: float
    max_excess: float


def _replay(r: _Replay) -> Replay:
    return Replay(r.iterations_run, r.divergences, r.first_div, bool(r.invalid), r.first_gap,
                  r.max_gap, r.max_scale, r.max_excess)


def _bound(bound):
    return None if bound is None else np.ascontiguousarray(bound, np.float64).reshape(2)


def _sel(sel, nblocks: int, iters: int) -> np.ndarray:
    sel = np.ascontiguousarray(sel, np.uint16).reshape(-1)
    assert sel.size == nblocks * max(1, iters), (sel.size, nblocks, iters)
    return sel


def fsr_block_replay(params: FsrParams, smp, msk, psum, pcnt, by, bx, sel, delta: float = 0.0,
                     conc=None, bound=None):
    """FSR of block (by, bx) following the selection sequence sel (``iterations`` uint16 entries,
    0xFFFF = no further iteration) instead of its own argmax, with concealed weighting delta and
    concealed values conc; bound = (bound_q, bound_u) for Replay.max_excess.  Returns (B x B
    output, Replay)."""
    lib = _load()
    smp, msk = _u8(smp), _u8(msk)
    H, W = smp.shape
    psum = None if psum is None else np.ascontiguousarray(psum, np.uint16)
    pcnt = None if pcnt is None else np.ascontiguousarray(pcnt, np.uint8)
    conc = None if conc is None else np.ascontiguousarray(conc, np.float64)
    sel = _sel(sel, 1, params.iterations)
    bound = _bound(bound)
    out = np.zeros((params.B, params.B))
    r = _Replay()
    lib.orc_fsr_block_replay(C.byref(params._c()), float(delta), _p(conc, C.c_double),
                             _p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(psum, C.c_uint16),
                             _p(pcnt, C.c_uint8), H, W, by, bx, _p(sel, C.c_uint16),
                             _p(bound, C.c_double), _p(out, C.c_double), None, None, None,
                             C.byref(r))
    return out, _replay(r)


def fsr_block_concealed(params: FsrParams, delta: float, conc, smp, msk, psum, pcnt, by, bx):
    """FSR of block (by, bx) with concealed weighting delta, the pixels of the blocks before it in
    raster order taking their values from conc (H x W).  Returns (B x B output, min gap, gaps per
    iteration)."""
    lib = _load()
    smp, msk = _u8(smp), _u8(msk)
    H, W = smp.shape
    conc = np.ascontiguousarray(conc, np.float64)
    psum = None if psum is None else np.ascontiguousarray(psum, np.uint16)
    pcnt = None if pcnt is None else np.ascontiguousarray(pcnt, np.uint8)
    out = np.zeros((params.B, params.B))
    gaps = np.zeros(max(1, params.iterations))
    gap = C.c_double()
    lib.orc_fsr_block_replay(C.byref(params._c()), float(delta), _p(conc, C.c_double),
                             _p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(psum, C.c_uint16),
                             _p(pcnt, C.c_uint8), H, W, by, bx, None, None, _p(out, C.c_double),
                             None, C.byref(gap), _p(gaps, C.c_double), None)
    return out, gap.value, gaps[:params.iterations]


def fsr_frame(params: FsrParams, smp, msk, psum=None, pcnt=None):
    """FSR of every block; returns (H x W float64 output, per-block min selection gap)."""
    lib = _load()
    smp, msk = _u8(smp), _u8(msk)
    H, W = smp.shape
    psum = None if psum is None else np.ascontiguousarray(psum, np.uint16)
    pcnt = None if pcnt is None else np.ascontiguousarray(pcnt, np.uint8)
    out = np.zeros((H, W))
    nby, nbx = -(-H // params.B), -(-W // params.B)
    gap = np.zeros((nby, nbx))
    cp = params._c()
    lib.orc_fsr_frame(C.byref(cp), _p(smp, C.c_uint8), _p(msk, C.c_uint8), _p(psum, C.c_uint16),
                      _p(pcnt, C.c_uint8), H, W, _p(out, C.c_double), _p(gap, C.c_double))
    return out, gap


def _replay_arrays(reps) -> dict:
    return {"iterations_run": np.array([r.iterations_run for r in reps], np.int32),
            "divergences": np.array([r.divergences for r in reps], np.int32),
            "first_div": np.array([r.first_div for r in reps], np.int32),
            "invalid": np.array([r.invalid for r in reps], bool),
            "first_gap": np.array([r.first_gap for r in reps]),
            "max_gap": np.array([r.max_gap for r in reps]),
            "max_scale": np.array([r.max_scale for r in reps]),
            "max_excess": np.array([r.max_excess for r in reps])}


def fsr_frame_replay(params: FsrParams, smp, msk, psum, pcnt, sel, bound=None):
    """FSR of every block following the selection sequences sel (nblocks x iterations uint16,
    block-major over the row-major blocks, 0xFFFF = no further iteration).  Returns (H x W
    output, dict of per-block arrays: iterations_run, divergences, first_div, invalid, first_gap,
    max_gap, max_scale, max_excess -- see Replay; bound as in fsr_block_replay)."""
    lib = _load()
    smp, msk = _u8(smp), _u8(msk)
    H, W = smp.shape
    psum = None if psum is None else np.ascontiguousarray(psum, np.uint16)
    pcnt = None if pcnt is None else np.ascontiguousarray(pcnt, np.uint8)
    nby, nbx = -(-H // params.B), -(-W // params.B)
    sel = _sel(sel, nby * nbx, params.iterations)
    bound = _bound(bound)
    out = np.zeros((H, W))
    reps = (_Replay * (nby * nbx))()
    lib.orc_fsr_frame_replay(C.byref(params._c()), _p(smp, C.c_uint8), _p(msk, C.c_uint8),
                             _p(psum, C.c_uint16), _p(pcnt, C.c_uint8), H, W, _p(sel, C.c_uint16),
                             _p(bound, C.c_double), _p(out, C.c_double), None, reps)
    return out, _replay_arrays(reps)


def fsr_frame_concealed(params: FsrParams, delta: float, smp, msk, psum=None, pcnt=None, sel=None,
                        bound=None):
    """FSR of every block in raster order with concealed weighting delta (the original FSR: the
    pixels of earlier blocks that are neither measured nor projected join the support with weight
    delta rho^d); delta = 0 equals fsr_frame.  Returns (H x W output, per-block min gap); with sel
    (nblocks x iterations, as in fsr_frame_replay) every block follows its selection sequence and
    a third element holds the per-block replay arrays."""
    lib = _load()
    smp, msk = _u8(smp), _u8(msk)
    H, W = smp.shape
    psum = None if psum is None else np.ascontiguousarray(psum, np.uint16)
    pcnt = None if pcnt is None else np.ascontiguousarray(pcnt, np.uint8)
    out = np.zeros((H, W))
    nby, nbx = -(-H // params.B), -(-W // params.B)
    gap = np.zeros((nby, nbx))
    cp = params._c()
    if sel is not None:
        sel = _sel(sel, nby * nbx, params.iterations)
    reps = (_Replay * (nby * nbx))() if sel is not None else None
    bound = _bound(bound)
    lib.orc_fsr_frame_concealed(C.byref(cp), float(delta), _p(smp, C.c_uint8), _p(msk, C.c_uint8),
                                _p(psum, C.c_uint16), _p(pcnt, C.c_uint8), H, W,
                                _p(sel, C.c_uint16), _p(bound, C.c_double), _p(out, C.c_double),
                                _p(gap, C.c_double), reps)
    if sel is None:
        return out, gap
    return out, gap, _replay_arrays(reps)


def fsr_support(params: FsrParams, delta: float, conc, smp, msk, psum, pcnt, by, bx):
    """(weights, values) of the N x N support of block (by, bx)."""
    lib = _load()
    smp, msk = _u8(smp), _u8(msk)
    H, W = smp.shape
    conc = None if conc is None else np.ascontiguousarray(conc, np.float64)
    psum = None if psum is None else np.ascontiguousarray(psum, np.uint16)
    pcnt = None if pcnt is None else np.ascontiguousarray(pcnt, np.uint8)
    w = np.zeros((params.N, params.N))
    f = np.zeros((params.N, params.N))
    cp = params._c()
    lib.orc_fsr_support(C.byref(cp), float(delta), _p(conc, C.c_double), _p(smp, C.c_uint8),
                        _p(msk, C.c_uint8), _p(psum, C.c_uint16), _p(pcnt, C.c_uint8), H, W, by, bx,
                        _p(w, C.c_double), _p(f, C.c_double))
    return w, f


def quantize(x, smp, msk) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    smp, msk = _u8(smp), _u8(msk)
    H, W = smp.shape
    out = np.zeros((H, W), np.uint8)
    lib.orc_quantize(_p(x, C.c_double), _p(smp, C.c_uint8), _p(msk, C.c_uint8), H, W,
                     _p(out, C.c_uint8))
    return out


# ----------------------------------------------------------------------------------------------
# one frame step (Fig. 1), given the history
# ----------------------------------------------------------------------------------------------
@dataclasses.dataclass
class StepResult:
    mv: List[np.ndarray]      # per past frame k = 1..K_eff: raw field (H, W, 2)
    fmv: List[np.ndarray]     # vector used by the checks / projection
    dec: List[np.ndarray]     # decision labels
    psum: np.ndarray
    pcnt: np.ndarray
    fsr: np.ndarray           # FSR output in [0, 1] scale (pre-quantisation), float64
    rec: np.ndarray           # 8-bit reconstruction
    min_gap: np.ndarray


def frame_step(smp, msk, history: Sequence[Tuple[np.ndarray, np.ndarray, np.ndarray]],
               cc_mode: int = CC_NNC_FRMC, T: int = 9, R: int = 8, Rc: Optional[int] = None,
               fsr: Optional[FsrParams] = None, run_fsr: bool = True,
               me_predict_radius: int = 0) -> StepResult:
    """history[k-1] = (reconstructed frame, sample plane, mask) of frame t-k, k = 1..K_eff.
    me_predict_radius > 0: past frames t-2.. use the predictive-centre search around k v_1."""
    Rc = R if Rc is None else Rc
    fsr = FsrParams() if fsr is None else fsr
    smp, msk = _u8(smp), _u8(msk)
    H, W = smp.shape
    psum = np.zeros((H, W), np.uint16)
    pcnt = np.zeros((H, W), np.uint8)
    mvs, fmvs, decs = [], [], []
    for k, (rec_k, smp_k, msk_k) in enumerate(history, start=1):
        if me_predict_radius > 0 and k >= 2:
            mv = me_field_predictive(smp, msk, rec_k, T, R, me_predict_radius, k, mvs[0])
        else:
            mv = me_field(smp, msk, rec_k, T, R)
        fmv, dec, psum, pcnt = cc_project(cc_mode, T, R, Rc, smp, msk, rec_k, smp_k, msk_k, mv,
                                          psum, pcnt)
        mvs.append(mv)
        fmvs.append(fmv)
        decs.append(dec)
    if run_fsr:
        out, gap = fsr_frame(fsr, smp, msk, psum, pcnt)
        rec = quantize(out, smp, msk)
    else:
        out, gap, rec = None, None, None
    return StepResult(mvs, fmvs, decs, psum, pcnt, out, rec, gap)
