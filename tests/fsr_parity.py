"""FSR parity by replay: the GPU's FP32 output against the FP64 oracle, block by block.

FSR (Sec. 2.1) selects one basis pair per iteration by an argmax of the weighted residual
energy and then updates the model and the residual with that pair.  Where two pairs' criteria are
within rounding of each other, FP32 and FP64 may select differently, and from there on the two
evaluations follow different (equally valid) continuations of the method.  The GPU therefore
records the pair it selected in every iteration (rfsr_debug_get RFSR_DBG_FSR_SEL, or
rfsr_fsr_device_trace), and the oracle replays exactly that sequence in FP64
(oracle.fsr_frame_replay).  Every block must then satisfy:

  * the GPU's output is within FSR_TOL (1e-4 max abs, [0, 1] scale) of the replay's output;
  * every recorded index is the canonical member of a conjugate pair;
  * at every iteration where the recorded pair is not the FP64 argmax (a divergence), the FP64
    criterion of the recorded pair falls short of the maximum by a relative gap no larger than
    FP32 can explain:  gap <= KEY_QUANTUM + ROUNDING_UNITS * 2^-24 * scale.
    KEY_QUANTUM = 2^-17: the GPU compares criteria with their 5 low mantissa bits replaced by the
    slot index (criteria within 2^-18 relative count as equal and go to the lower index), which
    both the winner's and the loser's key can contribute.  scale = 2 S / |R(best)| (oracle.Replay):
    S is the magnitude the residual's FP32 rounding scales with (the largest initial |R| plus the
    updates made so far), |R(best)| the residual of the FP64 winner, so 2^-24 * scale is one FP32
    rounding unit of S relative to the criterion.  ROUNDING_UNITS = 1: over whole 1920x1080 and
    1280x720 frames of the workloads, 0.15-0.3 % of the blocks diverge, with relative gaps up to
    4.9e-5 (iterations 3..100, scale up to 3900) and never more than 0.65 such units.

Blocks without divergence are then the oracle's own argmax continuation, within FSR_TOL.  The
count of diverged blocks and the worst gap are returned for the record.
"""
from __future__ import annotations

import numpy as np

import oracle

FSR_TOL = 1e-4
KEY_QUANTUM = 2.0 ** -17
ROUNDING_UNITS = 1.0
EPS32 = 2.0 ** -24


BOUND = (KEY_QUANTUM, ROUNDING_UNITS * EPS32)   # gap <= BOUND[0] + BOUND[1] * scale


def check_replay(got, sel, smp, msk, psum, pcnt, params=None, B=4):
    """Assert FSR parity of a whole frame by replay; returns a stats dict."""
    params = params or oracle.FsrParams()
    out, rep = oracle.fsr_frame_replay(params, smp, msk, psum, pcnt, sel, bound=BOUND)
    return check_against(got, out, rep, B=B)


def check_against(got, out, rep, B=4):
    """The rule of this module for a frame replayed with bound=BOUND."""
    H, W = got.shape
    assert not rep["invalid"].any(), f"{int(rep['invalid'].sum())} blocks record a non-canonical bin"
    err = np.abs(got.astype(np.float64) - out)
    nby, nbx = -(-H // B), -(-W // B)
    div = rep["divergences"] > 0
    over = rep["max_excess"] > 1.0
    assert not over.any(), (
        f"{int(over.sum())} blocks diverge at a gap FP32 cannot explain; worst "
        f"{float(rep['max_excess'].max()):.2f} x the bound (block {int(np.argmax(rep['max_excess']))})")
    emax = float(err.max()) if err.size else 0.0
    if emax > FSR_TOL:
        pad = np.zeros((nby * B, nbx * B))
        pad[:H, :W] = err
        eb = pad.reshape(nby, B, nbx, B).max(axis=(1, 3))
        bad = np.argwhere(eb > FSR_TOL)
        raise AssertionError(f"{len(bad)} blocks off the replay by more than {FSR_TOL}: worst "
                             f"{emax:.3e} at block {tuple(int(v) for v in bad[0])}")
    return {"blocks": int(nby * nbx), "diverged": int(div.sum()),
            "max_gap": float(rep["max_gap"][div].max()) if div.any() else 0.0,
            "max_excess": float(rep["max_excess"].max()) if div.any() else 0.0,
            "max_err": emax}


def check_blocks(got, sel, smp, msk, psum, pcnt, blocks, params=None, B=4):
    """check_replay on the listed blocks (by, bx) only (frames too large to replay whole); sel is
    the whole frame's selection plane (nblocks x iterations)."""
    params = params or oracle.FsrParams()
    H, W = got.shape
    nbx = -(-W // B)
    diverged, worst = 0, 0.0
    for by, bx in blocks:
        out, r = oracle.fsr_block_replay(params, smp, msk, psum, pcnt, by, bx, sel[by * nbx + bx],
                                         bound=BOUND)
        assert not r.invalid, (by, bx)
        if r.divergences:
            assert r.max_excess <= 1.0, (by, bx, r)
            diverged += 1
            worst = max(worst, r.max_gap)
        g = got[B * by:B * by + B, B * bx:B * bx + B].astype(np.float64)
        e = float(np.abs(g - out[:g.shape[0], :g.shape[1]]).max())
        assert e <= FSR_TOL, (by, bx, e)
    return {"blocks": len(blocks), "diverged": diverged, "max_gap": worst}
