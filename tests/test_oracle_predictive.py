"""Pins of the oracle's predictive-centre search (an opt-in ME variant that the paper does not
describe): past frame t-k, k >= 2, is searched only within radius Rp of k * v1(p), the
prediction clamped into [-R, R]^2 and into the frame, with the full search's cost and tie order.

The pins do not rest on the oracle's own code: a numpy brute force over every pixel of small
frames, the full search (itself pinned by brute force in test_oracle_pins.py) when the window
covers [-R, R]^2, and the optimality and window invariants on a larger frame.
"""
import numpy as np
import pytest

import oracle
import synth


def _cost_table(smp, msk, ref, T, R):
    """cost[y, x, vy + R, vx + R] by numpy: sum over the T x T template of the measured current
    pixels of |s - rec(clamped p + v + o)| (Sec. 2.2)."""
    H, W = smp.shape
    h = T // 2
    ys, xs = np.mgrid[0:H, 0:W]
    cost = np.zeros((H, W, 2 * R + 1, 2 * R + 1), np.int64)
    for vy in range(-R, R + 1):
        for vx in range(-R, R + 1):
            acc = np.zeros((H, W), np.int64)
            for oy in range(-h, h + 1):
                for ox in range(-h, h + 1):
                    y, x = ys + oy, xs + ox
                    ok = (y >= 0) & (y < H) & (x >= 0) & (x < W)
                    yc, xc = np.clip(y, 0, H - 1), np.clip(x, 0, W - 1)
                    m = ok & (msk[yc, xc] == 1)
                    ry, rx = np.clip(y + vy, 0, H - 1), np.clip(x + vx, 0, W - 1)
                    d = np.abs(smp[yc, xc].astype(np.int64) - ref[ry, rx].astype(np.int64))
                    acc += np.where(m, d, 0)
            cost[:, :, vy + R, vx + R] = acc
    return cost


def _brute_predictive(cost, R, Rp, k, mv1):
    H, W = cost.shape[:2]
    out = np.zeros((H, W, 2), np.int8)
    for y in range(H):
        for x in range(W):
            cy = min(max(k * int(mv1[y, x, 0]), max(-R, -y)), min(R, H - 1 - y))
            cx = min(max(k * int(mv1[y, x, 1]), max(-R, -x)), min(R, W - 1 - x))
            best = None
            for vy in range(cy - Rp, cy + Rp + 1):
                for vx in range(cx - Rp, cx + Rp + 1):
                    if abs(vy) > R or abs(vx) > R or not (0 <= y + vy < H and 0 <= x + vx < W):
                        continue
                    key = (int(cost[y, x, vy + R, vx + R]), abs(vy) + abs(vx), vy, vx)
                    best = key if best is None or key < best else best
            out[y, x] = best[2], best[3]
    return out


def _frames(H, W, seed):
    seq = synth.config2(seed=seed, H=H, W=W, F=3)
    t = 2
    msk = seq.masks[t]
    smp = (seq.frames[t] * msk).astype(np.uint8)
    return smp, msk, seq.frames[t - 2]


@pytest.mark.parametrize("T,R,Rp,k,seed", [(9, 3, 1, 2, 1), (5, 4, 2, 3, 2), (9, 2, 1, 3, 3)])
def test_predictive_brute_force(T, R, Rp, k, seed):
    smp, msk, ref = _frames(24, 20, 300 + seed)
    rng = np.random.default_rng(seed)
    mv1 = rng.integers(-R, R + 1, size=(24, 20, 2)).astype(np.int8)
    got = oracle.me_field_predictive(smp, msk, ref, T, R, Rp, k, mv1)
    want = _brute_predictive(_cost_table(smp, msk, ref, T, R), R, Rp, k, mv1)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("R,k", [(3, 2), (4, 3)])
def test_predictive_full_window_is_full_search(R, k):
    """Rp = 2R: every v in [-R, R]^2 lies in the window, whatever the prediction."""
    smp, msk, ref = _frames(36, 44, 310 + R)
    rng = np.random.default_rng(R)
    mv1 = rng.integers(-R, R + 1, size=(36, 44, 2)).astype(np.int8)
    got = oracle.me_field_predictive(smp, msk, ref, 9, R, 2 * R, k, mv1)
    np.testing.assert_array_equal(got, oracle.me_field(smp, msk, ref, 9, R))


def test_predictive_window_and_optimality():
    """On a larger frame: the vector lies in the clamped window and in the frame, its cost is
    never below the full search's minimum, and equals it where that minimiser is in the window
    (then the vectors agree, the tie order being the same)."""
    H, W, T, R, Rp, k = 48, 64, 9, 4, 1, 2
    smp, msk, ref = _frames(H, W, 320)
    mv1 = oracle.me_field(smp, msk, ref, T, R)          # a realistic t-1 field
    got = oracle.me_field_predictive(smp, msk, ref, T, R, Rp, k, mv1)
    full = oracle.me_field(smp, msk, ref, T, R)
    cost = _cost_table(smp, msk, ref, T, R)
    for y in range(H):
        for x in range(W):
            cy = min(max(k * int(mv1[y, x, 0]), max(-R, -y)), min(R, H - 1 - y))
            cx = min(max(k * int(mv1[y, x, 1]), max(-R, -x)), min(R, W - 1 - x))
            vy, vx = int(got[y, x, 0]), int(got[y, x, 1])
            fy, fx = int(full[y, x, 0]), int(full[y, x, 1])
            assert abs(vy - cy) <= Rp and abs(vx - cx) <= Rp
            assert abs(vy) <= R and abs(vx) <= R and 0 <= y + vy < H and 0 <= x + vx < W
            assert cost[y, x, vy + R, vx + R] >= cost[y, x, fy + R, fx + R]
            if abs(fy - cy) <= Rp and abs(fx - cx) <= Rp:
                assert (vy, vx) == (fy, fx)


def test_frame_step_predictive_first_reference_unchanged():
    """frame_step with the variant keeps t-1's full search and changes only t-2 and later."""
    seq = synth.config1()
    t = 4
    hist = [(seq.frames[t - k], seq.samples[t - k], seq.masks[t - k]) for k in (1, 2, 3)]
    a = oracle.frame_step(seq.samples[t], seq.masks[t], hist, run_fsr=False)
    b = oracle.frame_step(seq.samples[t], seq.masks[t], hist, run_fsr=False, me_predict_radius=2)
    np.testing.assert_array_equal(a.mv[0], b.mv[0])
    for k in (2, 3):
        want = oracle.me_field_predictive(seq.samples[t], seq.masks[t], hist[k - 1][0], 9, 8, 2, k,
                                          a.mv[0])
        np.testing.assert_array_equal(b.mv[k - 1], want)
