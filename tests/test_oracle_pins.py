"""Pins of the CPU oracle against things other than itself (no GPU needed).

Motion estimation and checks: brute force with independent numpy code on tiny frames, closed
forms with a 1x1 template (where the cost is one absolute difference), zero-motion and
known-translation invariants.  NNC: scipy's median filter and closed-form fields.  Projection:
closed forms for static / translated content.  FSR: numpy's FFT, the residual-spectrum invariant,
exact special cases.  Constants: tests/golden/paper_constants.json (each entry cites the paper).
"""
import json
import os

import numpy as np
import pytest
import scipy.ndimage

import oracle
import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


# ------------------------------------------------------------------------------------------------
# independent brute force (numpy) for the template cost and the tie order
# ------------------------------------------------------------------------------------------------
def tie_key(vy, vx):
    return (abs(vy) + abs(vx), vy, vx)


def brute_cost_volume(smp, msk, ref, T, R):
    """cost[vy+R, vx+R, y, x] = masked SAD with replicate-padded reference; n[y, x]."""
    H, W = smp.shape
    h = T // 2
    pad = h + R
    refp = np.pad(ref.astype(np.int64), pad, mode="edge")
    m = msk.astype(np.int64)
    s = smp.astype(np.int64)
    vol = np.zeros((2 * R + 1, 2 * R + 1, H, W), np.int64)
    for vy in range(-R, R + 1):
        for vx in range(-R, R + 1):
            shifted = refp[pad + vy:pad + vy + H, pad + vx:pad + vx + W]
            d = m * np.abs(s - shifted)
            # box sum over the T x T window, zero outside the frame
            dp = np.pad(d, h)
            box = np.zeros((H, W), np.int64)
            for oy in range(T):
                for ox in range(T):
                    box += dp[oy:oy + H, ox:ox + W]
            vol[vy + R, vx + R] = box
    mp = np.pad(m, h)
    n = np.zeros((H, W), np.int64)
    for oy in range(T):
        for ox in range(T):
            n += mp[oy:oy + H, ox:ox + W]
    return vol, n


def brute_me(smp, msk, ref, T, R):
    H, W = smp.shape
    vol, _ = brute_cost_volume(smp, msk, ref, T, R)
    out = np.zeros((H, W, 2), np.int8)
    cands = sorted([(vy, vx) for vy in range(-R, R + 1) for vx in range(-R, R + 1)],
                   key=lambda v: tie_key(*v))
    for y in range(H):
        for x in range(W):
            best = None
            for vy, vx in cands:
                if not (0 <= y + vy < H and 0 <= x + vx < W):
                    continue
                c = vol[vy + R, vx + R, y, x]
                if best is None or c < best[0]:
                    best = (c, vy, vx)
            out[y, x] = best[1], best[2]
    return out


@pytest.mark.parametrize("seed,H,W,T,R,levels", [
    (0, 12, 14, 5, 3, 256), (1, 9, 11, 3, 2, 2), (2, 16, 10, 9, 4, 3), (3, 7, 7, 3, 3, 256),
    (4, 14, 12, 5, 2, 1),
])
def test_me_field_matches_brute_force(seed, H, W, T, R, levels):
    """Dense ME equals an independent enumeration; few grey levels force many ties."""
    rng = np.random.default_rng(seed)
    frame = rng.integers(0, levels, size=(H, W)).astype(np.uint8) * (255 // max(1, levels - 1))
    ref = rng.integers(0, levels, size=(H, W)).astype(np.uint8) * (255 // max(1, levels - 1))
    msk = synth.positions_to_mask(synth.fixed_positions(H + H % 2, W + W % 2, rng))[:H, :W]
    smp = frame * msk
    got = oracle.me_field(smp, msk, ref, T, R)
    np.testing.assert_array_equal(got, brute_me(smp, msk, ref, T, R))


def test_cost_matches_brute_force_including_borders():
    rng = np.random.default_rng(7)
    H, W, T, R = 10, 13, 5, 3
    ref = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    msk = (rng.random((H, W)) < 0.4).astype(np.uint8)
    smp = (rng.integers(0, 256, size=(H, W)) * msk).astype(np.uint8)
    vol, n = brute_cost_volume(smp, msk, ref, T, R)
    for (y, x, vy, vx) in [(0, 0, -3, -3), (9, 12, 3, 3), (5, 6, 0, 0), (0, 12, 2, -1),
                           (4, 0, -2, 3)]:
        assert oracle.cost(smp, msk, ref, T, y, x, vy, vx) == (vol[vy + R, vx + R, y, x],
                                                               n[y, x])


def test_normalised_order_and_tie_order():
    # 10/20 = 0.5 beats 6/10 = 0.6 although its SAD is larger
    assert oracle.better((10, 20, 3, 3), (6, 10, 0, 0))
    assert not oracle.better((6, 10, 0, 0), (10, 20, 3, 3))
    # equal means: tie order |v|_1, then vy, then vx
    assert oracle.better((5, 10, 0, 1), (10, 20, 1, 1))
    assert oracle.better((5, 10, -1, 0), (5, 10, 0, -1))
    assert oracle.better((5, 10, 0, -1), (5, 10, 0, 1))
    assert oracle.better((5, 10, 1, 0), (5, 10, -1, -1))
    assert not oracle.better((5, 10, 0, 0), (5, 10, 0, 0))


def test_me_template1_closed_form():
    """With a 1x1 template the cost is |s(p) - ref(p+v)|: the vector goes to the nearest grey
    value, ties in tie order, and unmeasured pixels (cost 0 everywhere) get v = 0."""
    H = W = 9
    ref = np.full((H, W), 200, np.uint8)
    ref[6, 2] = 101           # p + (2, -2)  |diff| = 1
    ref[2, 6] = 99            # p + (-2, 2)  |diff| = 1, same |v|_1, smaller vy -> wins
    ref[4, 1] = 97
    msk = np.zeros((H, W), np.uint8)
    msk[4, 4] = 1
    smp = np.zeros((H, W), np.uint8)
    smp[4, 4] = 100
    assert oracle.me_pixel(smp, msk, ref, 1, 4, 4, 4) == (-2, 2)
    ref[5, 4] = 100           # exact match at (1, 0)
    assert oracle.me_pixel(smp, msk, ref, 1, 4, 4, 4) == (1, 0)
    assert oracle.me_pixel(smp, msk, ref, 1, 4, 0, 0) == (0, 0)   # unmeasured pixel


def test_me_zero_motion():
    s = synth.config1(seed=11, F=2)
    frame, msk = s.frames[0], s.masks[0]
    mv = oracle.me_field(frame * msk, msk, frame, 9, 8)
    assert not mv.any()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_me_recovers_known_translation(k):
    """Content moves (+2 rows, +1 col) per frame: against the true frame t-k the vector is
    (-2k, -k) at every pixel whose window stays inside the frame."""
    s = synth.config1(seed=1, F=4)
    t = 3
    smp, msk = s.samples[t], s.masks[t]
    T, R = 9, 8
    m = T // 2 + R + 1
    H, W = smp.shape
    for y in range(m, H - m, 3):
        for x in range(m, W - m, 3):
            assert oracle.me_pixel(smp, msk, s.frames[t - k], T, R, y, x) == (-2 * k, -k)


# ------------------------------------------------------------------------------------------------
# NNC, Eq. (1)
# ------------------------------------------------------------------------------------------------
def test_nnc_median_is_scipy_median():
    rng = np.random.default_rng(3)
    mv = rng.integers(-8, 9, size=(13, 17, 2)).astype(np.int8)
    fmv, _ = oracle.nnc_field(mv)
    for c in range(2):
        ref = scipy.ndimage.median_filter(mv[..., c], size=GOLDEN["nnc_median"]["value"],
                                          mode="nearest")
        np.testing.assert_array_equal(fmv[..., c], ref)


def test_nnc_pass_closed_forms():
    H, W = 8, 10
    const = np.zeros((H, W, 2), np.int8)
    const[...] = (3, -2)
    _, ok = oracle.nnc_field(const)
    assert ok.all()
    # vertical edge of size 1 in vy: every pair differs by <= 1 -> all pass
    step1 = np.zeros((H, W, 2), np.int8)
    step1[:, 5:, 0] = 1
    _, ok = oracle.nnc_field(step1)
    assert ok.all()
    # edge of size 2: exactly the two columns beside the edge fail
    step2 = np.zeros((H, W, 2), np.int8)
    step2[:, 5:, 0] = 2
    _, ok = oracle.nnc_field(step2)
    expect = np.ones((H, W), np.uint8)
    expect[:, 4:6] = 0
    np.testing.assert_array_equal(ok, expect)
    # diagonal change (1, 1): L1 distance 2 -> fails across the edge
    diag = np.zeros((H, W, 2), np.int8)
    diag[4:, :, :] = 1
    _, ok = oracle.nnc_field(diag)
    expect = np.ones((H, W), np.uint8)
    expect[3:5, :] = 0
    np.testing.assert_array_equal(ok, expect)
    # an isolated outlier is removed by the median and does not fail anyone
    iso = np.zeros((H, W, 2), np.int8)
    iso[4, 4] = (7, -7)
    fmv, ok = oracle.nnc_field(iso)
    assert not fmv.any() and ok.all()


def test_nnc_threshold_and_neighbours_from_paper():
    assert GOLDEN["nnc_threshold"]["value"] == 1
    # a diagonal neighbour difference is not checked (only the four nearest neighbours)
    H, W = 9, 9
    mv = np.zeros((H, W, 2), np.int8)
    mv[5:, 5:, 1] = 2      # a 4x4 corner block with vx = 2
    fmv, ok = oracle.nnc_field(mv)
    # after the median the corner block keeps vx = 2 except its own corner pixel (5, 5)
    for y in range(H):
        for x in range(W):
            nbrs = [(y + dy, x + dx) for dy, dx in GOLDEN["nnc_neighbours"]["value"]
                    if 0 <= y + dy < H and 0 <= x + dx < W]
            exp = all(abs(int(fmv[y, x, 0]) - int(fmv[a, b, 0])) +
                      abs(int(fmv[y, x, 1]) - int(fmv[a, b, 1])) <= 1 for a, b in nbrs)
            assert ok[y, x] == exp


# ------------------------------------------------------------------------------------------------
# reverse checks: 1x1 template constructions pin the candidate sets exactly
# ------------------------------------------------------------------------------------------------
def _one_pixel_scene(dstar, H=21, W=21):
    """All pixels measured; s(p) = 100, ref(q) = 90, s(p + d*) = 90, everything else 200.
    With a 1x1 template the reverse cost of candidate d is |s(p + d) - ref(q)|: the centre costs
    10, d* costs 0, all others 110.  So a check rejects iff it tests d*."""
    p = (10, 10)
    v = (1, -2)
    q = (p[0] + v[0], p[1] + v[1])
    msk = np.ones((H, W), np.uint8)
    smp = np.full((H, W), 200, np.uint8)
    ref = np.full((H, W), 0, np.uint8)
    smp[p] = 100
    ref[q] = 90
    if dstar is not None:
        smp[p[0] + dstar[0], p[1] + dstar[1]] = 90
    return smp, msk, ref, p, v


def test_frmc_candidate_set_is_the_papers():
    offs = set(GOLDEN["frmc_offsets"]["value"])
    assert len(offs) ** 2 == GOLDEN["frmc_count"]["value"]
    smp, msk, ref, p, v = _one_pixel_scene(None)
    assert oracle.check_frmc(smp, msk, ref, 1, p[0], p[1], v[0], v[1])
    for dy in range(-8, 9):
        for dx in range(-8, 9):
            if (dy, dx) == (0, 0):
                continue
            smp, msk, ref, p, v = _one_pixel_scene((dy, dx))
            acc = oracle.check_frmc(smp, msk, ref, 1, p[0], p[1], v[0], v[1])
            assert acc == (not (dy in offs and dx in offs)), (dy, dx)


@pytest.mark.parametrize("Rc", [2, 7, 8])
def test_rmc_candidate_set_is_the_full_window(Rc):
    for dy in range(-9, 10):
        for dx in range(-9, 10):
            if (dy, dx) == (0, 0):
                continue
            smp, msk, ref, p, v = _one_pixel_scene((dy, dx))
            acc = oracle.check_rmc(smp, msk, ref, 1, Rc, p[0], p[1], v[0], v[1])
            assert acc == (max(abs(dy), abs(dx)) > Rc), (dy, dx)


def test_reverse_check_centre_wins_ties():
    smp, msk, ref, p, v = _one_pixel_scene((3, 3))
    smp[13, 13] = 100        # d* now costs exactly the centre's 10
    assert oracle.check_frmc(smp, msk, ref, 1, p[0], p[1], v[0], v[1])
    assert oracle.check_rmc(smp, msk, ref, 1, 8, p[0], p[1], v[0], v[1])


def test_rme_closed_form_and_tie_order():
    """1x1 template: the reverse vector at q goes to the source whose sample is closest to
    ref(q); equal costs follow the tie order on w."""
    smp, msk, ref, p, v = _one_pixel_scene(None)
    q = (p[0] + v[0], p[1] + v[1])
    assert oracle.rme_vector(smp, msk, ref, 1, 8, *q) == (p[0] - q[0], p[1] - q[1])
    assert oracle.check_rme(smp, msk, ref, 1, 8, p[0], p[1], v[0], v[1])
    smpd, _, _, _, _ = _one_pixel_scene((2, 0))      # a better source two rows below p
    assert oracle.rme_vector(smpd, msk, ref, 1, 8, *q) == (p[0] + 2 - q[0], p[1] - q[1])
    assert not oracle.check_rme(smpd, msk, ref, 1, 8, p[0], p[1], v[0], v[1])
    smp2 = smp.copy()
    smp2[p] = 90
    smp3 = smp2.copy()
    smp3[q[0] - 1, q[1]] = 90     # w = (-1, 0): |w|_1 = 1 < |-v|_1 = 3 -> wins the tie
    assert oracle.rme_vector(smp3, msk, ref, 1, 8, *q) == (-1, 0)
    assert not oracle.check_rme(smp3, msk, ref, 1, 8, p[0], p[1], v[0], v[1])


def brute_rme(smp, msk, ref, T, R, qy, qx):
    """Reverse vector by enumerating (mean cost, tie key) with exact fractions."""
    from fractions import Fraction
    H, W = smp.shape
    vol, n = brute_cost_volume(smp, msk, ref, T, R)
    best = None
    for wy in range(-R, R + 1):
        for wx in range(-R, R + 1):
            sy, sx = qy + wy, qx + wx
            if not (0 <= sy < H and 0 <= sx < W):
                continue
            c = Fraction(int(vol[-wy + R, -wx + R, sy, sx]), int(n[sy, sx]))
            key = (c, tie_key(wy, wx))
            if best is None or key < best[0]:
                best = (key, (wy, wx))
    return best[1]


def test_rme_matches_brute_force_with_normalisation():
    rng = np.random.default_rng(5)
    H, W, T, R = 11, 12, 3, 2
    msk = (rng.random((H, W)) < 0.5).astype(np.uint8)
    msk[0, 0] = 1
    smp = (rng.integers(0, 4, size=(H, W)) * 60 * msk).astype(np.uint8)
    ref = (rng.integers(0, 4, size=(H, W)) * 60).astype(np.uint8)
    for qy in range(H):
        for qx in range(W):
            # every template must contain a measured pixel for the mean to be defined
            _, n = brute_cost_volume(smp, msk, ref, T, R)
            if (n == 0).any():
                pytest.skip("degenerate draw")
            assert oracle.rme_vector(smp, msk, ref, T, R, qy, qx) == \
                brute_rme(smp, msk, ref, T, R, qy, qx)


def test_rmc_accept_implies_frmc_accept():
    """FRMC tests a subset of RMC's candidates (Rc >= 7), so RMC-accept implies FRMC-accept."""
    s = synth.config2(seed=9, H=48, W=64, F=4)
    t = 3
    smp, msk = s.samples[t], s.masks[t]
    ref = s.frames[t - 1]
    rng = np.random.default_rng(0)
    for _ in range(60):
        y, x = int(rng.integers(0, 48)), int(rng.integers(0, 64))
        vy, vx = oracle.me_pixel(smp, msk, ref, 9, 8, y, x)
        vy, vx = vy + int(rng.integers(-2, 3)), vx + int(rng.integers(-2, 3))
        if not (0 <= y + vy < 48 and 0 <= x + vx < 64):
            continue
        if oracle.check_rmc(smp, msk, ref, 9, 8, y, x, vy, vx):
            assert oracle.check_frmc(smp, msk, ref, 9, y, x, vy, vx)


# ------------------------------------------------------------------------------------------------
# projection
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["none", "rme", "rmc", "frmc", "nnc", "nnc_frmc"])
def test_fixed_mask_static_scene_projects_nothing(mode):
    s = synth.config2(seed=3, H=32, W=40, F=4, mask_type=synth.MASK_FIXED)
    frame = s.frames[0]
    msk = s.masks[0]
    smp = frame * msk
    hist = [(frame, smp, msk)] * 3
    r = oracle.frame_step(smp, msk, hist, cc_mode=oracle.CC_NAMES[mode], T=9, R=4,
                          run_fsr=False)
    assert not r.pcnt.any()
    for d in r.dec:
        assert set(np.unique(d)) <= {oracle.DEC_MEASURED, oracle.DEC_NOT_PROJECTABLE}
        np.testing.assert_array_equal(d == oracle.DEC_MEASURED, msk == 1)


@pytest.mark.parametrize("mode", ["none", "rme", "rmc", "frmc", "nnc", "nnc_frmc"])
def test_dynamic_mask_static_scene_fills_every_missing_pixel_once(mode):
    """With a dynamic mask each pixel is measured once in any four consecutive frames, so with
    zero motion the three previous frames project exactly one true sample into every missing
    pixel."""
    s = synth.config2(seed=4, H=32, W=40, F=4)
    frame = s.frames[0]
    t = 3
    masks = [s.masks[i] for i in range(4)]
    smp = frame * masks[t]
    hist = [(frame, frame * masks[t - k], masks[t - k]) for k in (1, 2, 3)]
    r = oracle.frame_step(smp, masks[t], hist, cc_mode=oracle.CC_NAMES[mode], T=9, R=4,
                          run_fsr=False)
    missing = masks[t] == 0
    np.testing.assert_array_equal(r.pcnt[missing], 1)
    np.testing.assert_array_equal(r.pcnt[~missing], 0)
    np.testing.assert_array_equal(r.psum[missing], frame[missing])


def test_translation_projection_averages_true_values():
    """Known translation, true past frames, no check: every accepted projection carries the
    true value of the current pixel, so psum = pcnt * f(p) in the interior."""
    s = synth.config1(seed=1, F=4)
    t = 3
    smp, msk = s.samples[t], s.masks[t]
    hist = [(s.frames[t - k], s.samples[t - k], s.masks[t - k]) for k in (1, 2, 3)]
    r = oracle.frame_step(smp, msk, hist, cc_mode=oracle.CC_NONE, T=9, R=8, run_fsr=False)
    m = 13
    f = s.frames[t].astype(np.int64)
    inner = (slice(m, -m), slice(m, -m))
    np.testing.assert_array_equal(r.psum[inner].astype(np.int64),
                                  r.pcnt[inner].astype(np.int64) * f[inner])
    assert r.pcnt[inner].max() >= 1


# ------------------------------------------------------------------------------------------------
# FSR
# ------------------------------------------------------------------------------------------------
P0 = oracle.FsrParams()


def _block_scene(H=64, W=64, seed=0, fn=None, mask=None):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    img = fn(y, x) if fn is not None else rng.random((H, W))
    msk = mask if mask is not None else synth.positions_to_mask(synth.fixed_positions(H, W, rng))
    smp = np.clip(np.rint(img * 255), 0, 255).astype(np.uint8) * msk
    return img, smp.astype(np.uint8), msk.astype(np.uint8)


def test_fsr_spectra_are_numpy_fft():
    _, smp, msk = _block_scene(seed=1)
    tr = oracle.fsr_block(oracle.FsrParams(iterations=0), smp, msk, None, None, 7, 6)
    np.testing.assert_allclose(tr.R, np.fft.fft2(tr.w * tr.f), atol=1e-11)


def test_fsr_weights_closed_form():
    _, smp, msk = _block_scene(seed=2)
    by, bx = 7, 6
    tr = oracle.fsr_block(P0, smp, msk, None, None, by, bx)
    N, B = P0.N, P0.B
    o = (N - B) // 2
    c = (N - 1) / 2
    for m in range(N):
        for n in range(N):
            yy, xx = B * by - o + m, B * bx - o + n
            inside = 0 <= yy < 64 and 0 <= xx < 64
            known = inside and msk[yy, xx]
            exp = P0.rho ** np.hypot(m - c, n - c) if known else 0.0
            assert tr.w[m, n] == pytest.approx(exp, rel=1e-12, abs=0)


def test_fsr_residual_invariant():
    """After every iteration the residual spectrum equals the DFT of w * (f - g) with g the
    model evaluated over the support: pins the W(k-u) / W(k+u) update and the model update."""
    _, smp, msk = _block_scene(seed=3)
    for it in (1, 2, 7, 40):
        tr = oracle.fsr_block(oracle.FsrParams(iterations=it), smp, msk, None, None, 5, 9)
        np.testing.assert_allclose(tr.R, np.fft.fft2(tr.w * (tr.f - tr.g)), atol=1e-9)


def test_fsr_selection_rule():
    """The first bin maximises wf * |DFT(w f)|^2 over canonical members of conjugate pairs."""
    _, smp, msk = _block_scene(seed=4)
    tr = oracle.fsr_block(oracle.FsrParams(iterations=1), smp, msk, None, None, 3, 3)
    N = P0.N
    tr0 = oracle.fsr_block(oracle.FsrParams(iterations=0), smp, msk, None, None, 3, 3)
    k = np.arange(N)
    kn = np.minimum(k, N - k) / (N / 2)
    wf = (1 - np.sqrt(2) / 2 * np.sqrt(kn[:, None] ** 2 + kn[None, :] ** 2)) ** 2
    e = wf * np.abs(tr0.R) ** 2
    lin = k[:, None] * N + k[None, :]
    conj = ((N - k[:, None]) % N) * N + (N - k[None, :]) % N
    e = np.where(lin <= conj, e, -1)
    assert tr.selected[0] == int(np.argmax(e))


def test_fsr_fully_sampled_block_unchanged():
    img, _, _ = _block_scene(seed=5)
    msk = np.ones((64, 64), np.uint8)
    smp = np.clip(np.rint(img * 255), 0, 255).astype(np.uint8)
    tr = oracle.fsr_block(P0, smp, msk, None, None, 4, 4)
    np.testing.assert_array_equal(tr.out, smp[16:20, 16:20] / 255.0)


def test_fsr_constant_block_recovered():
    _, smp, msk = _block_scene(fn=lambda y, x: np.full(y.shape, 0.4))
    out, _ = oracle.fsr_frame(P0, smp, msk)
    v = np.rint(0.4 * 255) / 255
    np.testing.assert_allclose(out, v, atol=1e-6)


@pytest.mark.parametrize("u", [(1, 2), (3, 0), (2, 5)])
def test_fsr_single_basis_function_recovered(u):
    """A single real DFT basis function (period 32, amplitude 0.4 around 0.5) sampled on a
    quarter mask is recovered to 1e-4 in the interior blocks (exact, unquantised samples)."""
    N = 32
    H = W = 64
    f = lambda y, x: 0.5 + 0.4 * np.cos(2 * np.pi * (u[0] * y + u[1] * x) / N + 0.3)
    rng = np.random.default_rng(1)
    msk = synth.positions_to_mask(synth.fixed_positions(H, W, rng))
    y, x = np.mgrid[0:H, 0:W]
    img = f(y, x)
    # feed exact values through the projection channel (psum / (255 pcnt) with pcnt = 255):
    # the 8-bit sample channel would quantise; here the known values are exact to 1/65025
    psum = np.clip(np.rint(img * 255 * 255), 0, 65535).astype(np.uint16)
    pcnt = np.full((H, W), 255, np.uint8)
    known = msk.astype(bool)
    pcnt[~known] = 0
    psum[~known] = 0
    zero = np.zeros((H, W), np.uint8)
    params = oracle.FsrParams(iterations=200)
    for by, bx in [(6, 6), (8, 7), (5, 9)]:
        tr = oracle.fsr_block(params, zero, zero, psum, pcnt, by, bx)
        ref = img[4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
        np.testing.assert_allclose(tr.out, ref, atol=1e-4)


def test_fsr_overwrite_rules():
    """D-FSR overwrites only measured pixels; R-FSR also overwrites projected ones (Sec. 3.2)."""
    img, smp, msk = _block_scene(seed=6)
    H, W = msk.shape
    psum = np.zeros((H, W), np.uint16)
    pcnt = np.zeros((H, W), np.uint8)
    psum[20, 21], pcnt[20, 21] = 2 * 17, 2       # projected value 17 / 255
    msk[20, 21] = 0
    smp[20, 21] = 0
    d = oracle.fsr_block(P0, smp, msk, psum, pcnt, 5, 5)
    r = oracle.fsr_block(oracle.FsrParams(overwrite_projected=True), smp, msk, psum, pcnt, 5, 5)
    assert r.out[0, 1] == 17 / 255
    assert d.out[0, 1] != 17 / 255
    for m in range(4):
        for n in range(4):
            if msk[20 + m, 20 + n]:
                assert d.out[m, n] == smp[20 + m, 20 + n] / 255


def test_fsr_border_block_ignores_outside():
    _, smp, msk = _block_scene(seed=7)
    tr = oracle.fsr_block(P0, smp, msk, None, None, 0, 0)
    o = (P0.N - P0.B) // 2
    assert not tr.w[:o, :].any() and not tr.w[:, :o].any()


def _canonical_energy(R, N=32):
    """wf |R|^2 over canonical members of conjugate pairs (-1 elsewhere), written out in numpy."""
    k = np.arange(N)
    kn = np.minimum(k, N - k) / (N / 2)
    wf = (1 - np.sqrt(2) / 2 * np.sqrt(kn[:, None] ** 2 + kn[None, :] ** 2)) ** 2
    lin = k[:, None] * N + k[None, :]
    conj = ((N - k[:, None]) % N) * N + (N - k[None, :]) % N
    return np.where(lin <= conj, wf * np.abs(R) ** 2, -1.0).ravel()


def test_fsr_replay_of_its_own_selections_is_the_plain_run():
    """Replaying the oracle's own selection sequence gives its own output bit for bit, with no
    divergence, block by block and over a frame."""
    _, smp, msk = _block_scene(seed=8)
    tr = oracle.fsr_block(P0, smp, msk, None, None, 6, 5)
    out, rep = oracle.fsr_block_replay(P0, smp, msk, None, None, 6, 5,
                                       tr.selected.astype(np.uint16))
    np.testing.assert_array_equal(out, tr.out)
    assert rep.divergences == 0 and rep.first_div == -1 and not rep.invalid
    assert rep.iterations_run == P0.iterations
    plain, _ = oracle.fsr_frame(P0, smp, msk)
    nb = 16 * 16
    sel = np.stack([oracle.fsr_block(P0, smp, msk, None, None, b // 16, b % 16).selected
                    for b in range(nb)]).astype(np.uint16)
    rout, reps = oracle.fsr_frame_replay(P0, smp, msk, None, None, sel)
    np.testing.assert_array_equal(rout, plain)
    assert not reps["divergences"].any()


@pytest.mark.parametrize("it", [0, 9, 37])
def test_fsr_replay_follows_a_second_best_selection(it):
    """Forcing the second-best pair at iteration `it`: the replay reports its first divergence
    there, with the criterion gap (best - second) / best of the residual after `it` iterations,
    computed here from the oracle's residual spectrum by numpy; the output changes."""
    _, smp, msk = _block_scene(seed=9)
    by, bx = 7, 8
    tr = oracle.fsr_block(P0, smp, msk, None, None, by, bx)
    Rit = oracle.fsr_block(oracle.FsrParams(iterations=it), smp, msk, None, None, by, bx).R
    e = _canonical_energy(Rit)
    order = np.argsort(-e, kind="stable")
    assert order[0] == tr.selected[it]
    follow = tr.selected.astype(np.uint16).copy()
    follow[it] = order[1]
    out, rep = oracle.fsr_block_replay(P0, smp, msk, None, None, by, bx, follow,
                                       bound=(2.0 ** -17, 2.0 ** -24))
    assert rep.first_div == it and rep.divergences >= 1 and not rep.invalid
    gap = (e[order[0]] - e[order[1]]) / e[order[0]]
    assert rep.first_gap == pytest.approx(gap, rel=1e-9)
    assert rep.max_gap >= rep.first_gap
    assert rep.max_excess >= rep.first_gap / (2.0 ** -17 + 2.0 ** -24 * rep.max_scale) * (1 - 1e-12)
    assert np.abs(out - tr.out).max() > 0


def test_fsr_replay_stops_at_no_selection_and_flags_bad_indices():
    """0xFFFF at iteration i ends the replay there: the output equals i plain iterations.  A
    selection that is not the canonical member of its conjugate pair is flagged invalid."""
    _, smp, msk = _block_scene(seed=10)
    tr = oracle.fsr_block(P0, smp, msk, None, None, 5, 6)
    follow = tr.selected.astype(np.uint16).copy()
    follow[12:] = 0xFFFF
    out, rep = oracle.fsr_block_replay(P0, smp, msk, None, None, 5, 6, follow)
    assert rep.iterations_run == 12 and rep.divergences == 0
    np.testing.assert_array_equal(
        out, oracle.fsr_block(oracle.FsrParams(iterations=12), smp, msk, None, None, 5, 6).out)
    bad = tr.selected.astype(np.uint16).copy()
    k, l = divmod(int(bad[3]), 32)
    conj = ((32 - k) % 32) * 32 + (32 - l) % 32
    if conj != bad[3]:                              # the other member of the pair
        bad[3] = conj
        _, rep = oracle.fsr_block_replay(P0, smp, msk, None, None, 5, 6, bad)
        assert rep.invalid
    bad[3] = 32 * 32                                # outside the spectrum
    _, rep = oracle.fsr_block_replay(P0, smp, msk, None, None, 5, 6, bad)
    assert rep.invalid


def test_quantize_rounding():
    x = np.array([[2.5, 3.5, -0.2, 300.0, 0.1, 17.0]]) / 255.0
    msk = np.array([[0, 0, 0, 0, 0, 1]], np.uint8)
    smp = np.array([[0, 0, 0, 0, 0, 9]], np.uint8)
    np.testing.assert_array_equal(oracle.quantize(x, smp, msk), [[2, 4, 0, 255, 0, 9]])


# ------------------------------------------------------------------------------------------------
# generators (quarter sampling, Sec. 1)
# ------------------------------------------------------------------------------------------------
def test_masks_quarter_sampling():
    s = synth.config2(seed=1, H=32, W=48, F=9)
    m = s.masks.astype(np.int64)
    blocks = m.reshape(9, 16, 2, 24, 2).sum(axis=(2, 4))
    assert (blocks == GOLDEN["measured_per_block"]["value"]).all()
    per = GOLDEN["dynamic_mask_period"]["value"]
    for t in range(9 - per + 1):
        assert (m[t:t + per].sum(0) == 1).all()
    np.testing.assert_array_equal(m[0], m[per])
    f = synth.config1(seed=1, F=3)
    np.testing.assert_array_equal(f.masks[0], f.masks[2])


def test_openmp_build_gives_identical_results():
    """The -fopenmp build (frame loops over independent pixels and blocks on several threads)
    returns bit-identical fields, decisions, projections and FSR output."""
    seq = synth.config2(seed=9, H=48, W=64, F=4)
    t = 3
    smp, msk = seq.samples[t], seq.masks[t]
    hist = [(seq.frames[t - k], seq.samples[t - k], seq.masks[t - k]) for k in (1, 2, 3)]
    fsr = oracle.FsrParams(iterations=20)
    out = {}
    try:
        for n in (1, 4):
            oracle.set_threads(n)
            out[n] = [oracle.frame_step(smp, msk, hist, cc_mode=oracle.CC_NAMES[m], T=7, R=4,
                                        fsr=fsr) for m in ("nnc_frmc", "rmc", "rme")]
    finally:
        oracle.set_threads(1)
    for a, b in zip(out[1], out[4]):
        for k in range(3):
            np.testing.assert_array_equal(a.mv[k], b.mv[k])
            np.testing.assert_array_equal(a.fmv[k], b.fmv[k])
            np.testing.assert_array_equal(a.dec[k], b.dec[k])
        np.testing.assert_array_equal(a.psum, b.psum)
        np.testing.assert_array_equal(a.pcnt, b.pcnt)
        np.testing.assert_array_equal(a.fsr, b.fsr)
        np.testing.assert_array_equal(a.rec, b.rec)


# --------------------------------------------------------------------------------------------
# concealed weighting delta > 0 (the original FSR; the paper uses 0, Sec. 4)
# --------------------------------------------------------------------------------------------
def _conc_inputs(H=40, W=44, seed=12):
    seq = synth.config2(seed=seed, H=H, W=W, F=1)
    smp, msk = seq.samples[0], seq.masks[0]
    rng = np.random.default_rng(seed)
    pcnt = np.where((msk == 0) & (rng.random((H, W)) < 0.3), 1, 0).astype(np.uint8)
    psum = (pcnt.astype(np.uint16) * seq.frames[0]).astype(np.uint16)
    return seq, smp, msk, psum, pcnt


def test_concealed_support_follows_its_definition():
    """Weights: rho^d measured, mu rho^d projected, delta rho^d for the pixels of earlier blocks
    (raster order) that are neither, 0 otherwise -- built here independently in numpy."""
    seq, smp, msk, psum, pcnt = _conc_inputs()
    H, W = smp.shape
    P = oracle.FsrParams(proj_weight=0.8)
    delta = 0.37
    conc = np.random.default_rng(1).random((H, W))
    for by, bx in [(0, 0), (3, 5), (9, 10), (4, 0)]:
        w, f = oracle.fsr_support(P, delta, conc, smp, msk, psum, pcnt, by, bx)
        N, B, o = P.N, P.B, (P.N - P.B) // 2
        cc = (N - 1) / 2.0
        for m in range(N):
            for n in range(N):
                y, x = B * by - o + m, B * bx - o + n
                d = np.hypot(m - cc, n - cc)
                ew, ef = 0.0, 0.0
                if 0 <= y < H and 0 <= x < W:
                    earlier = y // B < by or (y // B == by and x // B < bx)
                    if msk[y, x]:
                        ew, ef = P.rho ** d, smp[y, x] / 255.0
                    elif pcnt[y, x]:
                        ew, ef = P.proj_weight * P.rho ** d, psum[y, x] / (255.0 * pcnt[y, x])
                    elif earlier:
                        ew, ef = delta * P.rho ** d, conc[y, x]
                assert abs(w[m, n] - ew) < 1e-12 and abs(f[m, n] - ef) < 1e-12, (by, bx, m, n)


def test_concealed_zero_delta_equals_parallel_fsr():
    seq, smp, msk, psum, pcnt = _conc_inputs()
    P = oracle.FsrParams(iterations=30)
    a, _ = oracle.fsr_frame(P, smp, msk, psum, pcnt)
    b, _ = oracle.fsr_frame_concealed(P, 0.0, smp, msk, psum, pcnt)
    np.testing.assert_array_equal(a, b)


def test_concealed_first_block_and_constant_frame():
    seq, smp, msk, psum, pcnt = _conc_inputs()
    P = oracle.FsrParams(iterations=30)
    a, _ = oracle.fsr_frame(P, smp, msk, psum, pcnt)
    b, _ = oracle.fsr_frame_concealed(P, 0.5, smp, msk, psum, pcnt)
    np.testing.assert_array_equal(a[:4, :4], b[:4, :4])      # block (0, 0) has nothing earlier
    assert np.abs(a - b).max() > 1e-6                         # later blocks see concealed pixels
    flat = np.full(smp.shape, 90, np.uint8)
    c, _ = oracle.fsr_frame_concealed(P, 0.5, (flat * msk).astype(np.uint8), msk)
    np.testing.assert_allclose(c, 90 / 255.0, atol=1e-12)


def test_concealed_block_reads_only_earlier_blocks():
    """A block of the raster-order frame equals the block computed alone from the frame's final
    output, and values of the block itself or of later blocks in conc change nothing."""
    seq, smp, msk, psum, pcnt = _conc_inputs()
    P = oracle.FsrParams(iterations=30)
    delta = 0.5
    out, gap = oracle.fsr_frame_concealed(P, delta, smp, msk, psum, pcnt)
    rng = np.random.default_rng(4)
    for by, bx in [(0, 0), (0, 7), (3, 0), (5, 6), (9, 10)]:
        blk, g, _ = oracle.fsr_block_concealed(P, delta, out, smp, msk, psum, pcnt, by, bx)
        np.testing.assert_array_equal(blk, out[4 * by:4 * by + 4, 4 * bx:4 * bx + 4])
        assert g == gap[by, bx]
        later = out.copy()
        ys, xs = np.mgrid[0:out.shape[0], 0:out.shape[1]]
        tail = (ys // 4 > by) | ((ys // 4 == by) & (xs // 4 >= bx))
        later[tail] = rng.random(int(tail.sum()))
        blk2, _, _ = oracle.fsr_block_concealed(P, delta, later, smp, msk, psum, pcnt, by, bx)
        np.testing.assert_array_equal(blk, blk2)
    # a value in an earlier block that is neither measured nor projected does change the result
    y, x = next((y, x) for y in range(4, 8) for x in range(4, 8)
                if msk[y, x] == 0 and pcnt[y, x] == 0)
    moved = out.copy()
    moved[y, x] += 0.25
    a, _, _ = oracle.fsr_block_concealed(P, delta, out, smp, msk, psum, pcnt, 2, 2)
    b, _, _ = oracle.fsr_block_concealed(P, delta, moved, smp, msk, psum, pcnt, 2, 2)
    assert np.abs(a - b).max() > 1e-6
