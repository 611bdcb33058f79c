"""Seeded synthetic quarter-sampled video, shared by the tests, the oracle checks and the bench.

This module only generates inputs: content, motion, the sensor's sampling masks and the sampled
frames f_sub = f * b (Sec. 2.1). None of the reconstruction method (motion estimation, checks,
projection, FSR) lives here, so both the oracle and the CUDA path can take their inputs from it
without sharing any of the method's arithmetic.

Mask conventions (Sec. 1, quarter sampling; Sec. 2.1 for f_sub = f * b):
  * per 2x2 block exactly one pixel is measured; its position index j in {0,1,2,3} maps to the
    in-block offset (dy, dx) = (j >> 1, j & 1);
  * fixed mask: one j per block, drawn uniformly, the same for every frame;
  * dynamic mask: one permutation of (0,1,2,3) per block, frame t measures perm[t mod 4], so every
    pixel of a block is read exactly once in four frames and the mask repeats every fourth frame.

Content recipes (all 8-bit luma, rounded half to even and clipped to [0, 255]):
  * ``sinusoid_translation``: sum of 6 random 2-D sinusoids (periods 4..32 px) plus Gaussian noise
    (sigma 2) frozen on the canvas, the whole frame translated by an integer (rows, cols) per frame;
  * ``moving_scene``: a band-limited or 1/f^2 noise background (optionally panned by an integer
    velocity) with textured rectangles / discs moving by integer velocities, drawn in a fixed
    z-order (occlusion), with optional seeded velocity changes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence as Seq, Tuple

import numpy as np

__all__ = [
    "MASK_FIXED", "MASK_DYNAMIC",
    "positions_to_mask", "fixed_positions", "dynamic_permutations", "dynamic_positions",
    "VideoSequence", "sinusoid_translation", "moving_scene",
    "config1", "config2", "config3", "config4_streams", "config5_arrivals",
    "StreamSpec", "Arrival", "random_frame_inputs",
]

MASK_FIXED = 0
MASK_DYNAMIC = 1


# ----------------------------------------------------------------------------------------------
# sampling masks
# ----------------------------------------------------------------------------------------------
def positions_to_mask(pos: np.ndarray) -> np.ndarray:
    """Expand per-block position indices (H/2, W/2) in {0..3} to a 0/1 u8 mask (H, W)."""
    pos = np.asarray(pos)
    hb, wb = pos.shape
    mask = np.zeros((2 * hb, 2 * wb), dtype=np.uint8)
    for j in range(4):
        dy, dx = j >> 1, j & 1
        mask[dy::2, dx::2] = (pos == j)
    return mask


def fixed_positions(H: int, W: int, rng: np.random.Generator) -> np.ndarray:
    """One uniformly drawn position index per 2x2 block."""
    return rng.integers(0, 4, size=(H // 2, W // 2), dtype=np.int64).astype(np.uint8)


def dynamic_permutations(H: int, W: int, rng: np.random.Generator) -> np.ndarray:
    """One random permutation of (0,1,2,3) per 2x2 block, shape (H/2, W/2, 4)."""
    keys = rng.random(size=(H // 2, W // 2, 4))
    return np.argsort(keys, axis=-1).astype(np.uint8)


def dynamic_positions(perm: np.ndarray, t: int) -> np.ndarray:
    """Position indices measured in frame t for a dynamic mask."""
    return perm[..., t % 4]


# ----------------------------------------------------------------------------------------------
# sequences
# ----------------------------------------------------------------------------------------------
@dataclasses.dataclass
class VideoSequence:
    frames: np.ndarray          # (F, H, W) u8 ground truth
    masks: np.ndarray           # (F, H, W) u8 in {0,1}
    mask_type: int              # MASK_FIXED or MASK_DYNAMIC
    name: str = ""

    @property
    def samples(self) -> np.ndarray:
        """f_sub = f * b, unmeasured bytes zero."""
        return (self.frames * self.masks).astype(np.uint8)

    @property
    def shape(self) -> Tuple[int, int]:
        return self.frames.shape[1], self.frames.shape[2]

    def __len__(self) -> int:
        return self.frames.shape[0]


def _quantize(img: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def _make_masks(F: int, H: int, W: int, mask_type: int, rng: np.random.Generator) -> np.ndarray:
    masks = np.empty((F, H, W), dtype=np.uint8)
    if mask_type == MASK_FIXED:
        m = positions_to_mask(fixed_positions(H, W, rng))
        masks[:] = m
    else:
        perm = dynamic_permutations(H, W, rng)
        for t in range(F):
            masks[t] = positions_to_mask(dynamic_positions(perm, t))
    return masks


def sinusoid_translation(H: int = 64, W: int = 64, F: int = 8, seed: int = 1,
                         velocity: Tuple[int, int] = (2, 1), mask_type: int = MASK_FIXED,
                         n_sinusoids: int = 6, noise_sigma: float = 2.0) -> VideoSequence:
    """Sum of random sinusoids + frozen noise, translated by ``velocity`` = (rows, cols) per frame.

    Content at frame-t pixel (y, x) equals the canvas at (y - vy*t, x - vx*t), so the true motion
    vector from frame t into frame t-k is (-vy*k, -vx*k).
    """
    rng = np.random.default_rng(seed)
    vy, vx = velocity
    pad_y, pad_x = abs(vy) * F + 1, abs(vx) * F + 1
    Hc, Wc = H + 2 * pad_y, W + 2 * pad_x
    y, x = np.mgrid[0:Hc, 0:Wc].astype(np.float64)
    canvas = np.full((Hc, Wc), 128.0)
    for _ in range(n_sinusoids):
        P = rng.uniform(4.0, 32.0)
        th = rng.uniform(0.0, math.pi)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        a = rng.uniform(8.0, 16.0)
        canvas += a * np.cos(2.0 * math.pi * (x * math.cos(th) + y * math.sin(th)) / P + ph)
    canvas += rng.normal(0.0, noise_sigma, size=canvas.shape)
    canvas = _quantize(canvas)
    frames = np.empty((F, H, W), dtype=np.uint8)
    for t in range(F):
        oy, ox = pad_y - vy * t, pad_x - vx * t
        frames[t] = canvas[oy:oy + H, ox:ox + W]
    masks = _make_masks(F, H, W, mask_type, rng)
    return VideoSequence(frames, masks, mask_type, name="sinusoid_translation")


def _bandlimited_noise(Hc: int, Wc: int, rng: np.random.Generator, cutoff: float = 0.15,
                       rolloff: float = 0.05) -> np.ndarray:
    """Periodic Gaussian noise low-passed at ``cutoff`` cycles/px with a raised-cosine roll-off,
    normalised to zero mean and unit standard deviation."""
    white = rng.normal(size=(Hc, Wc))
    fy = np.fft.fftfreq(Hc)[:, None]
    fx = np.fft.rfftfreq(Wc)[None, :]
    r = np.sqrt(fy * fy + fx * fx)
    lo, hi = cutoff - rolloff, cutoff + rolloff
    gain = np.where(r <= lo, 1.0, np.where(r >= hi, 0.0,
                                           0.5 * (1.0 + np.cos(math.pi * (r - lo) / (hi - lo)))))
    out = np.fft.irfft2(np.fft.rfft2(white) * gain, s=(Hc, Wc))
    out -= out.mean()
    sd = out.std()
    return out / (sd if sd > 0 else 1.0)


def _spectral_noise(Hc: int, Wc: int, rng: np.random.Generator) -> np.ndarray:
    """Periodic noise with a 1/f^2 power spectrum (amplitude ~ 1/|f|), DC removed, unit std."""
    fy = np.fft.fftfreq(Hc)[:, None]
    fx = np.fft.rfftfreq(Wc)[None, :]
    r = np.sqrt(fy * fy + fx * fx)
    amp = np.zeros_like(r)
    amp[r > 0] = 1.0 / r[r > 0]
    phase = rng.uniform(0.0, 2.0 * math.pi, size=r.shape)
    spec = amp * np.exp(1j * phase)
    out = np.fft.irfft2(spec, s=(Hc, Wc))
    out -= out.mean()
    sd = out.std()
    return out / (sd if sd > 0 else 1.0)


@dataclasses.dataclass
class _Obj:
    shape: str                  # "rect" or "disc"
    h: int
    w: int
    tex: np.ndarray             # (h, w) float texture
    y0: int
    x0: int
    # velocity schedule: list of (first frame, vy, vx); position(t) = start + sum of velocities
    schedule: List[Tuple[int, int, int]]

    def position(self, t: int) -> Tuple[int, int]:
        y, x = self.y0, self.x0
        for i, (f0, vy, vx) in enumerate(self.schedule):
            f1 = self.schedule[i + 1][0] if i + 1 < len(self.schedule) else None
            end = t if f1 is None else min(t, f1)
            n = max(0, end - f0)
            y += vy * n
            x += vx * n
        return y, x


def moving_scene(H: int, W: int, F: int, seed: int, mask_type: int = MASK_DYNAMIC,
                 background: str = "band", pan_max: int = 4, n_objects: int = 4,
                 size_range: Tuple[int, int] = (64, 256), vel_max: int = 6,
                 shapes: Seq[str] = ("rect",), redraw: Optional[Tuple[int, int]] = None,
                 mean: float = 128.0, std: float = 40.0) -> VideoSequence:
    """Noise background (``band``: band-limited, ``spectral``: 1/f^2), globally panned by a random
    integer velocity with |v|_inf <= ``pan_max``, plus ``n_objects`` textured objects with their own
    integer velocities |v|_inf <= ``vel_max`` drawn in a fixed z-order.  With ``redraw=(a, b)``
    each object's velocity is redrawn after U{a..b} frames (sudden direction changes)."""
    rng = np.random.default_rng(seed)
    gen = _bandlimited_noise if background == "band" else _spectral_noise
    pad = max(8, pan_max * F)
    Hc = H + 2 * pad if background == "spectral" else H
    Wc = W + 2 * pad if background == "spectral" else W
    bg = mean + std * gen(Hc, Wc, rng)
    pvy = int(rng.integers(-pan_max, pan_max + 1)) if pan_max > 0 else 0
    pvx = int(rng.integers(-pan_max, pan_max + 1)) if pan_max > 0 else 0

    lo, hi = size_range
    lo = min(lo, max(4, min(H, W) // 2))
    hi = max(lo, min(hi, max(lo, min(H, W))))
    objs: List[_Obj] = []
    for _ in range(n_objects):
        shape = shapes[int(rng.integers(0, len(shapes)))]
        h = int(rng.integers(lo, hi + 1))
        w = h if shape == "disc" else int(rng.integers(lo, hi + 1))
        tex = rng.uniform(60.0, 200.0) + rng.uniform(20.0, 50.0) * gen(h, w, rng)
        y0 = int(rng.integers(-h // 2, H - h // 2))
        x0 = int(rng.integers(-w // 2, W - w // 2))
        sched = [(0, int(rng.integers(-vel_max, vel_max + 1)), int(rng.integers(-vel_max, vel_max + 1)))]
        if redraw is not None:
            f = 0
            while True:
                f += int(rng.integers(redraw[0], redraw[1] + 1))
                if f >= F:
                    break
                sched.append((f, int(rng.integers(-vel_max, vel_max + 1)),
                              int(rng.integers(-vel_max, vel_max + 1))))
        objs.append(_Obj(shape, h, w, tex, y0, x0, sched))

    frames = np.empty((F, H, W), dtype=np.uint8)
    yy = np.arange(H)
    xx = np.arange(W)
    for t in range(F):
        if background == "spectral":
            oy, ox = pad - pvy * t, pad - pvx * t
            img = bg[oy:oy + H, ox:ox + W].copy()
        else:   # periodic canvas of frame size: wrap
            img = bg[np.ix_((yy - pvy * t) % H, (xx - pvx * t) % W)]
        for o in objs:
            py, px = o.position(t)
            y0, y1 = max(0, py), min(H, py + o.h)
            x0, x1 = max(0, px), min(W, px + o.w)
            if y0 >= y1 or x0 >= x1:
                continue
            patch = o.tex[y0 - py:y1 - py, x0 - px:x1 - px]
            if o.shape == "disc":
                cy, cx = (o.h - 1) / 2.0, (o.w - 1) / 2.0
                gy, gx = np.mgrid[y0 - py:y1 - py, x0 - px:x1 - px]
                inside = (gy - cy) ** 2 + (gx - cx) ** 2 <= (o.h / 2.0) ** 2
                img[y0:y1, x0:x1] = np.where(inside, patch, img[y0:y1, x0:x1])
            else:
                img[y0:y1, x0:x1] = patch
        frames[t] = _quantize(img)
    masks = _make_masks(F, H, W, mask_type, rng)
    return VideoSequence(frames, masks, mask_type, name=f"moving_scene_{background}")


# ----------------------------------------------------------------------------------------------
# the five workload recipes
# ----------------------------------------------------------------------------------------------
def config1(seed: int = 1, H: int = 64, W: int = 64, F: int = 8) -> VideoSequence:
    """64x64, 8 frames, fixed mask, 6 sinusoids + noise sigma 2, translation (1 col, 2 rows)/frame."""
    return sinusoid_translation(H, W, F, seed=seed, velocity=(2, 1), mask_type=MASK_FIXED)


def config2(seed: int = 2, H: int = 720, W: int = 1280, F: int = 32,
            mask_type: int = MASK_DYNAMIC) -> VideoSequence:
    """1280x720, 32 frames, dynamic mask, band-limited noise panned by |v|<=4 plus 4 rectangles
    (64..256 px) with independent velocities |v|<=6 and occlusion."""
    return moving_scene(H, W, F, seed, mask_type=mask_type, background="band", pan_max=4,
                        n_objects=4, size_range=(64, 256), vel_max=6, shapes=("rect",))


def config3(seed: int = 3, H: int = 1080, W: int = 1920, F: int = 64,
            mask_type: int = MASK_DYNAMIC) -> VideoSequence:
    """1920x1080, 64 frames, dynamic mask, static 1/f^2 background plus 16 rectangles / discs
    (48..320 px) with integer velocities |v|<=8 redrawn every U{8..24} frames."""
    return moving_scene(H, W, F, seed, mask_type=mask_type, background="spectral", pan_max=0,
                        n_objects=16, size_range=(48, 320), vel_max=8, shapes=("rect", "disc"),
                        redraw=(8, 24))


@dataclasses.dataclass
class StreamSpec:
    H: int
    W: int
    mask_type: int
    frames: int
    seed: int

    def sequence(self, content: str = "config2") -> VideoSequence:
        if content == "config3":
            return config3(self.seed, self.H, self.W, self.frames, self.mask_type)
        return config2(self.seed, self.H, self.W, self.frames, self.mask_type)


def config4_streams(seed: int = 4, n_streams: int = 64, frames: int = 16) -> List[StreamSpec]:
    """64 streams, sizes drawn from {320x240, 640x480, 1280x720, 1920x1080}, the first half with a
    fixed and the second half with a dynamic mask, 16 frames each, content as ``config2``."""
    rng = np.random.default_rng(seed)
    sizes = [(240, 320), (480, 640), (720, 1280), (1080, 1920)]
    out = []
    for i in range(n_streams):
        H, W = sizes[int(rng.integers(0, len(sizes)))]
        mt = MASK_FIXED if i < n_streams // 2 else MASK_DYNAMIC
        out.append(StreamSpec(H, W, mt, frames, int(rng.integers(0, 2 ** 31 - 1))))
    return out


@dataclasses.dataclass
class Arrival:
    time_s: float
    spec: StreamSpec


def config5_arrivals(seed: int = 5, n_streams: int = 256, rate_hz: float = 20.0,
                     frames: Tuple[int, int] = (30, 300)) -> List[Arrival]:
    """256 streams arriving as a Poisson process (mean 20/s), sizes from 320x240 to 3840x2160,
    U{30..300} frames, fixed or dynamic mask 50/50, content as ``config3``."""
    rng = np.random.default_rng(seed)
    sizes = [(240, 320), (480, 640), (720, 1280), (1080, 1920), (1440, 2560), (2160, 3840)]
    t = 0.0
    out = []
    for _ in range(n_streams):
        t += float(rng.exponential(1.0 / rate_hz))
        H, W = sizes[int(rng.integers(0, len(sizes)))]
        mt = MASK_FIXED if rng.random() < 0.5 else MASK_DYNAMIC
        nf = int(rng.integers(frames[0], frames[1] + 1))
        out.append(Arrival(t, StreamSpec(H, W, mt, nf, int(rng.integers(0, 2 ** 31 - 1)))))
    return out


def random_frame_inputs(H: int, W: int, seed: int, mask_type: int = MASK_DYNAMIC):
    """Independent random frames for edge-case tests: (sample plane, mask, reference frame)."""
    rng = np.random.default_rng(seed)
    frame = rng.integers(0, 256, size=(H, W), dtype=np.int64).astype(np.uint8)
    ref = rng.integers(0, 256, size=(H, W), dtype=np.int64).astype(np.uint8)
    mask = positions_to_mask(fixed_positions(H, W, rng))
    return (frame * mask).astype(np.uint8), mask, ref
