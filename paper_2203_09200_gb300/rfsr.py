"""ctypes binding of the C ABI in include/rfsr.h (argument marshalling only).

Every step of the frame path runs in the CUDA library ``librfsr.so``; there is no Python or CPU
fallback: if the library is missing, ``load()`` raises.  Device buffers may be given as torch
CUDA tensors (their ``data_ptr()`` is passed) or as integer device addresses.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librfsr.so")

RFSR_OK, RFSR_EINVAL, RFSR_EMASK, RFSR_ENOMEM, RFSR_EAGAIN, RFSR_EBUSY, RFSR_ETIMEDOUT, \
    RFSR_EDEVICE, RFSR_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7, -8
CC_MODES = {"none": 0, "rme": 1, "rmc": 2, "frmc": 3, "nnc": 4, "nnc_frmc": 5}
DEC_MEASURED, DEC_NOT_PROJECTABLE, DEC_NNC_REJECT, DEC_CHECK_REJECT, DEC_ACCEPT = range(5)
MASK_FIXED, MASK_DYNAMIC = 0, 1
DBG_MV, DBG_FMV, DBG_DECISION, DBG_PSUM, DBG_PCNT, DBG_FSR, DBG_REC, DBG_RMV, DBG_FSR_SEL = range(9)
FSR_SEL_NONE = 0xFFFF

_ERRNAMES = {RFSR_EINVAL: "EINVAL", RFSR_EMASK: "EMASK", RFSR_ENOMEM: "ENOMEM",
             RFSR_EAGAIN: "EAGAIN", RFSR_EBUSY: "EBUSY", RFSR_ETIMEDOUT: "ETIMEDOUT",
             RFSR_EDEVICE: "EDEVICE", RFSR_ESTATE: "ESTATE"}


class RfsrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class rfsr_engine_config(C.Structure):
    _fields_ = [("device", C.c_int), ("memory_budget", C.c_size_t), ("cuda_stream", C.c_void_p),
                ("max_inflight", C.c_int), ("batched", C.c_int), ("profile", C.c_int),
                ("serve", C.c_int), ("autotune", C.c_int), ("dev_alloc", ALLOC_FN),
                ("dev_free", FREE_FN), ("alloc_ctx", C.c_void_p), ("fuse_me_cc", C.c_int),
                ("wait_test", C.c_int)]


class rfsr_stream_config(C.Structure):
    _fields_ = [("height", C.c_int), ("width", C.c_int), ("mask_type", C.c_int),
                ("cc_mode", C.c_int), ("num_refs", C.c_int), ("template_size", C.c_int),
                ("search_radius", C.c_int), ("check_radius", C.c_int),
                ("fsr_iterations", C.c_int), ("fsr_rho", C.c_float), ("fsr_gamma", C.c_float),
                ("fsr_proj_weight", C.c_float), ("fsr_overwrite_projected", C.c_int),
                ("keep_f32", C.c_int), ("fsr_concealed_weight", C.c_float),
                ("fsr_trace", C.c_int), ("me_predict_radius", C.c_int)]


class rfsr_batch_shape(C.Structure):
    _fields_ = [("me_tile_rows", C.c_int), ("fsr_blocks", C.c_int), ("me_variant", C.c_int)]


class rfsr_tuning(C.Structure):
    _fields_ = [("tuned", C.c_int), ("steps", C.c_int), ("shape", rfsr_batch_shape),
                ("me_ns", C.c_float * 3), ("fsr_ns", C.c_float * 3)]


class rfsr_state_header(C.Structure):
    _fields_ = [("magic", C.c_uint32), ("version", C.c_uint32), ("bytes", C.c_uint64),
                ("config", rfsr_stream_config), ("hist", C.c_int32), ("reserved", C.c_int32),
                ("frames", C.c_int64)]


class rfsr_engine_info(C.Structure):
    _fields_ = [("device", C.c_int), ("memory_budget", C.c_size_t), ("memory_used", C.c_size_t),
                ("streams_live", C.c_int), ("streams_queued", C.c_int)]


class rfsr_stream_info(C.Structure):
    _fields_ = [("height", C.c_int), ("width", C.c_int), ("live", C.c_int),
                ("frames_pushed", C.c_longlong), ("frames_collected", C.c_longlong),
                ("history_frames", C.c_int), ("device_bytes", C.c_size_t)]


# exported symbols with their argument types (also used by the export test)
_VP, _I = C.c_void_p, C.c_int
SYMBOLS = {
    "rfsr_engine_config_default": ([C.POINTER(rfsr_engine_config)], None),
    "rfsr_stream_config_default": ([C.POINTER(rfsr_stream_config)], None),
    "rfsr_engine_create": ([C.POINTER(rfsr_engine_config), C.POINTER(_VP)], _I),
    "rfsr_engine_destroy": ([_VP], _I),
    "rfsr_engine_step": ([_VP], _I),
    "rfsr_engine_sync": ([_VP, _I], _I),
    "rfsr_engine_last_step_ms": ([_VP, C.POINTER(C.c_float), C.POINTER(C.c_int)], _I),
    "rfsr_engine_set_shape": ([_VP, C.POINTER(rfsr_batch_shape)], _I),
    "rfsr_engine_get_info": ([_VP, C.POINTER(rfsr_engine_info)], _I),
    "rfsr_stream_export": ([_VP, _VP, C.c_size_t, C.POINTER(C.c_size_t)], _I),
    "rfsr_stream_import": ([_VP, _VP, C.c_size_t, C.POINTER(_VP)], _I),
    "rfsr_engine_get_tuning": ([_VP, C.POINTER(rfsr_tuning)], _I),
    "rfsr_create_stream": ([_VP, C.POINTER(rfsr_stream_config), C.POINTER(_VP)], _I),
    "rfsr_push_frame": ([_VP, _VP, _VP], _I),
    "rfsr_push_frame_device": ([_VP, _VP, _VP, _VP], _I),
    "rfsr_get_frame": ([_VP, _VP, _VP, _I], _I),
    "rfsr_get_frame_device": ([_VP, _VP, _VP, _I], _I),
    "rfsr_destroy": ([_VP], _I),
    "rfsr_stream_state": ([_VP], _I),
    "rfsr_stream_get_info": ([_VP, C.POINTER(rfsr_stream_info)], _I),
    "rfsr_set_history": ([_VP, _I, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP)], _I),
    "rfsr_debug_get": ([_VP, _I, _I, _VP], _I),
    "rfsr_fsr_device": ([C.POINTER(rfsr_stream_config), _VP, _VP, _VP, _VP, _VP, _VP, _VP], _I),
    "rfsr_fsr_device_trace": ([C.POINTER(rfsr_stream_config), _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                               _VP], _I),
    "rfsr_stream_phase_ms": ([_VP, C.POINTER(C.c_float)], _I),
    "rfsr_me_cc_project_noalloc": ([C.POINTER(rfsr_stream_config), _VP, _VP, _I, C.POINTER(_VP),
                                    C.POINTER(_VP), C.POINTER(_VP), _VP, _VP, _VP, _VP, _VP], _I),
    "rfsr_alu_peak": ([_I, _I, _I, C.POINTER(C.c_double), C.POINTER(C.c_double)], _I),
    "rfsr_kernel_launches": ([], C.c_longlong),
    "rfsr_fused_schedule": ([_I, _I, _I, _I, _VP, _I], _I),
    "rfsr_last_error": ([], C.c_char_p),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load ``librfsr.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run __graft_entry__.build())")
        lib = C.CDLL(path)
        for name, (args, res) in SYMBOLS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _producer(stream, like):
    if stream is None:
        if getattr(like, "is_cuda", False):
            import torch
            return torch.cuda.current_stream(like.device).cuda_stream
        return None
    return getattr(stream, "cuda_stream", stream)


def _torch_allocator(device: int):
    import torch

    def alloc(n, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(n), device)
        except Exception:          # reported by the library as ENOMEM
            return None

    def free(p, ctx):
        torch.cuda.caching_allocator_delete(p)

    return ALLOC_FN(alloc), FREE_FN(free)


def _check(rc: int):
    if rc < 0:
        raise RfsrError(rc, load().rfsr_last_error().decode())
    return rc


def _ptr(x) -> Optional[int]:
    """Device / host address of a torch tensor, numpy array, or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_config(height: int, width: int, cc_mode="nnc_frmc", mask_type: int = MASK_DYNAMIC,
                  num_refs: int = 3, template_size: int = 9, search_radius: int = 8,
                  check_radius: Optional[int] = None, fsr_iterations: int = 100,
                  fsr_rho: float = 0.7, fsr_gamma: float = 0.5, fsr_proj_weight: float = 1.0,
                  fsr_overwrite_projected: bool = False, keep_f32: bool = False,
                  fsr_concealed_weight: float = 0.0, fsr_trace: bool = False,
                  me_predict_radius: int = 0) -> rfsr_stream_config:
    c = rfsr_stream_config()
    load().rfsr_stream_config_default(C.byref(c))
    c.height, c.width = height, width
    c.cc_mode = CC_MODES[cc_mode] if isinstance(cc_mode, str) else int(cc_mode)
    c.mask_type = mask_type
    c.num_refs = num_refs
    c.template_size = template_size
    c.search_radius = search_radius
    c.check_radius = search_radius if check_radius is None else check_radius
    c.fsr_iterations = fsr_iterations
    c.fsr_rho, c.fsr_gamma, c.fsr_proj_weight = fsr_rho, fsr_gamma, fsr_proj_weight
    c.fsr_overwrite_projected = int(bool(fsr_overwrite_projected))
    c.keep_f32 = int(bool(keep_f32))
    c.fsr_concealed_weight = fsr_concealed_weight
    c.fsr_trace = int(bool(fsr_trace))
    c.me_predict_radius = me_predict_radius
    return c


class Engine:
    """rfsr_engine_create / rfsr_engine_destroy."""

    def __init__(self, device: int = 0, memory_budget: int = 0, cuda_stream: Optional[int] = None,
                 max_inflight: int = 4, batched: bool = False, profile: bool = False,
                 serve: bool = False, autotune: bool = True, allocator: Optional[str] = None,
                 fuse_me_cc: bool = False, wait_test: bool = False):
        """allocator="torch": the engine's device memory comes from PyTorch's caching allocator
        (through the dev_alloc / dev_free callbacks of the engine config)."""
        lib = load()
        cfg = rfsr_engine_config()
        lib.rfsr_engine_config_default(C.byref(cfg))
        cfg.device, cfg.memory_budget = device, memory_budget
        cfg.cuda_stream = cuda_stream
        cfg.max_inflight, cfg.batched, cfg.profile = max_inflight, int(batched), int(profile)
        cfg.serve, cfg.autotune = int(serve), int(autotune)
        cfg.fuse_me_cc, cfg.wait_test = int(fuse_me_cc), int(wait_test)
        self._callbacks = None
        if allocator == "torch":
            self._callbacks = _torch_allocator(device)
            cfg.dev_alloc, cfg.dev_free = self._callbacks
        elif allocator is not None:
            raise ValueError("allocator must be None or 'torch'")
        h = C.c_void_p()
        _check(lib.rfsr_engine_create(C.byref(cfg), C.byref(h)))
        self.handle = h
        self.streams = []

    def create_stream(self, allow_queued: bool = False, **kw) -> "Stream":
        """rfsr_create_stream.  With allow_queued, a stream queued by memory admission (EAGAIN)
        is returned instead of raising; Stream.live tells when it is admitted."""
        cfg = stream_config(**kw)
        h = C.c_void_p()
        rc = load().rfsr_create_stream(self.handle, C.byref(cfg), C.byref(h))
        if not (allow_queued and rc == RFSR_EAGAIN):
            _check(rc)
        s = Stream(self, h, cfg)
        self.streams.append(s)
        return s

    def import_stream(self, state: bytes) -> "Stream":
        """rfsr_stream_import: a stream on this engine from rfsr_stream_export's bytes."""
        buf = C.create_string_buffer(bytes(state), len(state))
        h = C.c_void_p()
        _check(load().rfsr_stream_import(self.handle, buf, len(state), C.byref(h)))
        cfg = rfsr_state_header.from_buffer_copy(bytes(state)[:C.sizeof(rfsr_state_header)]).config
        st = Stream(self, h, cfg)
        self.streams.append(st)
        return st

    def info(self) -> dict:
        """rfsr_engine_get_info."""
        i = rfsr_engine_info()
        _check(load().rfsr_engine_get_info(self.handle, C.byref(i)))
        return {"device": i.device, "memory_budget": i.memory_budget, "memory_used": i.memory_used,
                "streams_live": i.streams_live, "streams_queued": i.streams_queued}

    def last_step_ms(self):
        """(device ms, frames) of the most recent batched step (profile engines)."""
        ms, n = C.c_float(), C.c_int()
        _check(load().rfsr_engine_last_step_ms(self.handle, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def step(self) -> int:
        return _check(load().rfsr_engine_step(self.handle))

    def set_shape(self, me_tile_rows: int = 64, fsr_blocks: int = 4, me_variant: int = 0):
        """rfsr_engine_set_shape: fix the batched tile shape (ends autotuning)."""
        sh = rfsr_batch_shape(me_tile_rows, fsr_blocks, me_variant)
        _check(load().rfsr_engine_set_shape(self.handle, C.byref(sh)))

    def tuning(self) -> dict:
        """rfsr_engine_get_tuning as a dict."""
        t = rfsr_tuning()
        _check(load().rfsr_engine_get_tuning(self.handle, C.byref(t)))
        return {"tuned": bool(t.tuned), "steps": t.steps,
                "shape": {"me_tile_rows": t.shape.me_tile_rows, "fsr_blocks": t.shape.fsr_blocks,
                          "me_variant": t.shape.me_variant},
                "me_ns_per_pixel_ref": {"strips64": round(t.me_ns[0], 5),
                                        "strips32": round(t.me_ns[1], 5),
                                        "box": round(t.me_ns[2], 5)},
                "fsr_ns_per_block": {"4": round(t.fsr_ns[0], 3), "2": round(t.fsr_ns[1], 3),
                                     "8": round(t.fsr_ns[2], 3)}}

    def sync(self, timeout_ms: int = -1):
        _check(load().rfsr_engine_sync(self.handle, timeout_ms))

    def destroy(self):
        if self.handle:
            for s in self.streams:
                s.handle = None
            _check(load().rfsr_engine_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.destroy()


class Stream:
    """rfsr_create_stream / rfsr_push_frame / rfsr_get_frame / rfsr_destroy and the debug calls."""

    def __init__(self, engine: Engine, handle, cfg: rfsr_stream_config):
        self.engine, self.handle, self.cfg = engine, handle, cfg
        self.H, self.W = cfg.height, cfg.width

    def push_frame(self, samples: np.ndarray, mask: np.ndarray):
        s = np.ascontiguousarray(samples, np.uint8)
        m = np.ascontiguousarray(mask, np.uint8)
        assert s.shape == (self.H, self.W) and m.shape == (self.H, self.W)
        _check(load().rfsr_push_frame(self.handle, s.ctypes.data, m.ctypes.data))

    def push_frame_device(self, d_samples, d_mask, stream=None):
        """stream: the CUDA stream that wrote the buffers (a torch.cuda.Stream, a cudaStream_t
        handle or None; None with torch tensors = the tensors' current torch stream)."""
        _check(load().rfsr_push_frame_device(self.handle, _ptr(d_samples), _ptr(d_mask),
                                             _producer(stream, d_samples)))

    def get_frame(self, timeout_ms: int = -1, f32: bool = False):
        out = np.empty((self.H, self.W), np.uint8)
        o32 = np.empty((self.H, self.W), np.float32) if f32 else None
        _check(load().rfsr_get_frame(self.handle, out.ctypes.data,
                                     None if o32 is None else o32.ctypes.data, timeout_ms))
        return (out, o32) if f32 else out

    def get_frame_device(self, d_out_u8=None, d_out_f32=None, timeout_ms: int = -1):
        _check(load().rfsr_get_frame_device(self.handle, _ptr(d_out_u8), _ptr(d_out_f32),
                                            timeout_ms))

    def export_state(self) -> bytes:
        """rfsr_stream_export: the stream's configuration and last K frames (checkpoint)."""
        n = C.c_size_t()
        _check(load().rfsr_stream_export(self.handle, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(load().rfsr_stream_export(self.handle, buf, n.value, C.byref(n)))
        return buf.raw[:n.value]

    def set_history(self, history: Sequence[Tuple[np.ndarray, np.ndarray, np.ndarray]]):
        """history[k-1] = (reconstruction, samples, 0/1 mask) of frame t-k."""
        n = len(history)
        keep = [tuple(np.ascontiguousarray(a, np.uint8) for a in h) for h in history]
        arr = C.c_void_p * max(1, n)
        rec = arr(*[h[0].ctypes.data for h in keep])
        smp = arr(*[h[1].ctypes.data for h in keep])
        msk = arr(*[h[2].ctypes.data for h in keep])
        _check(load().rfsr_set_history(self.handle, n, rec, smp, msk))

    def debug_get(self, what: int, k: int = 0) -> np.ndarray:
        H, W = self.H, self.W
        nb = (-(-H // 4)) * (-(-W // 4))
        shape, dt = {DBG_MV: ((H, W, 2), np.int8), DBG_FMV: ((H, W, 2), np.int8),
                     DBG_RMV: ((H, W, 2), np.int8), DBG_DECISION: ((H, W), np.uint8),
                     DBG_PSUM: ((H, W), np.uint16), DBG_PCNT: ((H, W), np.uint8),
                     DBG_FSR: ((H, W), np.float32), DBG_REC: ((H, W), np.uint8),
                     DBG_FSR_SEL: ((nb, max(1, self.cfg.fsr_iterations)), np.uint16)}[what]
        out = np.empty(shape, dt)
        _check(load().rfsr_debug_get(self.handle, what, k, out.ctypes.data))
        return out

    def phase_ms(self):
        """(ingest, ME, checks + projection, FSR) device ms of the last pushed frame."""
        a = (C.c_float * 4)()
        _check(load().rfsr_stream_phase_ms(self.handle, a))
        return tuple(float(x) for x in a)

    @property
    def live(self) -> bool:
        return _check(load().rfsr_stream_state(self.handle)) == 1

    def info(self) -> rfsr_stream_info:
        i = rfsr_stream_info()
        _check(load().rfsr_stream_get_info(self.handle, C.byref(i)))
        return i

    def destroy(self):
        if self.handle:
            _check(load().rfsr_destroy(self.handle))
            self.handle = None
            if self in self.engine.streams:
                self.engine.streams.remove(self)


def fsr_device(d_smp, d_msk, d_psum, d_pcnt, d_out_f32, d_out_u8, height: int, width: int,
               cuda_stream: Optional[int] = None, **fsr_kw):
    """rfsr_fsr_device: stand-alone FSR over device buffers."""
    cfg = stream_config(height, width, **fsr_kw)
    _check(load().rfsr_fsr_device(C.byref(cfg), _ptr(d_smp), _ptr(d_msk), _ptr(d_psum),
                                  _ptr(d_pcnt), _ptr(d_out_f32), _ptr(d_out_u8), cuda_stream))


def fused_schedule(height: int, width: int, num_refs: int, grid: int) -> np.ndarray:
    """rfsr_fused_schedule: the claim order of the fused ME + checks launch (uint32 items)."""
    n = _check(load().rfsr_fused_schedule(height, width, num_refs, grid, None, 0))
    out = np.zeros(max(1, n), np.uint32)
    _check(load().rfsr_fused_schedule(height, width, num_refs, grid, out.ctypes.data, n))
    return out[:n]


def fsr_device_trace(d_smp, d_msk, d_psum, d_pcnt, d_out_f32, d_out_u8, d_sel, height: int,
                     width: int, cuda_stream: Optional[int] = None, **fsr_kw):
    """rfsr_fsr_device_trace: stand-alone FSR that also records the selected basis pair of every
    iteration of every block in d_sel (nblocks x iterations uint16)."""
    cfg = stream_config(height, width, **fsr_kw)
    _check(load().rfsr_fsr_device_trace(C.byref(cfg), _ptr(d_smp), _ptr(d_msk), _ptr(d_psum),
                                        _ptr(d_pcnt), _ptr(d_out_f32), _ptr(d_out_u8),
                                        _ptr(d_sel), cuda_stream))


def me_cc_project_noalloc(d_smp, d_msk, refs, d_psum, d_pcnt, height: int, width: int,
                          d_dec=None, d_status=None, cuda_stream: Optional[int] = None, **cfg_kw):
    """rfsr_me_cc_project_noalloc: ME + checks + projection of one frame for callers that cannot
    allocate device memory; every intermediate lives in the library's fixed static scratch.
    refs[k] = (reconstruction, samples, 0/1 mask) of frame t-1-k as device buffers."""
    cfg = stream_config(height, width, **cfg_kw)
    n = len(refs)
    arr = C.c_void_p * max(1, n)
    rec = arr(*[_ptr(r[0]) for r in refs])
    smp = arr(*[_ptr(r[1]) for r in refs])
    msk = arr(*[_ptr(r[2]) for r in refs])
    _check(load().rfsr_me_cc_project_noalloc(C.byref(cfg), _ptr(d_smp), _ptr(d_msk), n, rec, smp,
                                             msk, _ptr(d_psum), _ptr(d_pcnt), _ptr(d_dec),
                                             _ptr(d_status), cuda_stream))


ALU_KINDS = ["iadd3", "lop3", "prmt", "vabsdiffu4", "vsadu4+add", "vimax3_u16x2",
             "vimin3_u16x2", "imad", "sad", "imin", "xor", "ffma", "iadd3+imad",
             "vabsdiff4.add", "min.s16x2", "vabsdiff2.add", "vimax3_s16x2", "vimax3_u32"]


def alu_peak(kind: str, device: int = 0, iters: int = 2000):
    """rfsr_alu_peak: (instructions per second, per clock per SM) of one instruction kind."""
    a, b = C.c_double(), C.c_double()
    _check(load().rfsr_alu_peak(device, ALU_KINDS.index(kind), iters, C.byref(a), C.byref(b)))
    return a.value, b.value


def kernel_launches() -> int:
    return int(load().rfsr_kernel_launches())


# C-ABI names, for callers who prefer the flat interface
rfsr_fsr_device = fsr_device
rfsr_kernel_launches = kernel_launches


class Router:
    """Streams over several engines (replicas, for example one per GPU; streams are independent,
    so nothing is exchanged between them).  A new stream goes to the engine with the most free
    memory budget; migrate() moves a stream between engines through its exported state, so its
    next frame gives exactly the result it would have given where it was."""

    def __init__(self, engines: Sequence[Engine]):
        self.engines = list(engines)

    def place(self) -> Engine:
        free = [(e.info()["memory_budget"] - e.info()["memory_used"], -i)
                for i, e in enumerate(self.engines)]
        return self.engines[-max(free)[1]]

    def create_stream(self, **kw) -> Stream:
        return self.place().create_stream(**kw)

    def migrate(self, stream: Stream, to: Engine) -> Stream:
        """Export, create on ``to``, then destroy the original (between frames)."""
        state = stream.export_state()
        moved = to.import_stream(state)
        stream.destroy()
        return moved
