"""GB300 (sm_103a) implementation of the per-frame hot path of recursive frequency-selective
reconstruction of quarter-sampled video (Grosche, Seiler, Kaup, ICIP 2021, arXiv 2203.09200):
motion estimation, consistency checks (RME, RMC, FRMC, NNC), projection and D-FSR, behind the C
ABI of ``include/rfsr.h``.  ``rfsr`` is the ctypes binding; ``build`` compiles the library.
"""
from . import rfsr  # noqa: F401
from .rfsr import Engine, Stream, RfsrError, load, stream_config, fsr_device  # noqa: F401
