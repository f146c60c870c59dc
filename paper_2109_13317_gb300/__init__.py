"""GB300-native pseudofermion FRG flow solver (arXiv:2109.13317 hot path).

The compute path is the CUDA library ``libsr.so`` (C ABI in ``include/sr.h``); this package
is a thin ctypes binding with the same entry-point names.  There is no CPU fallback: if
the library is missing or fails to load, every call raises.
"""
from .binding import (  # noqa: F401
    SR_EULER, SR_FP32_MIXED, SR_FP64, SR_RK_ADAPTIVE, SR_RK_FIXED, SR_SU2, SR_TRI, SR_XYZ,
    SR_OK, SR_EINVAL, SR_ENOMEM, SR_ECUDA, SR_ESYMMETRY, SR_ENONFINITE, SR_ETIMEOUT, SR_EUNSUPPORTED,
    Batch, Flow, Lattice, SrError, library_path, load_library, sr_couplings_linear, sr_frequency_mesh_exponential,
    sr_peak_fma,
)
