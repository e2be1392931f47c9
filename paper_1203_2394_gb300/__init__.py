"""GB300 look-ahead decentralized particle filter (arXiv:1203.2394).

The filter runs in the CUDA library ``_lib/libdpf.so`` behind the C ABI of
``include/dpf.h``; ``dpf`` is its Python binding and ``workloads`` draws the
synthetic models and observations.
"""
from . import workloads  # noqa: F401
from .dpf import (DPF_F32, DPF_F64, DPF_SYS_GLOBAL, DPF_SYS_LOCAL, DpfError,  # noqa: F401
                  DpfLibraryMissing, Filter, Model, resample)
