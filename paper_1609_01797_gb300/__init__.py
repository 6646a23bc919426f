"""GB300 (sm_103a) TASER detector: C ABI libtaser.so + thin torch binding.

The Python layer only marshals device pointers and the current CUDA stream into the
C ABI declared in include/taser.h; every step of the detector runs in CUDA kernels.
"""
from .api import (BPSK, GENERIC, JED_BPSK, QPSK, PRECISIONS, FLAG_ASCENT, build_T, detect, detect_monitored,  # noqa: F401
                  problem_size,
                  step_size, host_workspace_bytes, run_host, run_host_static,
                  unfolded_forward, unfolded_backward, UnfoldedTASER, ITEM_DTYPE, make_items,
                  uneven_workspace_bytes, tuning, detect_uneven, debug_report, debug_drop_copy)
