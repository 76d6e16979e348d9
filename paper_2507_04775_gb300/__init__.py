"""GB300-native CKKS hybrid key-switching engine (FIDESlib, arXiv 2507.04775).

The compute path is the CUDA library ``_build/libfides.so`` (hand-written
sm_103a kernels behind the C ABI of ``include/fides.h``); ``fides`` is its
ctypes binding.  Build with ``paper_2507_04775_gb300.build.build()``.
"""
from .fides import (Context, FidesError, Key, find_primes, lib, to_device, to_host, version, EXPORTS,  # noqa: F401
                    LIB_PATH, trace_enable, trace_reset, trace_read, kernel_launches, measure_modmul_peak, Batch, Op,
                    OP_HMULT, OP_ROTATE, OP_RESCALE, Server, Completion, now_ns, FAULT_LAUNCH_ERROR, FAULT_STALL)
