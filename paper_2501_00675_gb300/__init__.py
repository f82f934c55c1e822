"""GB300 (sm_103a) evaluator of combinatorial-summation (CoS) Feynman-diagram graphs.

The compute path is the CUDA library libcosgpu.so (C ABI in include/cos.h);
this package holds its sources, the in-tree build step and a ctypes binding
whose functions carry the C names and only marshal arguments.
"""
from .binding import (  # noqa: F401
    COS_OK, COS_ERR_INVALID, COS_ERR_OOM, COS_ERR_CUDA, COS_ERR_TIMEOUT, COS_ERR_OVERFLOW, COS_ERR_STATE,
    COS_ERR_BUSY,
    COS_MODE_FP64, COS_MODE_FP32_MIXED, COS_MODE_COUNT_I64, COS_EVAL_ABS, COS_T_DEVICE_DS, COS_T_HOST, COS_T_SAMPLE_MAJOR, COS_T_BORROW,
    Batch, CosError, CosTuning, Graph, Metropolis, ResidentServer, load_library, library_path, probe_fma_rate, evaluate_batch,
)
