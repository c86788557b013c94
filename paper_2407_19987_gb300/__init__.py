"""GB300-native HOBO contraction and batched Metropolis annealing.

The hot path (arXiv 2407.19987: HOBO tensor contracted with a batch of
binary states, Sec. II.C / IV.C, driven by simulated annealing, Sec. II.D.1)
runs in the CUDA kernels of libhobo.so behind the C ABI in include/hobo.h;
this package is its Python binding.
"""
from .binding import (aggregate, HOBO_ERR_ARG, HOBO_ERR_CUDA, HOBO_ERR_NOT_EXACT, HOBO_ERR_OOM, HOBO_ERR_ORDER,
                      HOBO_ERR_TIMEOUT, HOBO_ERR_UNSUPPORTED, MLP, SELECT_ORDER, SELECT_THRESHOLD, anneal_learned, HOBO_BATCH_GRAPH, HOBO_BATCH_PER_INSTANCE_PLAIN, HOBO_BATCH_PER_INSTANCE_TUNED, Batch,
                      HOBO_ANNEAL_PLAIN, HOBO_ANNEAL_TUNED, HOBO_FORCE_DENSE, HOBO_FORCE_SPARSE,
                      HOBO_INTEGER, HOBO_RESCORE_CUDA_CORES, HOBO_SPLIT2, HOBO_SPLIT3, PATH_AUTO, PATH_TENSOR_CORE, PATH_TENSOR_CORE_F32ACC, PATH_TERMS, HoboError,
                      Instance, load_library, probe_l2_read, selftest_philox, version, words)

__all__ = ["aggregate", "HOBO_ERR_ARG", "HOBO_ERR_CUDA", "HOBO_ERR_NOT_EXACT", "HOBO_ERR_OOM", "HOBO_ERR_ORDER",
           "HOBO_ERR_TIMEOUT", "HOBO_ERR_UNSUPPORTED", "Instance", "MLP", "anneal_learned", "SELECT_ORDER", "SELECT_THRESHOLD", "Batch", "HOBO_BATCH_GRAPH", "HOBO_BATCH_PER_INSTANCE_TUNED",
           "HOBO_BATCH_PER_INSTANCE_PLAIN", "HoboError", "load_library", "version", "words", "HOBO_INTEGER",
           "HOBO_FORCE_SPARSE", "HOBO_FORCE_DENSE", "HOBO_RESCORE_CUDA_CORES", "HOBO_SPLIT2", "HOBO_SPLIT3", "HOBO_ANNEAL_TUNED",
           "HOBO_ANNEAL_PLAIN", "PATH_AUTO", "PATH_TERMS", "PATH_TENSOR_CORE", "PATH_TENSOR_CORE_F32ACC", "probe_l2_read", "selftest_philox"]
