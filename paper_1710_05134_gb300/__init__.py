"""GB300-native k-th eigenpair library: sparse LDL^T inertia counts, shifted solves and the
three-stage method of Lee, Hoshi, Sogabe, Miyatake and Zhang, on hand-written sm_103a kernels.

The compute path is libkep.so (C ABI in include/kep.h); ``kep`` is its thin Python binding."""
from .kep import (EXPORTED, KERNEL_CLASSES, FactorResult, KepError, KthEigenvalue, Problem, lib,  # noqa: F401
                  symbolic_info, multisection_points, multisection_update,
                  status_str, KEP_OK, KEP_ERR_INVALID, KEP_ERR_NOT_SPD, KEP_ERR_SINGULAR,
                  KEP_ERR_NOT_CONVERGED, KEP_ERR_CLUSTER, KEP_ERR_POOL, KEP_ERR_CUDA,
                  KEP_ERR_NONFINITE, KEP_ERR_NOMEM, KEP_ERR_TIMEOUT, KEP_INIT_LANCZOS, KEP_INIT_GERSHGORIN)
