"""GB300 (sm_103a) implementation of the Monte-Carlo estimator of Pauli-Z
expectation values of parameterised IQP circuits, its gradient and the MMD^2
loss built from it (arxiv 2501.04776, Secs. 2.1-2.4 and 3.3.1).

The compute path is the C ABI in include/iqp.h, implemented by the CUDA
kernels under csrc/ and built into libiqp_gb300.so by build.py. `api` is the
PyTorch binding; `inputs` produces seeded synthetic workloads.
"""
from . import inputs  # noqa: F401  (pure numpy; no CUDA needed)

__all__ = ["inputs", "api"]


def __getattr__(name):
    if name == "api":
        import importlib
        return importlib.import_module(__name__ + ".api")
    raise AttributeError(name)
