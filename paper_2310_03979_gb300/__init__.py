"""GB300-native third-order SRM stochastic-wave sampler (arXiv 2310.03979).

The compute path is the CUDA library ``libsrm3.so`` behind the C ABI declared
in ``include/srm3.h``; ``paper_2310_03979_gb300.srm3`` is its ctypes binding.
Submodules are imported on first use, so ``workloads`` (pure input
definitions) loads without the CUDA library.
"""
import importlib

__all__ = ["srm3", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
