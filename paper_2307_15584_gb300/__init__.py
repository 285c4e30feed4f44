"""GB300-native QMC point generation and integro-approximation.

The compute path is the CUDA library ``libqmc_gb300.so`` (sources under
``csrc/``); ``binding`` marshals arguments to its C-ABI.  Attributes of the
binding are loaded on first use, so ``import paper_2307_15584_gb300.inputs``
works on a machine without the built library while any compute call fails
loudly when the library is missing.
"""
from importlib import import_module

__all__ = ["binding", "inputs"]


def __getattr__(name):
    if name in ("binding", "inputs", "build", "autograd"):
        return import_module(f"{__name__}.{name}")
    return getattr(import_module(f"{__name__}.binding"), name)
