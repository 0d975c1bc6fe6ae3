"""GB300-native matrix-free photoacoustic operator A and its adjoint A^T.

The compute path is the CUDA library behind ``include/pat.h`` (built in-tree
by ``paper_2609_29253_gb300.build``); ``_lib`` binds it with ctypes and ``api``
offers a ``Plan`` object, ``torch.autograd`` support and the reconstruction
loop on top.  ``workloads`` builds seeded synthetic inputs and does not touch
the GPU.  Heavy submodules load on first use.
"""
__version__ = "0.1.0"


def __getattr__(name):
    if name in ("Plan", "PatForward", "forward", "adjoint", "plan_from_workload", "system_taps"):
        from . import api

        return getattr(api, name)
    if name == "PatError":
        from ._lib import PatError

        return PatError
    raise AttributeError(name)
