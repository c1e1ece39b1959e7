"""GB300 (sm_103a) MPPI + Gate-SDF control-step library.

The compute path is the CUDA library ``libmppi_gb300.so`` built from
``csrc/`` (see ``build.py``); ``binding`` is its thin ctypes binding with the
C-ABI names of ``include/mppi.h``.  There is no CPU fallback: loading the
binding without the built library raises.
"""

__all__ = ["binding", "build"]
