"""GB300-native complex band structure by the Sakurai-Sugiura contour-integral method.

The compute path lives in ``libcbs.so`` (CUDA, sm_103a) behind a C ABI; ``cbs`` is its
thin ctypes binding and ``synth`` generates seeded synthetic inputs.  Importing the
package loads nothing; ``paper_1709_09347_gb300.cbs`` loads the library on first use.
"""
__all__ = ["cbs", "synth"]
