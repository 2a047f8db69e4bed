"""GB300-native Gauss-Newton accelerated MPPI (arXiv 2512.04579).

The solver lives in the CUDA library ``libgnmppi.so`` (C ABI, ``include/gnmppi.h``);
``paper_2512_04579_gb300.gnmppi`` is its thin ctypes binding.  Importing this
package loads nothing: the binding loads the library on first use and raises
if it is missing.
"""
__all__ = ["gnmppi", "inputs"]
