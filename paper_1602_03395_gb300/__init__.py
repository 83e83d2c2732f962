"""GB300-native free-flight expansion of wavefunctions (Deuar, arXiv:1602.03395).

The compute path lives in the CUDA library ``libffx.so`` built from ``csrc/``;
``paper_1602_03395_gb300.ffx`` is its thin Python binding.  Importing the
package does not load the library, so the input generators in ``inputs`` can be
used without a GPU.
"""
__all__ = ["inputs", "ffx"]
