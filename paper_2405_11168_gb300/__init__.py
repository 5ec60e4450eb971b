"""GB300-native tetrahedral-stencil FFT homogenization solver (arXiv 2405.11168).

The compute path is the CUDA library ``libhs.so`` (C ABI: ``include/hs.h``);
``paper_2405_11168_gb300.hs`` is its thin ctypes binding.  Importing this
package loads nothing; ``hs.load()`` loads the library and raises if it is
missing.
"""
