"""GB300-native downsampled STFT-based synchrosqueezing transform.

The compute path is the CUDA library ``libsst.so`` (see ``include/sst.h``);
:mod:`paper_2003_07065_gb300.sst` is its thin ctypes binding.  Importing this
package does not load the library; ``sst`` loads it on first use and raises
if it has not been built.
"""
__all__ = ["sst", "signals", "workloads"]
