"""GB300-native NUMARCK compression hot path.

The compute path is the CUDA library ``libnumarck.so`` (hand-written sm_103a kernels behind a
C ABI, declared in include/numarck.h). ``paper_1703_02438_gb300.numarck`` is the thin Python
binding over it; importing this package does not load the library.
"""

__all__ = ["numarck", "synth", "build"]
