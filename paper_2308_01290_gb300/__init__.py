"""GB300-native one-step Z / rho_e estimation for dual-energy CT (arXiv 2308.01290).

The compute path is the CUDA library ``librecon.so`` (sources in ``csrc/``,
C ABI in ``include/recon.h``); ``recon`` is its ctypes binding and
``build_lib`` compiles it for sm_103a.  Import ``paper_2308_01290_gb300.recon``
to load the library; it raises ImportError when the library is not built.
"""
