"""One-ring neighbor nodes and elements of generic meshes on GB300 (sm_103a).

The compute path is the CUDA library ``libnn.so`` (sources in ``csrc/``,
C interface in ``include/nn.h``); ``nn`` is its thin ctypes binding, which
loads the library on first use, so ``meshgen`` stays importable on machines
without a GPU.
"""
