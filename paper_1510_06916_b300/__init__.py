"""NXgraph DSSS update sweep on one B300 (sm_103a).

The compute path is the C-ABI library ``csrc/libnxgraph.so`` (hand-written CUDA);
``nxgraph`` is its thin ctypes binding and ``autograd`` wraps the
weighted-PageRank adjoint as a ``torch.autograd.Function``.
"""
