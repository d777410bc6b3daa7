"""GB300-native explicit discrete-ordinates transient step of the non-gray phonon BTE
(arXiv 2306.14181, Sec. 4).

The compute path is the C-ABI library ``libbte_gb300.so`` (hand-written CUDA for sm_103a,
declared in ``include/bte.h``); ``paper_2306_14181_gb300.bte`` is its thin ctypes binding and
``paper_2306_14181_gb300.autograd`` wraps the discrete adjoint as a ``torch.autograd.Function``.
``paper_2306_14181_gb300.inputs`` holds the seeded synthetic inputs.
"""
