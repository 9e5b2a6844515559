"""libpwa: B300-native likelihood, gradient, Hessian-vector products and
Newton-CG fit for partial-wave analysis (method of arXiv:2403.09225).

The compute path is the CUDA library ``_lib/libpwa.so`` behind the C ABI of
``include/pwa.h``; ``binding`` marshals arguments to it, ``autograd`` wraps it
as a ``torch.autograd.Function``, ``workload`` generates seeded synthetic
inputs.  Importing the package does not load the library; the first use of
the binding does, and fails loudly when it is not built.
"""
