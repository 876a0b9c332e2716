"""Multi-robot MotionValidation / FindFirstConflict on GB300 (sm_103a).

``workloads`` draws seeded inputs (numpy only); ``mrv`` binds the C ABI of
``libmrv.so`` (built in-tree by ``build.build()``).  Importing the package
loads nothing: the CUDA library is loaded on first use and a missing build is
an error, never a fallback.
"""
