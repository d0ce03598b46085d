"""GB300-native matrix-free Poisson element operator (AxLocal / CEED BK5).

The compute path is the C-ABI library ``libax.so`` (hand-written CUDA for
sm_103a); ``paper_2504_07042_gb300.ax`` is its thin ctypes binding and
``paper_2504_07042_gb300.inputs`` builds seeded synthetic meshes.
Importing the package does not load the library.
"""
__all__ = ["ax", "inputs"]
