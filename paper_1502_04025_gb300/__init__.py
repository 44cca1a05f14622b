"""GB300-native Schwarz-preconditioned FGMRES solver for the Wilson-clover
Dirac equation (arXiv:1502.04025, Sec. 3).

The compute path is the C-ABI library ``libqdd.so`` (hand-written CUDA for
sm_103a); ``qdd`` is its thin ctypes binding.
"""
