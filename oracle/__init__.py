"""Plain FP64 CPU oracle of the Wilson-clover SAP-FGMRES method.

Test infrastructure only: imported by tests/, the smoke check and the
benchmark's CPU-baseline leg.  The library never imports it.
"""
