"""GB300-native 1D3V PIC-MCC particle loop for capacitively coupled RF oxygen
discharges (Bronold et al., ICPIG 2007).

The compute path is the CUDA library ``libo2pic.so`` (C ABI declared in
``include/o2pic.h``); this package holds its thin ctypes binding
(:mod:`.api`), the seeded input generators (:mod:`.inputs`) and the
cross-section data (:mod:`.xsec`).  The library is loaded on first use of
:mod:`.api`; there is no CPU fallback.
"""
__all__ = ["inputs", "xsec"]
