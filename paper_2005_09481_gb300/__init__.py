"""xe: an exact GB300 (sm_103a) X-engine correlator.

Computes, per frequency channel, the visibilities V_ij = sum_t x_i(t) conj(x_j(t)) for
i <= j over 4+4-bit complex voltages, exactly in int32 (Denman et al. 2020, sections 1
and 2.2).  The arithmetic runs in the CUDA library ``libxe.so`` behind a C ABI
(``include/xe.h``); ``paper_2005_09481_gb300.xe`` is the thin ctypes binding.
"""
__all__ = ["synth", "xe"]
