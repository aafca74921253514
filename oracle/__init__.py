"""FP64 CPU oracle of the funnel transform.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import, call or execute it.  It shares no code, table
or helper with the CUDA library; both sides take their inputs from the seeded
generator in ``paper_1904_09409_gb300.synth`` (pictures only, no transform
arithmetic).

Modules
-------
transform     the transform step by step (Sec. 3.1 steps 1-4, Sec. 4.2 padding)
funnel_direct brute-force evaluation of the same definition without any FFT
peaks_ref     the list-based peak detection of Sec. 4.4 and eqs. (22)-(25)
adjoint_ref   the exact transpose of the (linear) transform, for gradients
verification  the line verification of Sec. 4.5 (band profile along a candidate line)
"""
from .transform import (centred, pad_rows, fourier_y, nvmt_positions, nvmt,
                         fourier_xprime, inverse_fourier_omega2, funnel_ref,
                         interp_weights, inverse_funnel_ref)
from .funnel_direct import funnel_direct
from .peaks_ref import peaks_ref, peak_to_line, inverse_peak_to_line
from .adjoint_ref import adjoint_ref, map_loss_grad_ref
from .verification import band_profile, verify_ref

__all__ = [
    "centred", "pad_rows", "fourier_y", "nvmt_positions", "nvmt", "fourier_xprime",
    "inverse_fourier_omega2", "funnel_ref", "interp_weights", "inverse_funnel_ref",
    "funnel_direct", "peaks_ref", "peak_to_line", "inverse_peak_to_line",
    "adjoint_ref", "map_loss_grad_ref", "band_profile", "verify_ref",
]
