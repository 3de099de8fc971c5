"""Plain FP64 CPU oracle of the swept-source holographic OCT reconstruction.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` may import or run anything in this
package.  The product path (the C-ABI library and its Python binding) never calls
it and shares no code with it.

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against things the paper or the mathematics fix (printed numbers, the literal
convolution form of Eq. 6, brute-force sums, Parseval, the Dirichlet kernel, and
point scatterers reconstructing at closed-form positions).  No function is left
"parity unpinned".
"""

from .ssoct_oracle import (  # noqa: F401
    start_wavelength,
    scale_factors,
    reconstructed_pixel,
    fresnel_limit,
    synthetic_wavelength,
    axial_range,
    coherence_length,
    rescale_taps,
    rescale,
    fresnel_prefactor,
    fresnel,
    axial,
    reconstruct,
    intensity,
    cuts,
    pixel_sample,
)
from . import aberration  # noqa: F401,E402  (Zernike pupil, sharpness and its gradient)
