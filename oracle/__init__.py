"""FP64 CPU oracle for Doppler resampling and FFT ionospheric correction.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import or execute anything in this package.  It shares
no code with the CUDA library (``paper_2508_04951_gb300``) and neither side
imports the other; the seeded waveform generators in ``synth`` feed both.

Everything here is plain numpy in float64/complex128, written from the paper
(arXiv 2508.04951, "Real-Time Doppler and Ionospheric Distortion Correction
Techniques for Arbitrary Waveforms Utilizing GPU Compute"):

* ``core``          -- range-rate factor (Eq. 1), time-dilated resampling
                       (Eq. 2) by windowed and exact Whittaker-Shannon
                       interpolation (Eq. 17, Sec. III-B, Table I) or by
                       frequency conversion (Sec. I, Table I), the carrier
                       term of a passband dilation, ionospheric
                       group delay (Eq. 3) and the FFT distortion / correction
                       (Eqs. 15-16).
* ``compression``   -- pulse compression bundled with the correction
                       (Sec. II-B, the pulse-compression path): the corrected
                       pulse's cross-correlation with a replica.
* ``predistortion`` -- the comparison waveforms of Sec. II-A/II-C: the Halpin
                       cubic (Eq. 4) and its closed-form root (Eqs. 11-14), the
                       pseudo-Chebyshev expansion (Eqs. 5-10, and the original
                       factor-4 coefficients of Eqs. 23-24), trapezoidal phase
                       integration, and the correlation-peak SNR-loss metric.

Every function is pinned by ``tests/test_oracle_*.py`` against values the
paper prints, closed forms, invariants, library special cases or brute force.
"""

from .core import (  # noqa: F401
    C_LIGHT,
    KAPPA,
    TECU,
    alpha,
    alpha_minus_one,
    i0,
    kaiser,
    kernel_windowed,
    resample_windowed,
    resample_exact,
    resample_exact_rows,
    carrier_term,
    frequency_conversion,
    resample,
    fft_length,
    bin_frequencies,
    iono_phase,
    iono_correct,
    iono_distort,
    correct,
    correct_bank,
)
