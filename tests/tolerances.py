"""Amplitude tolerances of the GPU parity tests.

complex128 (FP64 arithmetic): 1e-12 absolute, as the benchmark spec's tolerance for
FP64 results.

complex64 (FP32 arithmetic): the benchmark spec's 1e-5 taken relative to the size of
the amplitudes compared, not as an absolute number.  An absolute 1e-5 is far
looser than that for a state spread over 2^n amplitudes of size 2^{-n/2} (at
n = 20 it would accept an error of 1 % of every amplitude).  The check is
element by element:

    |got_i - want_i| <= k 1e-5 (|want_i| + scale),

scale = the root-mean-square magnitude of the nonzero entries of `want`
(2^{-n/2} for a state spread evenly, such as a QFT output), so an entry near
zero, the result of a cancellation, is held to 1e-5 of the typical entry and a
large one to 1e-5 of itself.  k (default 1) widens the bound for long random
circuits whose rounding errors add up over more gates.
"""
import numpy as np

from paper_1412_2293_gb300 import qs


def rms_scale(want):
    w = np.abs(np.asarray(want)).ravel()
    nz = w[w > 0]
    return float(np.sqrt(np.mean(nz * nz))) if nz.size else 0.0


def assert_amplitudes_close(got, want, dtype, k=1.0, err_msg=""):
    got = np.asarray(got)
    want = np.asarray(want)
    if dtype == qs.QS_C128:
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * k, err_msg=err_msg)
        return
    tol = 1e-5 * k
    np.testing.assert_allclose(got, want, rtol=tol, atol=tol * rms_scale(want), err_msg=err_msg)


def amplitude_error(got, want):
    """Largest |got - want| in units of the rms magnitude of want (for reports)."""
    s = rms_scale(want)
    return float(np.abs(np.asarray(got) - np.asarray(want)).max() / s) if s else 0.0
