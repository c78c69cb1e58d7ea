"""Plain FP32 CPU path of one propagation: a timed CPU baseline, not a parity reference.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): only ``bench.py``'s CPU legs and
``tests/`` use it; the product path never imports it.

The paper computes the method as whole-array operations and library FFTs on the host
(Sec. 3, Algorithms 2 and 3).  This module restates those steps in complex64, with
``scipy.fft`` on every host core, so that the GPU numbers can be set beside the method as a
plain multi-threaded CPU program runs it (the FP64 oracle, by contrast, is slow on purpose):

  1. source: W0 = A gx(a, c) gy(b, d) conj(m(a, b)) m(c, d)        (Sec. 5.4 GSM with the
     standard signs, times the mask m as Y* W Y of Sec. 5.3 / T* W T of Sec. 2.2);
  2. input propagators q*(xi1) q(xi2)                               (Algorithm 3, Eq. q_factor);
  3. forward 2D FFT over the point-2 pair, inverse-sign unnormalised 2D FFT over the point-1
     pair                                                           (Algorithm 2);
  4. output propagators q*(x1) q(x2) and the scale dxi^4/(lambda z)^2;
  5. S = Re W(x, x) and mu(P1, x)                                   (Algorithm 4, Eq. defMu).

Centring (the DFTs act on indices n - N/2): for even N, multiplying the input by (-1)^n and the
output by (-1)^k turns the centred sums into plain FFTs; the leftover constant exp(-+ i pi N/2)
per axis cancels between the forward and the inverse pair.  Both checkerboards are folded into
the per-axis factors.  The chirp phases are taken mod 1 turn in FP64 before the FP32 cast (the
single-precision phase of |x|^2/(lambda z) would otherwise lose the fractional turns).
"""
import os

import numpy as np

__all__ = ["propagate_gsm_fp32", "host_cores"]


def host_cores():
    """Threads the FFTs use: every core this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _coords(N, d):
    n = np.arange(N, dtype=np.float64)
    return (n - N / 2) * d, (N / 2 - n) * d


def _chirp(N, d, lam, z, sign):
    """exp(sign i pi |r|^2/(lambda z)) (-1)^(i+j) on the N x N grid of spacing d, complex64."""
    x, y = _coords(N, d)
    turns = (x[:, None] ** 2 + y[None, :] ** 2) / (2.0 * lam * z)
    turns = turns - np.floor(turns)
    n = np.arange(N)
    chk = np.where((n[:, None] + n[None, :]) % 2 == 0, 1.0, -1.0)
    return (chk * np.exp(sign * 2j * np.pi * turns)).astype(np.complex64)


def _gsm_axis(N, dxi, sigma_S, sigma_mu, coords):
    u = coords[:, None]
    v = coords[None, :]
    return np.exp(-(u * u + v * v) / (4 * sigma_S ** 2) - (u - v) ** 2 / (2 * sigma_mu ** 2)).astype(np.float32)


def propagate_gsm_fp32(N, dxi, lam, z, sigma_S, sigma_mu, A=1.0, mask=None, P1=None, workers=None):
    """One Fresnel propagation of a GSM source times an optional complex N x N mask, in complex64.

    Returns (W, S, mu, dx): the propagated CSDA W[a', b', c', d'] (point 1 first), S (float32),
    mu(P1, .) (complex64) and the output sampling dx = lambda z / (N dxi)."""
    import scipy.fft as sfft
    if N < 2 or N % 2:
        raise ValueError("N must be even")
    workers = workers or host_cores()
    P1 = P1 or (N // 2, N // 2)
    x, y = _coords(N, dxi)
    gx = _gsm_axis(N, dxi, sigma_S, sigma_mu, x)
    gy = _gsm_axis(N, dxi, sigma_S, sigma_mu, y)
    F = _chirp(N, dxi, lam, z, +1)  # q(xi2) (-1)^(c+d); point 1 takes its conjugate
    if mask is not None:
        F = F * np.asarray(mask, dtype=np.complex64)
    Fc = np.conj(F)
    W = np.empty((N, N, N, N), dtype=np.complex64)
    A32 = np.float32(A)
    for a in range(N):  # steps 1-2, one point-1 row at a time
        W[a] = (A32 * Fc[a][:, None, None] * gy[:, None, :]) * (gx[a][:, None] * F)[None, :, :]
    W = sfft.fft2(W, axes=(2, 3), workers=workers, overwrite_x=True)  # step 3, point 2
    W = sfft.ifft2(W, axes=(0, 1), norm="forward", workers=workers, overwrite_x=True)  # point 1
    dx = lam * z / (N * dxi)
    E = _chirp(N, dx, lam, z, +1)  # q(x2) (-1)^(c'+d')
    s = np.float32(dxi ** 4 / (lam * z) ** 2)
    Ec = np.conj(E) * s
    for a in range(N):  # step 4
        W[a] *= Ec[a][:, None, None] * E[None, :, :]
    n = np.arange(N)
    S = np.real(W[n[:, None], n[None, :], n[:, None], n[None, :]]).astype(np.float32)  # step 5
    den = S * S[P1]
    mu = np.zeros((N, N), dtype=np.complex64)
    ok = den > 0
    mu[ok] = W[P1[0], P1[1]][ok] / np.sqrt(den[ok])
    return W, S, mu, dx
