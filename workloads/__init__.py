"""Seeded synthetic inputs and workload parameter sets.

Shared by the tests, ``__graft_entry__.smoke()`` and ``bench.py``; imported by both the
CUDA-side tests and the oracle-side tests.  It holds none of the propagation method's
arithmetic: only physical parameter sets, a counter-based PRNG (SplitMix64, Steele,
Lea & Flood 2014), and random masks / random cross-spectral densities built from it.

The random masks are generated once here in float64 and handed to both sides; the CUDA
path receives them rounded to complex64, and the tests hand the oracle the same rounded
values, so both sides read identical input bytes.
"""
import math

import numpy as np

SEED = 20220305
C_LIGHT = 299792458.0

# Workload parameter sets (SI units).  Where a configuration leaves a parameter open, the
# value of the single-frequency GSM configuration is used (dxi = 20 um, lambda = 633 nm,
# sigma_S = 0.1 mm, sigma_mu = 0.05 mm, A = 1).
GSM_N32 = dict(name="gsm_fresnel_n32", N=32, dxi=20e-6, lam=633e-9, sigma_S=0.1e-3,
               sigma_mu=0.05e-3, A=1.0, z=0.5, P1=(16, 16))
GSM_APERTURE_LENS_N128 = dict(name="gsm_aperture_lens_fresnel_n128", N=128, dxi=20e-6,
                              lam=633e-9, sigma_S=0.1e-3, sigma_mu=0.05e-3, A=1.0,
                              aperture=0.8e-3, lens_f=0.3, z=0.3, P1=(64, 64))
GSM_APERTURE_FARFIELD_N128 = dict(GSM_APERTURE_LENS_N128, name="gsm_aperture_farfield_n128",
                                  lens_f=None)
POLYCHROMATIC_BATCH = dict(name="polychromatic_batch", Ns=(64, 96, 128), zs=(0.1, 0.5, 1.0, 5.0),
                           lam0=600e-9, fwhm_lam=100e-9, n_freq=16, dxi=20e-6,
                           sigma_S=0.1e-3, sigma_mu=0.05e-3)
PHASE_SCREEN_N256 = dict(name="phase_screen_gsm_n256", N=256, dxi=20e-6, lam=633e-9,
                         sigma_S=0.1e-3, sigma_mu=0.05e-3, A=1.0, z=0.5, corr_px=3.0,
                         P1=(128, 128))
# Zero padding with cropped output at the paper's padded sizes (Sec. 5.1 / 5.2 use N = 200 and
# Nz = 512): the N = 256 workload's phase-screen GSM source on that grid.
PADDED_PHASE_SCREEN_N200 = dict(name="padded_phase_screen_gsm_n200", N=200, Nz=512, dxi=20e-6,
                                lam=633e-9, sigma_S=0.1e-3, sigma_mu=0.05e-3, A=1.0, z=0.5,
                                corr_px=3.0, P1=(100, 100), sample_N=24, sample_Nz=62)
# The padded workload scaled to a size a full profiler capture can take (N^4 complex64 = 0.33 GB,
# above the L2 size; the same padding ratio 2.5).
PADDED_PHASE_SCREEN_N80 = dict(PADDED_PHASE_SCREEN_N200, name="padded_phase_screen_gsm_n80", N=80, Nz=200,
                               P1=(40, 40), sample_N=24, sample_Nz=60)
INVERSE_N96 = dict(name="amplitude_mask_gsm_n96", N=96, dxi=20e-6, lam=633e-9, sigma_S=0.1e-3,
                   sigma_mu=0.05e-3, A=1.0, z=1.0, P1=(48, 48))

_MASK64 = (1 << 64) - 1


def splitmix64(seed, idx):
    """SplitMix64 output for counter values `idx` (uint64 array) under `seed`:
    state = seed + (idx + 1) * 0x9E3779B97F4A7C15, then the published finaliser."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + (idx + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, n, offset=0):
    """n doubles in [0, 1) from the top 53 bits of SplitMix64(seed, offset + k)."""
    bits = splitmix64(seed, np.arange(offset, offset + n, dtype=np.uint64))
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _periodic_gaussian_blur(a, sigma):
    """Separable circular convolution with a normalised Gaussian of std `sigma` pixels."""
    K = int(math.ceil(4 * sigma))
    k = np.arange(-K, K + 1)
    w = np.exp(-(k ** 2) / (2.0 * sigma ** 2))
    w /= w.sum()
    out = np.zeros_like(a)
    for kk, ww in zip(k, w):
        out += ww * np.roll(a, kk, axis=0)
    out2 = np.zeros_like(out)
    for kk, ww in zip(k, w):
        out2 += ww * np.roll(out, kk, axis=1)
    return out2


def phase_screen(N, seed=SEED, corr_px=3.0):
    """Unit-modulus random phase screen m = t/|t|: t = exp(i phi0) blurred periodically by a
    Gaussian of std `corr_px` pixels, phi0 iid uniform in [0, 2 pi) (complex128, N x N)."""
    phi0 = 2.0 * np.pi * uniform01(seed, N * N).reshape(N, N)
    t = _periodic_gaussian_blur(np.exp(1j * phi0), corr_px)
    return t / np.abs(t)


def amplitude_mask(N, seed=SEED, lo=0.5, hi=1.0):
    """Real amplitude mask, iid uniform in [lo, hi] per pixel (complex128, N x N)."""
    u = uniform01(seed + 1, N * N).reshape(N, N)
    return (lo + (hi - lo) * u).astype(np.complex128)


def random_modes(N, seed=SEED, n_modes=3):
    """Random smooth-ish complex fields phi_k (n_modes, N, N) and positive weights w_k,
    used to build a Hermitian non-negative definite test CSDA sum_k w_k phi_k*(x1) phi_k(x2)."""
    u = uniform01(seed + 2, 2 * n_modes * N * N).reshape(2, n_modes, N, N)
    re = _periodic_gaussian_blur_stack(u[0] - 0.5, 1.0)
    im = _periodic_gaussian_blur_stack(u[1] - 0.5, 1.0)
    w = 0.5 + uniform01(seed + 3, n_modes)
    return re + 1j * im, w


def _periodic_gaussian_blur_stack(a, sigma):
    return np.stack([_periodic_gaussian_blur(x, sigma) for x in a])


def random_csd(N, seed=SEED, n_modes=3):
    """Hermitian, non-negative definite CSDA (N,N,N,N) complex128 from random_modes."""
    phi, w = random_modes(N, seed, n_modes)
    W = np.zeros((N, N, N, N), dtype=np.complex128)
    for k in range(n_modes):
        W += w[k] * np.conj(phi[k])[:, :, None, None] * phi[k][None, None, :, :]
    return W


def polychromatic_samples(lam0=600e-9, fwhm_lam=100e-9, n_freq=16):
    """Gaussian spectrum S0(omega) ~ exp(-(omega-omega0)^2 / (2 sigma_w^2)), omega0 = 2 pi c/lam0,
    FWHM_omega = 2 pi c fwhm_lam / lam0^2; n_freq samples uniform in omega over
    omega0 +- 2 sigma_w (endpoints included).  Returns (lambdas, weights)."""
    w0 = 2 * np.pi * C_LIGHT / lam0
    fwhm_w = 2 * np.pi * C_LIGHT * fwhm_lam / lam0 ** 2
    sw = fwhm_w / (2 * math.sqrt(2 * math.log(2)))
    om = np.linspace(w0 - 2 * sw, w0 + 2 * sw, n_freq)
    return 2 * np.pi * C_LIGHT / om, np.exp(-((om - w0) ** 2) / (2 * sw ** 2))


def to_c64(a):
    """Round a complex128 input to the complex64 bytes the CUDA path reads."""
    return np.ascontiguousarray(np.asarray(a).astype(np.complex64))
