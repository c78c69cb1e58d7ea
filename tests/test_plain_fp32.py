"""The plain FP32 CPU path (the timed multi-threaded CPU baseline) against the FP64 oracle.

It is a baseline, not a reference; this only makes sure that the CPU number the benchmark
reports is for a propagation that computes the same thing: the GSM x aperture x thin lens source
of the N = 128 workload, at grids the oracle finishes in a second."""
import numpy as np
import pytest

import oracle as O
from oracle import plain_fp32 as P
import workloads as WL

CFG = WL.GSM_APERTURE_LENS_N128


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("N", [16, 24])
def test_plain_fp32_matches_oracle(N):
    pytest.importorskip("scipy.fft")
    dxi = CFG["dxi"]
    radius = CFG["aperture"] * N / 128  # the aperture's 40 pixels scaled onto the small grid
    m = O.circle_aperture(N, dxi, radius) * O.thin_lens(N, dxi, CFG["lam"], CFG["lens_f"])
    W0 = O.apply_mask(O.gsm_source(N, dxi, CFG["sigma_S"], CFG["sigma_mu"], 1.0), m)
    Wr, dxr = O.propagate_fft(W0, dxi, CFG["lam"], CFG["z"])
    W, S, mu, dx = P.propagate_gsm_fp32(N, dxi, CFG["lam"], CFG["z"], CFG["sigma_S"], CFG["sigma_mu"], 1.0,
                                        mask=m, workers=2)
    assert dx == pytest.approx(dxr, rel=1e-15)
    assert _rel(W, Wr) < 1e-5
    Sr = np.real(O.spectral_density(Wr))
    assert _rel(S, Sr) < 1e-5
    mur = O.degree_of_coherence(Wr, N // 2, N // 2)
    keep = Sr >= 1e-6 * Sr.max()
    assert np.abs(mu - mur)[keep].max() < 1e-4


def test_plain_fp32_rejects_odd_n():
    with pytest.raises(ValueError):
        P.propagate_gsm_fp32(15, 1e-5, 6e-7, 0.3, 1e-4, 5e-5)


def test_plain_fp32_padded_matches_padded_oracle():
    # the padded workload's CPU leg: the source on the Nz grid (zeros around it), FFTs at Nz, the
    # central N^4 block
    pytest.importorskip("scipy.fft")
    N, Nz, z = 12, 30, 0.5
    m = WL.phase_screen(N, seed=WL.SEED, corr_px=3.0)
    o = (Nz - N) // 2
    mp = np.zeros((Nz, Nz), dtype=np.complex128)
    mp[o:o + N, o:o + N] = m
    W, S, mu, dx = P.propagate_gsm_fp32(Nz, CFG["dxi"], CFG["lam"], z, CFG["sigma_S"], CFG["sigma_mu"], 1.0,
                                        mask=mp, workers=2)
    Wc = W[o:o + N, o:o + N, o:o + N, o:o + N]
    W0 = O.apply_mask(O.gsm_source(N, CFG["dxi"], CFG["sigma_S"], CFG["sigma_mu"]), m)
    Wr, dxr = O.propagate_padded(W0, CFG["dxi"], CFG["lam"], z, Nz)
    assert dx == pytest.approx(dxr, rel=1e-15)
    assert _rel(Wc, Wr) < 1e-5
