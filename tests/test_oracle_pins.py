"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties an oracle function to the paper's printed numbers, to brute force, to an
independent closed form, or to an exact invariant, so that a dropped term, a wrong sign, a
swapped index or a transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as WL

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")

DXI, LAM, SS, SM = 20e-6, 633e-9, 0.1e-3, 0.05e-3


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _rand_mask(N, seed):
    u = WL.uniform01(seed, 2 * N * N).reshape(2, N, N)
    return (u[0] + 0.2) * np.exp(2j * np.pi * u[1])


# --------------------------------------------------------------------------- brute force
@pytest.mark.parametrize("N", [4, 6, 8])
@pytest.mark.parametrize("farfield", [False, True])
def test_fft_route_equals_direct_quadrature(N, farfield):
    """Algorithm 2 route == brute-force quadrature of Eq. W_general (no chirp/DFT
    factorisation), on a non-symmetric masked GSM source and a random CSDA."""
    W0 = O.apply_mask(O.gsm_source(N, DXI, SS, SM, 1.3), _rand_mask(N, 7))
    a, dxa = O.propagate_fft(W0, DXI, LAM, 0.5, farfield)
    b, dxb = O.propagate_direct(W0, DXI, LAM, 0.5, farfield)
    assert dxa == dxb
    assert rel(a, b) < 1e-11
    W1 = WL.random_csd(N, seed=11, n_modes=2)
    a, _ = O.propagate_fft(W1, DXI, LAM, 0.3, farfield)
    b, _ = O.propagate_direct(W1, DXI, LAM, 0.3, farfield)
    assert rel(a, b) < 1e-11


def test_direct_quadrature_is_not_symmetric_in_points():
    """A conjugation or point swap in the kernel must show: propagating the transposed
    (point-swapped) source of a non-Hermitian array gives a different result."""
    N = 4
    rng = np.random.default_rng(3)
    W0 = rng.standard_normal((N,) * 4) + 1j * rng.standard_normal((N,) * 4)
    a, _ = O.propagate_direct(W0, DXI, LAM, 0.5)
    b, _ = O.propagate_direct(W0.transpose(2, 3, 0, 1), DXI, LAM, 0.5)
    assert rel(a, b.transpose(2, 3, 0, 1)) > 1e-2


# --------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("farfield", [False, True])
def test_gsm_closed_form_equals_fft_route(farfield):
    """Continuous Gaussian integral == discrete route once the grid holds the beam."""
    N = 64
    W0 = O.gsm_source(N, DXI, SS, SM, 1.0)
    a, _ = O.propagate_fft(W0, DXI, LAM, 0.5, farfield)
    c = O.gsm_closed_form(N, DXI, LAM, 0.5, SS, SM, 1.0, farfield)
    assert rel(a, c) < 1e-7


def test_gsm_closed_form_matches_textbook_beam():
    """Closed form vs the textbook GSM beam: S(X) = (A/Delta^2) exp(-|X|^2/(2 sigma_S^2 Delta^2)),
    |mu| = exp(-|X1-X2|^2/(2 sigma_mu^2 Delta^2)), arg W = k(|X2|^2 - |X1|^2)/(2 R(z))."""
    N, z, A = 64, 0.5, 1.7
    Wc = O.gsm_closed_form(N, DXI, LAM, z, SS, SM, A, False)
    Delta, Rz = O.gsm_beam_parameters(LAM, z, SS, SM)
    dx = O.output_sampling(N, DXI, LAM, z)
    X, Y = O.axis_coords(N, dx)
    S = np.real(O.spectral_density(Wc))
    r2 = X[:, None] ** 2 + Y[None, :] ** 2
    S_tb = (A / Delta ** 2) * np.exp(-r2 / (2 * SS ** 2 * Delta ** 2))
    assert rel(S, S_tb) < 1e-10
    k = 2 * np.pi / LAM
    for (a, b) in [(32, 32), (20, 40), (45, 30)]:
        for (c, d) in [(32, 35), (28, 36), (40, 22)]:
            w = Wc[a, b, c, d]
            d2 = (X[a] - X[c]) ** 2 + (Y[b] - Y[d]) ** 2
            mu = w / np.sqrt(S[a, b] * S[c, d])
            assert abs(abs(mu) - np.exp(-d2 / (2 * SM ** 2 * Delta ** 2))) < 1e-10
            ph = k * ((X[c] ** 2 + Y[d] ** 2) - (X[a] ** 2 + Y[b] ** 2)) / (2 * Rz)
            assert abs(np.angle(mu * np.exp(-1j * ph))) < 1e-9


@pytest.mark.parametrize("N", [16, 32])
@pytest.mark.parametrize("farfield", [False, True])
@pytest.mark.parametrize("lens", [None, 0.3])
def test_separable_quadrature_equals_fft_route(N, farfield, lens):
    """Per-axis N x N quadrature (Kronecker) == 4D Algorithm-2 route, any N."""
    W0 = O.gsm_source(N, DXI, SS, SM, 0.8)
    if lens is not None:
        W0 = O.apply_mask(W0, O.thin_lens(N, DXI, LAM, lens))
    a, _ = O.propagate_fft(W0, DXI, LAM, 0.5, farfield)
    b = O.gsm_separable_quadrature(N, DXI, LAM, 0.5, SS, SM, 0.8, farfield, lens_f=lens)
    assert rel(a, b) < 1e-12


def test_propagate_rows_equals_fft_route():
    N = 16
    W0 = O.apply_mask(O.gsm_source(N, DXI, SS, SM), _rand_mask(N, 5))
    full, _ = O.propagate_fft(W0, DXI, LAM, 0.4)
    rows = [(8, 8), (3, 11), (15, 0)]
    got = O.propagate_rows(lambda i, j: W0[i, j], N, DXI, LAM, 0.4, rows)
    for r, (a, b) in enumerate(rows):
        assert rel(got[r], full[a, b]) < 1e-12
    gotf = O.propagate_rows(lambda i, j: W0[i, j], N, DXI, LAM, 0.4, rows, farfield=True)
    fullf, _ = O.propagate_fft(W0, DXI, LAM, 0.4, True)
    assert rel(gotf[1], fullf[3, 11]) < 1e-12


def test_propagate_rows_blocks_equals_fft_route():
    N = 12
    W0 = O.apply_mask(O.gsm_source(N, DXI, SS, SM), _rand_mask(N, 6))
    rows = [(6, 6), (1, 10)]
    for ff in (False, True):
        full, _ = O.propagate_fft(W0, DXI, LAM, 0.4, ff)
        got = O.propagate_rows_blocks(lambda i: W0[i], N, DXI, LAM, 0.4, rows, ff)
        for r, (a, b) in enumerate(rows):
            assert rel(got[r], full[a, b]) < 1e-12


@pytest.mark.parametrize("farfield", [False, True])
def test_propagate_rows_gsm_equals_fft_route(farfield):
    N = 14
    m = _rand_mask(N, 8)
    W0 = O.apply_mask(O.gsm_source(N, DXI, SS, SM, 1.4), m)
    full, _ = O.propagate_fft(W0, DXI, LAM, 0.45, farfield)
    rows = [(7, 7), (2, 11), (13, 0)]
    got = O.propagate_rows_gsm(m, N, DXI, LAM, 0.45, SS, SM, 1.4, rows, farfield)
    for r, (a, b) in enumerate(rows):
        assert rel(got[r], full[a, b]) < 1e-12


# --------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("farfield", [False, True])
def test_parseval_and_trace(farfield):
    """Power conservation with the scale of reading R4: sum|W_B|^2 dx^4 = sum|W0|^2 dxi^4 and
    sum S_B dx^2 = sum S_0 dxi^2 (the chirps are unimodular, the DFTs unitary up to N)."""
    N = 12
    W0 = O.apply_mask(O.gsm_source(N, DXI, SS, SM), _rand_mask(N, 9))
    WB, dx = O.propagate_fft(W0, DXI, LAM, 0.7, farfield)
    assert abs(np.sum(np.abs(WB) ** 2) * dx ** 4 / (np.sum(np.abs(W0) ** 2) * DXI ** 4) - 1) < 1e-12
    S0 = np.real(O.spectral_density(W0))
    SB = np.real(O.spectral_density(WB))
    assert abs(SB.sum() * dx ** 2 / (S0.sum() * DXI ** 2) - 1) < 1e-12


def test_hermitian_and_non_negative_definite():
    """W(x2, x1) = W*(x1, x2) (Sec. 3.3) and the non-negative definiteness constraint of Sec. 2.1,
    for a random CSDA and its propagation."""
    N = 6
    W0 = WL.random_csd(N, seed=21, n_modes=4)
    WB, _ = O.propagate_fft(W0, DXI, LAM, 0.2)
    for W in (W0, WB):
        M = W.reshape(N * N, N * N)
        assert np.abs(M - M.conj().T).max() < 1e-12 * np.abs(M).max()
        ev = np.linalg.eigvalsh((M + M.conj().T) / 2)
        assert ev.min() > -1e-11 * ev.max()
    assert np.linalg.matrix_rank(WB.reshape(N * N, N * N), tol=1e-9 * np.abs(WB).max()) == 4


def test_thin_lens_cancels_input_propagator():
    """Eq. qprop3: a lens of focal length f = z in the source plane cancels the input
    propagators, so Fresnel with the lens equals far field without it."""
    N = 16
    W0 = O.apply_mask(O.gsm_source(N, DXI, SS, SM), O.circle_aperture(N, DXI, 5.5 * DXI))
    a, _ = O.propagate_fft(O.apply_mask(W0, O.thin_lens(N, DXI, LAM, 0.3)), DXI, LAM, 0.3)
    b, _ = O.propagate_fft(W0, DXI, LAM, 0.3, farfield=True)
    assert rel(a, b) < 1e-13
    c, _ = O.propagate_fft(W0, DXI, LAM, 0.3)
    assert rel(c, b) > 1e-3


def test_s_non_negative_and_mu_bounded():
    N = 16
    W0 = O.apply_mask(O.gsm_source(N, DXI, SS, SM), O.circle_aperture(N, DXI, 6 * DXI))
    WB, _ = O.propagate_fft(W0, DXI, LAM, 0.5)
    S = np.real(O.spectral_density(WB))
    assert S.min() > -1e-12 * S.max()
    mu = O.degree_of_coherence(WB, 8, 8)
    assert np.abs(mu).max() <= 1 + 1e-12
    assert abs(mu[8, 8] - 1) < 1e-13


def test_coherent_source_has_unit_coherence():
    """A rank-one CSDA phi*(x1) phi(x2) is fully coherent: |mu| = 1 wherever S > 0, before and
    after propagation (Eq. defMu, Algorithm coherence)."""
    N = 8
    phi = _rand_mask(N, 31)
    W0 = np.conj(phi)[:, :, None, None] * phi[None, None]
    for W in (W0, O.propagate_fft(W0, DXI, LAM, 0.5)[0]):
        mu = O.degree_of_coherence(W, 3, 5)
        assert np.allclose(np.abs(mu), 1.0, atol=1e-12)
    mu = O.degree_of_coherence(W0, 3, 5)
    assert np.allclose(mu, np.conj(phi[3, 5]) * phi / (np.abs(phi[3, 5]) * np.abs(phi)), atol=1e-13)


def test_mu_zero_where_s_vanishes():
    N = 8
    W0 = O.apply_mask(O.gsm_source(N, DXI, SS, SM), O.circle_aperture(N, DXI, 2 * DXI))
    mu = O.degree_of_coherence(W0, 4, 4)
    assert mu[0, 0] == 0 and abs(mu[4, 5] - np.exp(-DXI ** 2 / (2 * SM ** 2))) < 1e-13


# --------------------------------------------------------------------------- source models
def test_gsm_source_special_cases():
    """S0(xi) = A exp(-|xi|^2/(2 sigma_S^2)); mu0 = exp(-|xi1-xi2|^2/(2 sigma_mu^2)) (Sec. 5.4)."""
    N, A = 10, 2.5
    W0 = O.gsm_source(N, DXI, SS, SM, A)
    x, y = O.axis_coords(N, DXI)
    S = np.real(O.spectral_density(W0))
    assert np.allclose(S, A * np.exp(-(x[:, None] ** 2 + y[None, :] ** 2) / (2 * SS ** 2)), rtol=1e-14)
    mu = O.degree_of_coherence(W0, 2, 7)
    d2 = (x[:, None] - x[2]) ** 2 + (y[None, :] - y[7]) ** 2
    assert np.allclose(mu, np.exp(-d2 / (2 * SM ** 2)), rtol=1e-13)
    assert x[N // 2] == 0 and y[N // 2] == 0 and y[0] > 0 and x[0] < 0


def test_circle_aperture_brute_force():
    N, r = 24, 7.0
    Y = O.circle_aperture(N, DXI, r * DXI)
    cnt = 0
    for i in range(N):
        for j in range(N):
            inside = (i - N // 2) ** 2 + (N // 2 - j) ** 2 <= r * r
            assert Y[i, j] == (1.0 if inside else 0.0)
            cnt += inside
    assert cnt == int(Y.sum()) == 149  # lattice points with x^2 + y^2 <= 49


def test_q_identities():
    """Eqs. qprop1 - qprop3 of Sec. 2.1."""
    R, R1, R2, beta = 0.7, 0.4, 1.3, 2.5
    r2a, r2b = np.array([1e-6, 4e-6, 9e-7]), np.array([2e-6, 5e-6, 1e-6])
    assert np.allclose(O.q(R, r2a / beta ** 2, LAM), O.q(beta ** 2 * R, r2a, LAM), rtol=1e-13)
    assert np.allclose(O.q(R, r2b, LAM) * np.conj(O.q(R, r2a, LAM)), O.q(R, r2b - r2a, LAM), rtol=1e-13)
    assert np.allclose(O.q(R1, r2a, LAM) * np.conj(O.q(R2, r2a, LAM)),
                       O.q(R1 * R2 / (R2 - R1), r2a, LAM), rtol=1e-12)
    assert np.allclose(O.q(R, r2a, LAM) * np.conj(O.q(R, r2a, LAM)), 1.0, rtol=1e-15)


# --------------------------------------------------------------------------- adjoint
@pytest.mark.parametrize("farfield", [False, True])
def test_adjoint_dot_product(farfield):
    """<P X, Y> = <X, P^H Y> for the propagation map P (FP64)."""
    N = 8
    rng = np.random.default_rng(17)
    X = rng.standard_normal((N,) * 4) + 1j * rng.standard_normal((N,) * 4)
    Y = rng.standard_normal((N,) * 4) + 1j * rng.standard_normal((N,) * 4)
    PX, _ = O.propagate_fft(X, DXI, LAM, 0.5, farfield)
    PhY = O.propagate_adjoint(Y, DXI, LAM, 0.5, farfield)
    lhs = np.vdot(PX, Y)
    rhs = np.vdot(X, PhY)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# --------------------------------------------------------------------------- paper numbers
def test_golden_paper_numbers():
    g = json.load(open(GOLDEN))["entries"]
    by = {e["id"]: e for e in g}
    e = by["ex3_lens_plane_sampling"]
    i = e["inputs"]
    lam = 2 * math.pi * i["c"] / i["omega0"]
    dx = O.output_sampling(i["N"], i["dxi"], lam, i["R"])
    assert abs(dx / e["printed"]["dx"] - 1) < e["rel_tol"]
    e = by["ex4_sampling_equals_source"]
    i = e["inputs"]
    lam = 2 * math.pi * i["c"] / i["omega0"]
    assert abs(lam / e["printed"]["lambda0"] - 1) < e["rel_tol"]
    dx = O.output_sampling(i["N"], i["dxi"], lam, i["R"])
    assert abs(dx / e["printed"]["dx"] - 1) < e["rel_tol"]
    e = by["ex1_dark_spot"]
    i, p = e["inputs"], e["printed"]
    lam = 2 * math.pi * i["c"] / i["omega0"]
    assert abs(lam / p["lambda0"] - 1) < e["rel_tol"]
    Na = round(math.sqrt(2 * math.pi * i["Nz"]))
    assert Na == p["Na"]
    assert abs(Na * i["dxi"] / p["a"] - 1) < e["rel_tol"]
    R = i["a"] ** 2 / (2 * math.pi * lam)
    assert abs(R / p["R1"] - 1) < e["rel_tol"]
    assert abs(i["a"] ** 2 / (lam * p["R1"]) / p["NF"] - 1) < e["rel_tol"]
    dx = O.output_sampling(i["Nz"], i["dxi"], lam, R)
    assert abs(dx / i["dxi"] - p["dx_over_dxi"]) < e["rel_tol_dx_over_dxi"]


def test_odd_n_rejected():
    with pytest.raises(ValueError):
        O.axis_coords(7, DXI)


# --------------------------------------------------------------------------- gradients
@pytest.mark.parametrize("farfield", [False, True])
def test_s_loss_gradient_matches_central_differences(farfield):
    """Adjoint gradient of the S loss vs central finite differences (FP64), for sigma_S, sigma_mu,
    the amplitude A and two mask pixels."""
    N, z, lam = 8, 0.6, 633e-9
    rng = np.random.default_rng(2)
    amask = 0.5 + 0.5 * rng.random((N, N))
    target = O.s_loss(1.2 * SS, 0.8 * SM, 1.1, 0.7 + 0.3 * rng.random((N, N)), N, DXI, lam, z,
                      np.zeros((N, N)), np.ones((N, N)), farfield)[1]
    weight = 1.0 + rng.random((N, N))
    L, gS, gM, gA, ga = O.s_loss_gradient(SS, SM, 1.0, amask, N, DXI, lam, z, target, weight, farfield)

    def f(sS=SS, sM=SM, A=1.0, am=amask):
        return O.s_loss(sS, sM, A, am, N, DXI, lam, z, target, weight, farfield)[0]
    h = 1e-6
    assert abs((f(sS=SS * (1 + h)) - f(sS=SS * (1 - h))) / (2 * h * SS) - gS) < 1e-6 * abs(gS)
    assert abs((f(sM=SM * (1 + h)) - f(sM=SM * (1 - h))) / (2 * h * SM) - gM) < 1e-6 * abs(gM)
    assert abs((f(A=1 + h) - f(A=1 - h)) / (2 * h) - gA) < 1e-6 * abs(gA)
    for (a, b) in [(3, 4), (0, 7)]:
        ap, am_ = amask.copy(), amask.copy()
        ap[a, b] += h
        am_[a, b] -= h
        fd = (f(am=ap) - f(am=am_)) / (2 * h)
        assert abs(fd - ga[a, b]) < 1e-6 * np.abs(ga).max()


def test_imaging_system_maps_source_onto_image():
    """Sec. 2.3 imaging system: source plane A, a thin lens f at plane B (R1 from A), image plane C
    (R2 from B) with the lens law 1/R1 + 1/R2 = 1/f (Eq. imaging).  At unit magnification
    (R1 = R2 = 2 f) the output sampling equals the source sampling and S_C = C' S_A with C' = 1
    under the power-conserving scale, on the inverted grid (the two transforms of each point
    compose to x -> -x; index i -> (N - i) mod N); exact for the discrete method, whatever the
    input chirp.  At magnification 2 the sampling doubles and the power is conserved."""
    N, d, lam, f = 32, 20e-6, 633e-9, 0.2
    m = WL.amplitude_mask(N, seed=5) * (np.arange(N)[:, None] < 20)  # asymmetric: shows an inversion
    W0 = O.apply_mask(O.gsm_source(N, d, 0.1e-3, 0.05e-3, 1.0), m)
    SA = np.real(O.spectral_density(W0))

    def image(R1, R2):
        WB, dB = O.propagate_fft(W0, d, lam, R1)
        return O.propagate_fft(O.apply_mask(WB, O.thin_lens(N, dB, lam, f)), dB, lam, R2)

    WC, dC = image(2 * f, 2 * f)
    assert abs(dC / d - 1) < 1e-14
    rev = (-np.arange(N)) % N
    SC = np.real(O.spectral_density(WC))
    assert np.linalg.norm(SC - SA[rev][:, rev]) <= 1e-12 * np.linalg.norm(SA)
    WC2, dC2 = image(1.5 * f, 3 * f)
    assert abs(dC2 / d - 2) < 1e-14
    assert abs(np.real(O.spectral_density(WC2)).sum() * dC2 ** 2 / (SA.sum() * d ** 2) - 1) < 1e-12


# ---------------------------------------------------------------- zero padding (Sec. 3.2)
def _lens_aperture_gsm(N, dxi=DXI):
    m = O.circle_aperture(N, dxi, 2.2 * dxi) * O.thin_lens(N, dxi, LAM, 0.3)
    return O.apply_mask(O.gsm_source(N, dxi, 0.1e-3, 0.05e-3), m)


@pytest.mark.parametrize("farfield", [False, True])
def test_padded_route_equals_direct_quadrature(farfield):
    # brute force at the padded output samples (dx = lambda z / (Nz dxi), central N of Nz)
    W0 = _lens_aperture_gsm(6)
    a, dxa = O.propagate_padded(W0, DXI, LAM, 0.5, 10, farfield)
    b, dxb = O.propagate_direct(W0, DXI, LAM, 0.5, farfield, Nz=10)
    assert dxa == dxb == pytest.approx(LAM * 0.5 / (10 * DXI), rel=1e-15)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12


def test_padded_route_without_padding_is_algorithm2():
    W0 = _lens_aperture_gsm(8)
    a, _ = O.propagate_padded(W0, DXI, LAM, 0.5, 8)
    b, _ = O.propagate_fft(W0, DXI, LAM, 0.5)
    assert np.array_equal(a, b)


def test_padded_rows_match_padded_route():
    rng = np.random.default_rng(3)
    N, Nz = 12, 20
    m = np.exp(2j * np.pi * rng.random((N, N)))
    W0 = O.apply_mask(O.gsm_source(N, DXI, 0.1e-3, 0.05e-3), m)
    a, _ = O.propagate_padded(W0, DXI, LAM, 0.5, Nz)
    rows = [(6, 6), (3, 9), (11, 0)]
    r = O.propagate_rows_gsm_padded(m, N, DXI, LAM, 0.5, 0.1e-3, 0.05e-3, 1.0, rows, Nz)
    for k, (i, j) in enumerate(rows):
        assert np.linalg.norm(r[k] - a[i, j]) / np.linalg.norm(a[i, j]) < 1e-12


@pytest.mark.parametrize("Nz,farfield", [(128, False), (160, True)])
def test_padded_gsm_matches_closed_form(Nz, farfield):
    # the continuous Gaussian integral on the finer output grid of the padded transform
    N = 64
    rows = [(32, 32), (20, 40)]
    r = O.propagate_rows_gsm_padded(np.ones((N, N)), N, DXI, LAM, 0.5, 0.1e-3, 0.05e-3, 1.0, rows, Nz,
                                    farfield=farfield)
    cf = O.gsm_closed_form(N, DXI, LAM, 0.5, 0.1e-3, 0.05e-3, 1.0, farfield=farfield, Nz=Nz)
    for k, (i, j) in enumerate(rows):
        assert np.linalg.norm(r[k] - cf[i, j]) / np.linalg.norm(cf[i, j]) < 1e-8


def test_padded_rejects_bad_sizes():
    W0 = _lens_aperture_gsm(6)
    for Nz in (4, 9):
        with pytest.raises(ValueError):
            O.propagate_padded(W0, DXI, LAM, 0.5, Nz)


def test_padded_rows_match_padded_route_far_field():
    rng = np.random.default_rng(4)
    N, Nz = 10, 26
    m = np.exp(2j * np.pi * rng.random((N, N)))
    W0 = O.apply_mask(O.gsm_source(N, DXI, 0.1e-3, 0.05e-3), m)
    a, _ = O.propagate_padded(W0, DXI, LAM, 2.0, Nz, farfield=True)
    rows = [(5, 5), (2, 8)]
    r = O.propagate_rows_gsm_padded(m, N, DXI, LAM, 2.0, 0.1e-3, 0.05e-3, 1.0, rows, Nz, farfield=True)
    for k, (i, j) in enumerate(rows):
        assert np.linalg.norm(r[k] - a[i, j]) / np.linalg.norm(a[i, j]) < 1e-12


# --------------------------------------------------------------------------- bilinear probes
def _probe_fields(N, K, seed):
    u = WL.uniform01(seed, 4 * K * N * N).reshape(4, K, N, N)
    return (u[0] - 0.5) + 1j * (u[1] - 0.5), (u[2] - 0.5) + 1j * (u[3] - 0.5)


@pytest.mark.parametrize("farfield", [False, True])
def test_bilinear_probes_match_fft_route(farfield):
    """u^H W_B v from W0 through the kernel sums (no FFT) == the same form of Algorithm 2's output,
    and of the brute-force quadrature; a random non-Hermitian W0 at N = 6, 8."""
    for N in (6, 8):
        rng = np.random.default_rng(N)
        W0 = rng.standard_normal((N,) * 4) + 1j * rng.standard_normal((N,) * 4)
        U, V = _probe_fields(N, 3, 40 + N)
        got = O.bilinear_probes(W0, DXI, LAM, 0.45, U, V, farfield)
        WB, _ = O.propagate_fft(W0, DXI, LAM, 0.45, farfield)
        Wd, _ = O.propagate_direct(W0, DXI, LAM, 0.45, farfield)
        M, Md = WB.reshape(N * N, N * N), Wd.reshape(N * N, N * N)
        want = np.array([np.conj(U[k].ravel()) @ M @ V[k].ravel() for k in range(3)])
        want_d = np.array([np.conj(U[k].ravel()) @ Md @ V[k].ravel() for k in range(3)])
        assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()
        assert np.abs(got - want_d).max() < 1e-11 * np.abs(want).max()
        # a probe is not symmetric in u and v: swapping them changes the value
        swapped = O.bilinear_probes(W0, DXI, LAM, 0.45, V, U, farfield)
        assert np.abs(swapped - got).max() > 1e-3 * np.abs(got).max()


@pytest.mark.parametrize("farfield", [False, True])
def test_bilinear_probes_gsm_match_general_form(farfield):
    """The separable masked-GSM form equals bilinear_probes on the materialised source (N = 12,
    random complex mask: a transposed g or a dropped conjugate of the mask fails this)."""
    N = 12
    m = _rand_mask(N, 11)
    W0 = O.apply_mask(O.gsm_source(N, DXI, SS, SM, 1.7), m)
    U, V = _probe_fields(N, 4, 90)
    a = O.bilinear_probes_gsm(m, N, DXI, LAM, 0.6, SS, SM, 1.7, U, V, farfield)
    b = O.bilinear_probes(W0, DXI, LAM, 0.6, U, V, farfield)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


# --------------------------------------------------------------------------- mu-loss adjoint
def _sm_problem(N, farfield):
    P1 = (N // 2 - 1, N // 2 + 1)
    amask = 0.5 + 0.5 * WL.uniform01(77, N * N).reshape(N, N)
    S_t = 0.7 * np.ones((N, N)) * 1e-3
    mu_t = 0.3 * np.exp(1j * np.linspace(0, 1, N * N)).reshape(N, N)
    wS = 1e6 * (0.5 + WL.uniform01(78, N * N).reshape(N, N))
    wmu = 0.5 + WL.uniform01(79, N * N).reshape(N, N)
    return P1, amask, S_t, wS, mu_t, wmu


@pytest.mark.parametrize("farfield", [False, True])
def test_sm_loss_gradient_matches_central_differences(farfield):
    """Adjoint gradient of a loss on S and mu (reading R22) against central finite differences of
    the forward loss in FP64: sigma_S, sigma_mu, A and two mask pixels (N = 8, z = 0.35 m)."""
    N, z = 8, 0.35
    P1, amask, S_t, wS, mu_t, wmu = _sm_problem(N, farfield)
    sS, sM, A = 0.09e-3, 0.06e-3, 1.3

    def L(sS_, sM_, A_, am_):
        W0 = O.apply_mask(O.gsm_source(N, DXI, sS_, sM_, A_), am_)
        return O.sm_loss(W0, DXI, LAM, z, P1, S_t, wS, mu_t, wmu, farfield)[0]
    L0, gS, gM, gA, ga, _ = O.sm_loss_gradient(sS, sM, A, amask, N, DXI, LAM, z, P1, S_t, wS, mu_t, wmu, farfield)
    assert L0 > 0

    def cd(f, x, h):
        return (f(x + h) - f(x - h)) / (2 * h)
    fS = cd(lambda v: L(v, sM, A, amask), sS, 1e-6 * sS)
    fM = cd(lambda v: L(sS, v, A, amask), sM, 1e-6 * sM)
    fA = cd(lambda v: L(sS, sM, v, amask), A, 1e-6 * A)
    for g, f in [(gS, fS), (gM, fM), (gA, fA)]:
        assert abs(g - f) <= 1e-6 * abs(f), (g, f)
    for (i, j) in [(3, 4), (P1[0], P1[1])]:
        def Lm(v, i=i, j=j):
            am = amask.copy()
            am[i, j] = v
            return L(sS, sM, A, am)
        f = cd(Lm, amask[i, j], 1e-6)
        assert abs(ga[i, j] - f) <= 1e-6 * max(abs(f), 1e-3 * np.abs(ga).max()), (i, j, ga[i, j], f)


def test_sm_loss_gradient_in_w0_matches_central_differences():
    """The real gradient with respect to a general complex W0 (not only Hermitian perturbations):
    central differences of the loss in Re and Im of single entries, one of them on the P1 row."""
    N, z = 6, 0.4
    P1, _, S_t, wS, mu_t, wmu = _sm_problem(N, False)
    # a GSM source plus a random Hermitian part: S stays well away from zero, so mu is smooth enough
    # for central differences with a step of 1e-6 max |W0|
    R = WL.random_csd(N, seed=12, n_modes=3)
    W0 = O.gsm_source(N, DXI, SS, SM) + 0.1 * R / np.abs(R).max()
    L0, WB, S, mu = O.sm_loss(W0, DXI, LAM, z, P1, S_t, wS, mu_t, wmu)
    Y = O.adjoint_source(WB, P1, 2.0 * wS * (S - S_t), 2.0 * wmu * (mu - mu_t))
    g = 2.0 * O.propagate_adjoint(Y, DXI, LAM, z)
    h = 1e-6 * np.abs(W0).max()
    for idx in [(1, 2, 3, 4), (P1[0], P1[1], 0, 5), (2, 2, 2, 2)]:
        for unit in (1.0, 1j):
            Wp, Wm = W0.copy(), W0.copy()
            Wp[idx] += unit * h
            Wm[idx] -= unit * h
            f = (O.sm_loss(Wp, DXI, LAM, z, P1, S_t, wS, mu_t, wmu)[0]
                 - O.sm_loss(Wm, DXI, LAM, z, P1, S_t, wS, mu_t, wmu)[0]) / (2 * h)
            got = g[idx].real if unit == 1.0 else g[idx].imag
            assert abs(got - f) <= 1e-6 * np.abs(g).max(), (idx, unit, got, f)


def test_adjoint_source_reduces_to_s_loss():
    """With no mu term the adjoint source is the diagonal (1/2) dL/dS of s_loss_gradient (R18)."""
    N = 6
    W0 = O.gsm_source(N, DXI, SS, SM)
    WB, _ = O.propagate_fft(W0, DXI, LAM, 0.5)
    gS = WL.uniform01(5, N * N).reshape(N, N)
    Y = O.adjoint_source(WB, (2, 3), gS, np.zeros((N, N)))
    i = np.arange(N)
    D = np.zeros_like(Y)
    D[i[:, None], i[None, :], i[:, None], i[None, :]] = 0.5 * gS
    assert np.abs(Y - D).max() == 0


@pytest.mark.parametrize("farfield", [False, True])
def test_diagonal_rows_match_general_rows(farfield):
    """propagate_rows_diagonal (the delta-correlated source's collapsed point-1 sum) against
    propagate_rows on the same source written out slice by slice, and against the FFT route."""
    N = 12
    d = 0.3 + WL.uniform01(5, N * N).reshape(N, N)
    w = 0.7
    rows = [(0, 0), (5, 7), (11, 3)]

    def slice_fn(i, j):
        s = np.zeros((N, N), dtype=np.complex128)
        s[i, j] = w * d[i, j]
        return s
    got = O.propagate_rows_diagonal(d, w, N, DXI, LAM, 0.4, rows, farfield=farfield)
    ref = O.propagate_rows(slice_fn, N, DXI, LAM, 0.4, rows, farfield=farfield)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    W0 = np.zeros((N,) * 4, dtype=np.complex128)
    for i in range(N):
        for j in range(N):
            W0[i, j, i, j] = w * d[i, j]
    full, _ = O.propagate_fft(W0, DXI, LAM, 0.4, farfield=farfield)
    for r, (a, b) in enumerate(rows):
        assert np.abs(got[r] - full[a, b]).max() <= 1e-12 * np.abs(full).max()
