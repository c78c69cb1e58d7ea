"""FP64 oracle: source models, Fresnel / far-field propagation, S and mu.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain NumPy, complex128.

Notation follows the paper:
  * a 4D cross-spectral density array (CSDA) W[i1, j1, i2, j2] samples
    W(xi1, xi2) with xi = (xi, eta) = dxi * ((i, -j) - (N/2, -N/2))   (Sec. 3.1, Eqs. point, n12),
    i.e. xi(i) = (i - N/2) dxi and eta(j) = (N/2 - j) dxi;
  * the propagator is q(R, xi) = exp(i pi |xi|^2 / (lambda R))          (Eq. q_factor);
  * the output sampling is dx = lambda R / (N dxi)                      (Eq. spatial_resolution).

Readings of passages that are garbled, ambiguous or silent:
  R1  GSM source: W = A exp(-(|xi1|^2+|xi2|^2)/(4 sigma_S^2)) exp(-|xi1-xi2|^2/(2 sigma_mu^2))
      (Sec. 5.4; the printed exponents lost their minus signs).
  R2  Circular aperture: the product Y(xi1) Y(xi2) of the text (appendix), boundary
      inclusive |xi| <= a, decided in pixel units as integer r^2 <= (a/dxi)^2 in FP64.
  R3  DFT signs: conj kernel h* acts on point 1 (Eq. W_general) so point 1 gets
      exp(+2 pi i X1.xi1/(lambda z)) and point 2 exp(-2 pi i X2.xi2/(lambda z));
      Algorithm 2 applies the direct FFT to the point-2 slices and the inverse to point 1.
  R4  Scale: secondary source with paraxial obliquity, Lambda = 1/(i lambda), so
      C = Lambda1* Lambda2 / R^2 = 1/(lambda R)^2 (Eq. C), and the quadrature measure
      dxi^4: s = dxi^4 / (lambda z)^2.  Far field uses the same s.
  R5  N must be even (M = N/2 is an index, Sec. 3.1).
  R6  mu := 0 where S(P1) S(x) <= 0 (Algorithm coherence divides by zero there).
  R7  Centring: the DFTs act on centred indices, sum_n f[n] exp(s 2 pi i (k-N/2)(n-N/2)/N).
  R8  GSM closed form: Eq. Wbeam is garbled; the continuous Gaussian integral is restated.
"""
import numpy as np

__all__ = [
    "axis_coords", "output_sampling", "q", "gsm_source", "circle_aperture", "thin_lens",
    "apply_mask", "centred_dft2", "propagate_fft", "propagate_direct", "propagate_rows",
    "propagate_adjoint", "spectral_density", "degree_of_coherence", "gsm_closed_form",
    "gsm_separable_quadrature", "propagation_scale", "gsm_beam_parameters", "propagate_rows_blocks",
    "propagate_rows_gsm", "propagate_rows_diagonal", "s_loss", "s_loss_gradient", "propagate_padded",
    "padded_dft_matrix",
    "propagate_rows_gsm_padded", "axis_kernels", "bilinear_probes", "bilinear_probes_gsm",
    "sm_loss", "adjoint_source", "sm_loss_gradient",
]


def _check_even(N):
    if N < 2 or N % 2:
        raise ValueError("N must be even and >= 2 (M = N/2 is an array index, Sec. 3.1)")


def axis_coords(N, d):
    """Sample positions of the centred grid, Sec. 3.1 Eqs. point and n12.

    Returns (x, y) with x[i] = (i - N/2) d (first index) and y[j] = (N/2 - j) d
    (second index); the second axis is flipped because n = (i, -j)."""
    _check_even(N)
    n = np.arange(N, dtype=np.float64)
    return (n - N / 2) * d, (N / 2 - n) * d


def output_sampling(N, dxi, lam, z):
    """Eq. spatial_resolution with omega = 2 pi c / lambda:  dx = lambda z / (N dxi)."""
    return lam * z / (N * dxi)


def q(R, r2, lam):
    """Propagator of Eq. q_factor: q(R, xi) = exp(i pi |xi|^2 / (lambda R)); r2 = |xi|^2."""
    return np.exp(1j * np.pi * np.asarray(r2, dtype=np.float64) / (lam * R))


def propagation_scale(dxi, lam, z):
    """Reading R4: C dxi^4 with C = Lambda1* Lambda2 / z^2 (Eq. C) and Lambda = 1/(i lambda)."""
    Lam = 1.0 / (1j * lam)
    C = np.conj(Lam) * Lam / z ** 2
    return float(np.real(C)) * dxi ** 4


def _r2_grid(N, d):
    x, y = axis_coords(N, d)
    return x[:, None] ** 2 + y[None, :] ** 2


def gsm_source(N, dxi, sigma_S, sigma_mu, A=1.0):
    """Gaussian Schell-model CSDA, Sec. 5.4 (Eq. of W_rho4) with reading R1.

    W0[i1,j1,i2,j2] = A exp(-(|xi1|^2 + |xi2|^2) / (4 sigma_S^2)) exp(-|xi1 - xi2|^2 / (2 sigma_mu^2))."""
    x, y = axis_coords(N, dxi)
    X1 = x[:, None, None, None]
    Y1 = y[None, :, None, None]
    X2 = x[None, None, :, None]
    Y2 = y[None, None, None, :]
    e = -((X1 ** 2 + Y1 ** 2) + (X2 ** 2 + Y2 ** 2)) / (4.0 * sigma_S ** 2)
    e = e - ((X1 - X2) ** 2 + (Y1 - Y2) ** 2) / (2.0 * sigma_mu ** 2)
    return (A * np.exp(e)).astype(np.complex128)


def circle_aperture(N, dxi, radius):
    """Circular geometry Y_c of the appendix (Eq. circle), reading R2:
    Y = 1 where (i - N/2)^2 + (N/2 - j)^2 <= (a/dxi)^2, else 0."""
    _check_even(N)
    n = np.arange(N)
    r2 = (n[:, None] - N // 2) ** 2 + (N // 2 - n[None, :]) ** 2
    rp = radius / dxi
    return (r2.astype(np.float64) <= rp * rp).astype(np.float64)


def thin_lens(N, dxi, lam, f):
    """Thin-lens transmission T = P q*(f, xi) of Sec. 2.2 with pupil P = 1."""
    return np.conj(q(f, _r2_grid(N, dxi), lam))


def apply_mask(W0, m):
    """Mask applied as m*(xi1) W m(xi2)  (Sec. 2.2 T* W T; Sec. 5.3 Y* W Y)."""
    m = np.asarray(m, dtype=np.complex128)
    return np.conj(m)[:, :, None, None] * W0 * m[None, None, :, :]


def centred_dft2(A, axes, sign):
    """Unnormalised 2D DFT over `axes` on centred indices (reading R7):
    out[k] = sum_n A[n] exp(sign 2 pi i (k - N/2)(n - N/2) / N), per axis.
    NumPy's FFT (a library primitive) evaluates the sum; the shifts move the centre."""
    N = A.shape[axes[0]]
    B = np.fft.ifftshift(A, axes=axes)
    if sign < 0:
        B = np.fft.fft2(B, axes=axes)
    else:
        B = np.fft.ifft2(B, axes=axes) * (N * N)
    return np.fft.fftshift(B, axes=axes)


def propagate_fft(W0, dxi, lam, z, farfield=False):
    """Algorithm 2 (freespaceprop), steps in the paper's order, FP64.

    W1 = qfunction(W0)                  (Algorithm 3: W * q*(xi1) q(xi2)); skipped for far field
    W2 = N^2 direct 2D DFTs over the point-2 pair (i2, j2)
    W3 = transpose(W2, 2, 3, 0, 1)
    W4 = N^2 inverse-sign (unnormalised) 2D DFTs over axes 2, 3 (= point 1)
    W5 = transpose(W4, 2, 3, 0, 1)
    dx = lambda z / (N dxi)             (Eq. spatial_resolution)
    W6 = s q*(x1) q(x2) W5              (qfunction at the output grid, scale of reading R4)
    Returns (W6, dx)."""
    N = W0.shape[0]
    _check_even(N)
    W0 = np.asarray(W0, dtype=np.complex128)
    if not farfield:
        qin = q(z, _r2_grid(N, dxi), lam)
        W1 = np.conj(qin)[:, :, None, None] * W0 * qin[None, None, :, :]
    else:
        W1 = W0.copy()
    W2 = centred_dft2(W1, axes=(2, 3), sign=-1)
    del W1
    W3 = W2.transpose(2, 3, 0, 1)
    W4 = centred_dft2(W3, axes=(2, 3), sign=+1)
    del W2, W3
    W5 = W4.transpose(2, 3, 0, 1)
    dx = output_sampling(N, dxi, lam, z)
    qout = q(z, _r2_grid(N, dx), lam)
    W6 = propagation_scale(dxi, lam, z) * np.conj(qout)[:, :, None, None] * W5 * qout[None, None, :, :]
    return W6, dx


def _kernel_matrix(N, dxi, lam, z, farfield, Nz=None):
    """h(X, xi) on flattened 2D point lists (row: output point X, column: source point xi).

    Fresnel: h = exp(i pi |X - xi|^2 / (lambda z)), i.e. Eq. h_free with r expanded to
    second order and Lambda/r -> Lambda/R (Eq. approx_L); the constant exp(ikz) and
    |Lambda|/z are moved into the scale s (they cancel in h* W h up to |Lambda|^2/z^2).
    Far field: q(xi) -> 1, so h = q(X) exp(-2 pi i X.xi / (lambda z))   (Eq. W_farfield).
    Nz: the output grid is the central N x N of the grid of a transform of size Nz (zero padding,
    Sec. 3.2), spacing lambda z / (Nz dxi)."""
    x, y = axis_coords(N, dxi)
    dx = output_sampling(Nz or N, dxi, lam, z)
    X, Y = axis_coords(N, dx)
    sx = np.stack(np.meshgrid(x, y, indexing="ij"), -1).reshape(-1, 2)
    ox = np.stack(np.meshgrid(X, Y, indexing="ij"), -1).reshape(-1, 2)
    if farfield:
        dot = ox @ sx.T
        qX = q(z, (ox ** 2).sum(1), lam)
        return qX[:, None] * np.exp(-2j * np.pi * dot / (lam * z))
    d2 = ((ox[:, None, :] - sx[None, :, :]) ** 2).sum(-1)
    return np.exp(1j * np.pi * d2 / (lam * z))


def propagate_direct(W0, dxi, lam, z, farfield=False, Nz=None):
    """Brute-force quadrature of Eq. W_general on the grid, O(N^8) terms:

    W_B(X1, X2) = s * sum_{xi1, xi2} h*(X1, xi1) W0(xi1, xi2) h(X2, xi2),

    evaluated as conj(H) @ W0 @ H^T over flattened point indices (two matmuls).
    Independent of the chirp/DFT factorisation used by propagate_fft.  Small N only.
    Nz: output samples of a zero-padded transform of size Nz (see _kernel_matrix)."""
    N = W0.shape[0]
    H = _kernel_matrix(N, dxi, lam, z, farfield, Nz)
    Wf = np.asarray(W0, dtype=np.complex128).reshape(N * N, N * N)
    WB = propagation_scale(dxi, lam, z) * (np.conj(H) @ Wf @ H.T)
    return WB.reshape(N, N, N, N), output_sampling(Nz or N, dxi, lam, z)


def propagate_rows(source_slice, N, dxi, lam, z, rows, farfield=False):
    """Rows W_B(X1 = (i1', j1'), . ) of the propagated CSDA for large N, Eq. W_fresnel
    with the two integrals in the printed order:

      inner(X1, xi2) = sum_{xi1} q*(xi1) exp(+2 pi i X1.xi1/(lambda z)) W0(xi1, xi2)
      W_B(X1, X2)    = s q*(X1) q(X2) sum_{xi2} inner(X1, xi2) q(xi2) exp(-2 pi i X2.xi2/(lambda z))

    The point-1 sum uses the exponential directly; the point-2 sum is a centred DFT.
    `source_slice(i1, j1)` returns W0[i1, j1, :, :] (complex128, N x N); rows is a list
    of (i1', j1').  Returns an array (len(rows), N, N).  Cost O(N^4) per call."""
    x, y = axis_coords(N, dxi)
    dx = output_sampling(N, dxi, lam, z)
    X, Y = axis_coords(N, dx)
    rows = list(rows)
    inner = np.zeros((len(rows), N, N), dtype=np.complex128)
    r2 = _r2_grid(N, dxi)
    qin = np.ones((N, N), dtype=np.complex128) if farfield else q(z, r2, lam)
    # c[r, i1, j1] = q*(xi1) exp(+2 pi i X1.xi1 / (lambda z))
    c = np.empty((len(rows), N, N), dtype=np.complex128)
    for r, (a, b) in enumerate(rows):
        ph = (X[a] * x[:, None] + Y[b] * y[None, :]) / (lam * z)
        c[r] = np.conj(qin) * np.exp(2j * np.pi * ph)
    for i1 in range(N):
        for j1 in range(N):
            inner += c[:, i1, j1, None, None] * source_slice(i1, j1)[None]
    inner *= qin[None]
    out = centred_dft2(inner, axes=(1, 2), sign=-1)
    qout = q(z, _r2_grid(N, dx), lam)
    for r, (a, b) in enumerate(rows):
        out[r] *= propagation_scale(dxi, lam, z) * np.conj(qout[a, b]) * qout
    return out


def propagate_rows_diagonal(d, w, N, dxi, lam, z, rows, farfield=False):
    """Rows of the propagated CSDA of the delta-correlated source W0(xi1, xi2) = w d(xi1) when
    xi1 = xi2 and 0 otherwise (Sec. 2.3's incoherent limit on the grid): in the point-1 sum of
    propagate_rows only xi1 = xi2 survives, so
      inner(X1, xi2) = q*(xi2) exp(+2 pi i X1.xi2/(lambda z)) w d(xi2)
    and the point-2 sum is the same centred DFT.  d is N x N (real), rows a list of (i1', j1')."""
    x, y = axis_coords(N, dxi)
    dx = output_sampling(N, dxi, lam, z)
    X, Y = axis_coords(N, dx)
    rows = list(rows)
    qin = np.ones((N, N), dtype=np.complex128) if farfield else q(z, _r2_grid(N, dxi), lam)
    inner = np.empty((len(rows), N, N), dtype=np.complex128)
    for r, (a, b) in enumerate(rows):
        ph = (X[a] * x[:, None] + Y[b] * y[None, :]) / (lam * z)
        inner[r] = np.conj(qin) * np.exp(2j * np.pi * ph) * (w * np.asarray(d, dtype=np.float64)) * qin
    out = centred_dft2(inner, axes=(1, 2), sign=-1)
    qout = q(z, _r2_grid(N, dx), lam)
    for r, (a, b) in enumerate(rows):
        out[r] *= propagation_scale(dxi, lam, z) * np.conj(qout[a, b]) * qout
    return out


def propagate_rows_blocks(source_block, N, dxi, lam, z, rows, farfield=False):
    """Same rows as propagate_rows, with the point-1 sum taken one first index at a time:
    source_block(i1) returns W0[i1, :, :, :] (N x N x N), and for each i1 the sum over j1 is a
    matrix product of the (rows x N) exponential weights with that block.  For large N."""
    x, y = axis_coords(N, dxi)
    dx = output_sampling(N, dxi, lam, z)
    X, Y = axis_coords(N, dx)
    rows = list(rows)
    qin = np.ones((N, N), dtype=np.complex128) if farfield else q(z, _r2_grid(N, dxi), lam)
    c = np.empty((len(rows), N, N), dtype=np.complex128)
    for r, (a, b) in enumerate(rows):
        ph = (X[a] * x[:, None] + Y[b] * y[None, :]) / (lam * z)
        c[r] = np.conj(qin) * np.exp(2j * np.pi * ph)
    inner = np.zeros((len(rows), N * N), dtype=np.complex128)
    for i1 in range(N):
        inner += c[:, i1, :] @ source_block(i1).reshape(N, N * N)
    inner = inner.reshape(len(rows), N, N) * qin[None]
    out = centred_dft2(inner, axes=(1, 2), sign=-1)
    qout = q(z, _r2_grid(N, dx), lam)
    for r, (a, b) in enumerate(rows):
        out[r] *= propagation_scale(dxi, lam, z) * np.conj(qout[a, b]) * qout
    return out


def propagate_rows_gsm(m, N, dxi, lam, z, sigma_S, sigma_mu, A, rows, farfield=False):
    """Rows of the propagated CSDA of the masked GSM source W0 = A m*(xi1) g(i1,i2) g(j1,j2) m(xi2)
    (g the per-axis GSM factor of Sec. 5.4, reading R1), with the point-1 sum of Eq. W_fresnel
    written as sum_{i1} g(i1, i2) sum_{j1} w(i1, j1) m*(i1, j1) g(j1, j2), i.e. G^T (w o m*) G
    for the exponential weights w of each row (the GSM factor is separable).  O(N^3) per row."""
    x, y = axis_coords(N, dxi)
    dx = output_sampling(N, dxi, lam, z)
    X, Y = axis_coords(N, dx)
    m = np.asarray(m, dtype=np.complex128)
    g = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / (4 * sigma_S ** 2)
               - (x[:, None] - x[None, :]) ** 2 / (2 * sigma_mu ** 2))
    qin = np.ones((N, N), dtype=np.complex128) if farfield else q(z, _r2_grid(N, dxi), lam)
    qout = q(z, _r2_grid(N, dx), lam)
    out = np.empty((len(rows), N, N), dtype=np.complex128)
    for r, (a, b) in enumerate(rows):
        ph = (X[a] * x[:, None] + Y[b] * y[None, :]) / (lam * z)
        w = np.conj(qin) * np.exp(2j * np.pi * ph)
        inner = A * m * (g.T @ (w * np.conj(m)) @ g) * qin
        out[r] = centred_dft2(inner, axes=(0, 1), sign=-1)
        out[r] *= propagation_scale(dxi, lam, z) * np.conj(qout[a, b]) * qout
    return out


def axis_kernels(N, dxi, lam, z, farfield=False):
    """Per-axis factors of the kernel h(X, xi) of propagate_direct: h(X, xi) = Hx[i', i] Hy[j', j]
    for the output point X = (X(i'), Y(j')) and the source point xi = (x(i), y(j)).
    Fresnel: |X - xi|^2 splits into the two axes, Hx[i', i] = exp(i pi (X(i') - x(i))^2/(lambda z));
    far field: q(X) exp(-2 pi i X.xi/(lambda z)) splits likewise (Eq. W_farfield)."""
    x, y = axis_coords(N, dxi)
    X, Y = axis_coords(N, output_sampling(N, dxi, lam, z))
    lz = lam * z

    def one(out, src):
        if farfield:
            return q(z, out ** 2, lam)[:, None] * np.exp(-2j * np.pi * out[:, None] * src[None, :] / lz)
        return np.exp(1j * np.pi * (out[:, None] - src[None, :]) ** 2 / lz)
    return one(X, x), one(Y, y)


def _probe_vectors(U, V, N, dxi, lam, z, farfield):
    """alpha_k(xi) = sum_X h(X, xi) u_k(X) and beta_k likewise for v_k (the kernel applied to the
    probe fields, per axis: Hx^T u Hy)."""
    Hx, Hy = axis_kernels(N, dxi, lam, z, farfield)
    U = np.asarray(U, dtype=np.complex128).reshape(-1, N, N)
    V = np.asarray(V, dtype=np.complex128).reshape(-1, N, N)
    al = np.matmul(np.matmul(Hx.T, U), Hy)
    be = np.matmul(np.matmul(Hx.T, V), Hy)
    return al, be


def bilinear_probes(W0, dxi, lam, z, U, V, farfield=False):
    """Quadratic forms p_k = u_k^H W_B v_k = sum_{X1, X2} conj(u_k(X1)) W_B(X1, X2) v_k(X2) of the
    propagated CSDA, from the source CSDA W0 without forming W_B: with W_B = s h* W0 h^T
    (Eq. W_general on the grid, as in propagate_direct),
      p_k = s sum_{xi1, xi2} conj(alpha_k(xi1)) W0(xi1, xi2) beta_k(xi2),
      alpha_k(xi) = sum_X h(X, xi) u_k(X),  beta_k(xi) = sum_X h(X, xi) v_k(X).
    U, V: (K, N, N) probe fields on the output grid.  O(N^4) per probe: small N."""
    N = W0.shape[0]
    al, be = _probe_vectors(U, V, N, dxi, lam, z, farfield)
    Wf = np.asarray(W0, dtype=np.complex128).reshape(N * N, N * N)
    s = propagation_scale(dxi, lam, z)
    return np.array([s * (np.conj(al[k].ravel()) @ (Wf @ be[k].ravel())) for k in range(al.shape[0])])


def bilinear_probes_gsm(m, N, dxi, lam, z, sigma_S, sigma_mu, A, U, V, farfield=False):
    """bilinear_probes for the masked GSM source W0 = A m*(xi1) g(i1, i2) g(j1, j2) m(xi2) (Sec. 5.4,
    reading R1; g the per-axis GSM factor, the same matrix on both axes because y(j) = -x(j)):
    the source sum becomes sum_{i1, j1} conj(alpha m)(i1, j1) [g (m beta) g](i1, j1), O(N^3) per
    probe, for large N."""
    x, _ = axis_coords(N, dxi)
    g = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / (4 * sigma_S ** 2)
               - (x[:, None] - x[None, :]) ** 2 / (2 * sigma_mu ** 2))
    m = np.asarray(m, dtype=np.complex128)
    al, be = _probe_vectors(U, V, N, dxi, lam, z, farfield)
    s = propagation_scale(dxi, lam, z)
    return np.array([s * A * np.sum(np.conj(al[k] * m) * (g @ (m * be[k]) @ g)) for k in range(al.shape[0])])


def _check_padding(N, Nz):
    if Nz < N or (Nz - N) % 2:
        raise ValueError("the padded size Nz must be >= N with Nz - N even (the source sits at the centre)")


def propagate_padded(W0, dxi, lam, z, Nz, farfield=False):
    """Zero padding with cropped output (Sec. 3.2, the note after Eq. spatial_resolution): the
    FFT runs on a grid of size Nz > N, N_z takes the place of N in dx = lambda z / (Nz dxi), and
    the result is cropped back to N x N.  Written out: W0 is placed at the centre of an Nz^4
    array of zeros (source coordinates unchanged, xi(n) = (n - N/2) dxi), propagated by
    Algorithm 2 at size Nz (propagate_fft), and the central N^4 block is returned with dx.
    Small N only (the padded array has Nz^4 elements)."""
    N = W0.shape[0]
    _check_even(N)
    _check_padding(N, Nz)
    o = (Nz - N) // 2
    Wp = np.zeros((Nz,) * 4, dtype=np.complex128)
    Wp[o:o + N, o:o + N, o:o + N, o:o + N] = W0
    WB, dx = propagate_fft(Wp, dxi, lam, z, farfield)
    return WB[o:o + N, o:o + N, o:o + N, o:o + N].copy(), dx


def padded_dft_matrix(N, Nz, sign):
    """E[k, n] = exp(sign 2 pi i (k - N/2)(n - N/2) / Nz): the centred DFT of size Nz restricted
    to its central N inputs (the source; the rest are the padding zeros) and its central N
    outputs (the crop) -- the pruned transform of propagate_padded along one axis."""
    k = np.arange(N, dtype=np.float64) - N / 2
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / Nz)


def propagate_rows_gsm_padded(m, N, dxi, lam, z, sigma_S, sigma_mu, A, rows, Nz, farfield=False):
    """Rows W_B(X1 = (i1', j1'), .) of propagate_padded for the masked GSM source of
    propagate_rows_gsm, for large N: the point-1 sum as in propagate_rows_gsm (exponential
    weights at the padded output sampling), the point-2 sum as E inner E^T with the pruned matrix
    E = padded_dft_matrix(N, Nz, -1) instead of a size-N DFT.  O(N^3) per row."""
    _check_padding(N, Nz)
    x, y = axis_coords(N, dxi)
    dx = output_sampling(Nz, dxi, lam, z)
    X, Y = axis_coords(N, dx)
    m = np.asarray(m, dtype=np.complex128)
    g = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / (4 * sigma_S ** 2)
               - (x[:, None] - x[None, :]) ** 2 / (2 * sigma_mu ** 2))
    qin = np.ones((N, N), dtype=np.complex128) if farfield else q(z, _r2_grid(N, dxi), lam)
    qout = q(z, _r2_grid(N, dx), lam)
    E = padded_dft_matrix(N, Nz, -1)
    out = np.empty((len(rows), N, N), dtype=np.complex128)
    for r, (a, b) in enumerate(rows):
        ph = (X[a] * x[:, None] + Y[b] * y[None, :]) / (lam * z)
        w = np.conj(qin) * np.exp(2j * np.pi * ph)
        inner = A * m * (g.T @ (w * np.conj(m)) @ g) * qin
        out[r] = E @ inner @ E.T
        out[r] *= propagation_scale(dxi, lam, z) * np.conj(qout[a, b]) * qout
    return out


def propagate_adjoint(Y, dxi, lam, z, farfield=False):
    """Adjoint P^H of the linear map P: W0 -> W_B of propagate_fft (Hilbert-Schmidt inner
    product <A, B> = sum conj(A) B).  P = s * D_out . F . D_in with diagonal chirp factors
    D_in = q*(xi1) q(xi2), D_out = q*(X1) q(X2) and F = (+ sign DFT over point 1) x
    (- sign DFT over point 2); hence P^H = s * conj(D_in) . F^H . conj(D_out), where F^H
    flips both DFT signs (the centred DFT matrices are symmetric)."""
    N = Y.shape[0]
    Y = np.asarray(Y, dtype=np.complex128)
    dx = output_sampling(N, dxi, lam, z)
    qout = q(z, _r2_grid(N, dx), lam)
    Y1 = qout[:, :, None, None] * Y * np.conj(qout)[None, None, :, :]
    Y2 = centred_dft2(Y1, axes=(0, 1), sign=-1)
    Y3 = centred_dft2(Y2, axes=(2, 3), sign=+1)
    if not farfield:
        qin = q(z, _r2_grid(N, dxi), lam)
        Y3 = qin[:, :, None, None] * Y3 * np.conj(qin)[None, None, :, :]
    return propagation_scale(dxi, lam, z) * Y3


def spectral_density(W):
    """Algorithm 4 (specdensity): S[i, j] = W[i, j, i, j] (complex; Re is S, Im a
    Hermiticity residual)."""
    N = W.shape[0]
    i = np.arange(N)
    return W[i[:, None], i[None, :], i[:, None], i[None, :]]


def degree_of_coherence(W, iP, jP):
    """Algorithm coherence with Eq. defMu: c[i, j] = W[iP, jP, i, j] / sqrt(S[i,j] S[iP,jP]),
    S = Re W[i,j,i,j]; reading R6: c := 0 where S(P1) S(x) <= 0."""
    S = np.real(spectral_density(W))
    den = S * S[iP, jP]
    out = np.zeros(S.shape, dtype=np.complex128)
    ok = den > 0
    out[ok] = W[iP, jP][ok] / np.sqrt(den[ok])
    return out


def _gsm_axis_gaussian(sigma_S, sigma_mu):
    a = 1.0 / (2.0 * sigma_S ** 2) + 1.0 / sigma_mu ** 2
    g = 1.0 / sigma_mu ** 2
    return a, g


def gsm_closed_form(N, dxi, lam, z, sigma_S, sigma_mu, A=1.0, farfield=False, Nz=None):
    """Continuous-integral GSM propagation on the output grid.  The printed Eq. Wbeam of
    Sec. 5.4 is garbled (alpha undefined), so the same integral is restated (reading R8).

    Per axis, with u = (xi1, xi2):  int exp(-u^T M u / 2 + i J^T u) d^2u = 2 pi / sqrt(det M)
    exp(-J^T M^-1 J / 2), M = [[a, -g], [-g, a]] + diag(2 pi i/(lambda z), -2 pi i/(lambda z))
    (no diagonal term for far field), a = 1/(2 sigma_S^2) + 1/sigma_mu^2, g = 1/sigma_mu^2,
    J = (2 pi X1/(lambda z), -2 pi X2/(lambda z)).  Each axis carries 1/(lambda z) and the
    output propagators q*(X1) q(X2); the 4D result is A * Wx[i1', i2'] * Wy[j1', j2'].
    Nz: evaluated on the central N x N samples of the output grid of a transform of size Nz."""
    dx = output_sampling(Nz or N, dxi, lam, z)
    X, Yc = axis_coords(N, dx)
    a, g = _gsm_axis_gaussian(sigma_S, sigma_mu)
    beta = 0.0 if farfield else 2.0 * np.pi / (lam * z)
    M = np.array([[a + 1j * beta, -g], [-g, a - 1j * beta]], dtype=np.complex128)
    detM = M[0, 0] * M[1, 1] - M[0, 1] * M[1, 0]
    Minv = np.array([[M[1, 1], -M[0, 1]], [-M[1, 0], M[0, 0]]]) / detM

    def axis(P):
        J1 = 2 * np.pi * P[:, None] / (lam * z)
        J2 = -2 * np.pi * P[None, :] / (lam * z)
        quad = Minv[0, 0] * J1 * J1 + 2 * Minv[0, 1] * J1 * J2 + Minv[1, 1] * J2 * J2
        val = (2 * np.pi / np.sqrt(detM)) * np.exp(-0.5 * quad) / (lam * z)
        qP = q(z, P ** 2, lam)
        return np.conj(qP)[:, None] * val * qP[None, :]

    Wx = axis(X)
    Wy = axis(Yc)
    return A * Wx[:, None, :, None] * Wy[None, :, None, :]


def gsm_separable_quadrature(N, dxi, lam, z, sigma_S, sigma_mu, A=1.0, farfield=False,
                             lens_f=None):
    """Discrete per-axis quadrature of Eq. W_general for the (separable) GSM source, optionally
    behind a thin lens T = q*(f) (also separable): per axis an N x N matrix
      Wx = (dxi^2/(lambda z)) conj(H) g H^T, H[X, xi] = exp(i pi (X - xi)^2/(lambda z)),
      g[xi1, xi2] = exp(-(xi1^2 + xi2^2)/(4 sigma_S^2) - (xi1 - xi2)^2/(2 sigma_mu^2)),
    and the 4D array A Wx[i1', i2'] Wy[j1', j2'].  Exact on the grid for any N (no FFT)."""
    x, y = axis_coords(N, dxi)
    dx = output_sampling(N, dxi, lam, z)
    X, Yc = axis_coords(N, dx)

    def axis(src, out):
        g = np.exp(-(src[:, None] ** 2 + src[None, :] ** 2) / (4 * sigma_S ** 2)
                   - (src[:, None] - src[None, :]) ** 2 / (2 * sigma_mu ** 2)).astype(np.complex128)
        if lens_f is not None:
            t = np.conj(q(lens_f, src ** 2, lam))
            g = np.conj(t)[:, None] * g * t[None, :]
        if farfield:
            H = q(z, out ** 2, lam)[:, None] * np.exp(-2j * np.pi * out[:, None] * src[None, :] / (lam * z))
        else:
            H = np.exp(1j * np.pi * (out[:, None] - src[None, :]) ** 2 / (lam * z))
        return (dxi ** 2 / (lam * z)) * (np.conj(H) @ g @ H.T)

    Wx = axis(x, X)
    Wy = axis(y, Yc)
    return A * Wx[:, None, :, None] * Wy[None, :, None, :]


def gsm_beam_parameters(lam, z, sigma_S, sigma_mu):
    """Textbook GSM beam: expansion factor Delta(z) = [1 + (z/(k sigma_S delta))^2]^(1/2),
    1/delta^2 = 1/(4 sigma_S^2) + 1/sigma_mu^2, radius of curvature R(z) = z [1 + (k sigma_S
    delta / z)^2] (textbook GSM beam formulas of Mandel & Wolf ch. 5, which Sec. 5.4 cites
    for Eq. Wbeam).  Independent of gsm_closed_form; used to pin it."""
    k = 2 * np.pi / lam
    delta = (1.0 / (4 * sigma_S ** 2) + 1.0 / sigma_mu ** 2) ** -0.5
    Delta = np.sqrt(1 + (z / (k * sigma_S * delta)) ** 2)
    Rz = z * (1 + (k * sigma_S * delta / z) ** 2)
    return Delta, Rz


def s_loss(sigma_S, sigma_mu, A, amask, N, dxi, lam, z, S_target, weight, farfield=False):
    """Least-squares loss on the propagated spectral density of the amplitude-masked GSM source
    W0 = A a(xi1) a(xi2) G(xi1, xi2):  L = sum_x weight(x) (S_B(x) - S_target(x))^2."""
    W0 = apply_mask(gsm_source(N, dxi, sigma_S, sigma_mu, A), amask)
    WB, _ = propagate_fft(W0, dxi, lam, z, farfield)
    S = np.real(spectral_density(WB))
    return float(np.sum(weight * (S - S_target) ** 2)), S


def s_loss_gradient(sigma_S, sigma_mu, A, amask, N, dxi, lam, z, S_target, weight, farfield=False):
    """Gradient of s_loss by the adjoint: dL/dS = 2 weight (S - S_target); since S = Re W_B(x, x),
    dL/dW_B* is the diagonal array (1/2) dL/dS; W0bar = P^H of it (propagate_adjoint); for each
    real parameter theta, dL/dtheta = 2 Re sum conj(W0bar) dW0/dtheta with
      dW0/dA = W0 / A,  dW0/dsigma_S = W0 (|xi1|^2 + |xi2|^2) / (2 sigma_S^3),
      dW0/dsigma_mu = W0 |xi1 - xi2|^2 / sigma_mu^3,
      dW0/da(eta) = A G (delta(xi1 = eta) a(xi2) + a(xi1) delta(xi2 = eta)).
    Returns (L, dL/dsigma_S, dL/dsigma_mu, dL/dA, dL/da (N x N))."""
    amask = np.asarray(amask, dtype=np.float64)
    L, S = s_loss(sigma_S, sigma_mu, A, amask, N, dxi, lam, z, S_target, weight, farfield)
    dLdS = 2.0 * weight * (S - S_target)
    Ybar = np.zeros((N, N, N, N), dtype=np.complex128)
    i = np.arange(N)
    Ybar[i[:, None], i[None, :], i[:, None], i[None, :]] = 0.5 * dLdS
    W0bar = propagate_adjoint(Ybar, dxi, lam, z, farfield)
    G = gsm_source(N, dxi, sigma_S, sigma_mu, 1.0).real
    W0 = A * amask[:, :, None, None] * amask[None, None, :, :] * G
    x, y = axis_coords(N, dxi)
    r2 = x[:, None] ** 2 + y[None, :] ** 2
    R1 = r2[:, :, None, None]
    R2 = r2[None, None, :, :]
    D2 = (x[:, None, None, None] - x[None, None, :, None]) ** 2 + (y[None, :, None, None] - y[None, None, None, :]) ** 2
    cW = np.conj(W0bar)
    gA = 2.0 * np.real(np.sum(cW * W0 / A))
    gS = 2.0 * np.real(np.sum(cW * W0 * (R1 + R2) / (2.0 * sigma_S ** 3)))
    gM = 2.0 * np.real(np.sum(cW * W0 * D2 / sigma_mu ** 3))
    AG = A * G
    ga = 2.0 * np.real(np.einsum("abcd,abcd,cd->ab", cW, AG, amask) + np.einsum("abcd,abcd,ab->cd", cW, AG, amask))
    return L, gS, gM, gA, ga


def sm_loss(W0, dxi, lam, z, P1, S_target, wS, mu_target, wmu, farfield=False):
    """Least-squares loss on S and mu of the propagated CSDA (Algorithm 4, Algorithm coherence):
      L = sum_x wS(x) (S_B(x) - S_target(x))^2 + sum_x wmu(x) |mu_B(P1, x) - mu_target(x)|^2.
    Returns (L, W_B, S_B, mu_B)."""
    WB, _ = propagate_fft(W0, dxi, lam, z, farfield)
    S = np.real(spectral_density(WB))
    mu = degree_of_coherence(WB, *P1)
    L = float(np.sum(wS * (S - S_target) ** 2) + np.sum(wmu * np.abs(mu - mu_target) ** 2))
    return L, WB, S, mu


def adjoint_source(WB, P1, gS, gmu):
    """dL/dW_B* of a loss L(S_B, mu_B) given the real gradients gS = dL/dS_B (N x N) and
    gmu = dL/dRe mu + i dL/dIm mu (N x N) of mu_B(P1, .) (reading R22).  With S(x) = Re W_B(x, x),
    w(x) = W_B(P1, x), D(x) = sqrt(S(P1) S(x)) and mu = w / D (0 where D = 0, held constant there):
      dmu = dw / D - (mu / 2) (dS(P1) / S(P1) + dS(x) / S(x)),
    so with r(x) = Re(conj(gmu(x)) mu(x)) the loss sees
      dL/dS(y) = gS(y) - r(y) / (2 S(y)) - [y = P1] sum_x r(x) / (2 S(P1)),
      dL/dw(x) (real gradient) = gmu(x) / D(x),
    and dL/dW_B* is half the real gradient: (1/2) dL/dS(y) on the diagonal (y, y) plus
    (1/2) gmu(x) / D(x) on the row (P1, x).  Returns that N^4 array (not Hermitian)."""
    N = WB.shape[0]
    S = np.real(spectral_density(WB))
    iP, jP = P1
    D = np.sqrt(np.maximum(S * S[iP, jP], 0.0))
    ok = D > 0
    mu = np.zeros((N, N), dtype=np.complex128)
    mu[ok] = WB[iP, jP][ok] / D[ok]
    gmu = np.where(ok, gmu, 0.0)
    r = np.real(np.conj(gmu) * mu)
    dS = np.array(gS, dtype=np.float64)
    okS = ok & (S > 0)
    dS[okS] -= r[okS] / (2.0 * S[okS])
    if S[iP, jP] > 0:
        dS[iP, jP] -= np.sum(r) / (2.0 * S[iP, jP])
    Y = np.zeros((N, N, N, N), dtype=np.complex128)
    i = np.arange(N)
    Y[i[:, None], i[None, :], i[:, None], i[None, :]] = 0.5 * dS
    gw = np.zeros((N, N), dtype=np.complex128)
    gw[ok] = gmu[ok] / D[ok]
    Y[iP, jP] += 0.5 * gw
    return Y


def sm_loss_gradient(sigma_S, sigma_mu, A, amask, N, dxi, lam, z, P1, S_target, wS, mu_target, wmu,
                     farfield=False):
    """Gradient of sm_loss for the amplitude-masked GSM source W0 = A a(xi1) a(xi2) G by the adjoint
    (readings R16-R18, R22): Y = adjoint_source, W0bar = P^H(Y) (propagate_adjoint), and for each
    real parameter theta, dL/dtheta = 2 Re sum conj(W0bar) dW0/dtheta with the derivatives listed
    in s_loss_gradient.  Also returns the real gradient with respect to W0 itself (a general complex
    N^4 array), 2 W0bar.  Returns (L, dL/dsigma_S, dL/dsigma_mu, dL/dA, dL/da, dL/dW0)."""
    amask = np.asarray(amask, dtype=np.float64)
    W0 = apply_mask(gsm_source(N, dxi, sigma_S, sigma_mu, A), amask)
    L, WB, S, mu = sm_loss(W0, dxi, lam, z, P1, S_target, wS, mu_target, wmu, farfield)
    gS = 2.0 * wS * (S - S_target)
    gmu = 2.0 * wmu * (mu - mu_target)
    Y = adjoint_source(WB, P1, gS, gmu)
    W0bar = propagate_adjoint(Y, dxi, lam, z, farfield)
    G = gsm_source(N, dxi, sigma_S, sigma_mu, 1.0).real
    x, y = axis_coords(N, dxi)
    r2 = x[:, None] ** 2 + y[None, :] ** 2
    R1 = r2[:, :, None, None]
    R2 = r2[None, None, :, :]
    D2 = (x[:, None, None, None] - x[None, None, :, None]) ** 2 + (y[None, :, None, None] - y[None, None, None, :]) ** 2
    cW = np.conj(W0bar)
    W0r = np.real(W0)
    gA = 2.0 * np.real(np.sum(cW * W0r / A))
    gS_ = 2.0 * np.real(np.sum(cW * W0r * (R1 + R2) / (2.0 * sigma_S ** 3)))
    gM = 2.0 * np.real(np.sum(cW * W0r * D2 / sigma_mu ** 3))
    AG = A * G
    ga = 2.0 * np.real(np.einsum("abcd,abcd,cd->ab", cW, AG, amask) + np.einsum("abcd,abcd,ab->cd", cW, AG, amask))
    return L, gS_, gM, gA, ga, 2.0 * W0bar
