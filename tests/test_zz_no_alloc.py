"""The allocation-free propagation entry point against the handle path (GPU).

Some callers cannot allocate device memory: a framework that reserves all device memory in its
own pool and does not let libraries call the CUDA allocator, or a latency-critical loop that
cannot take the device synchronisation of cudaMalloc / cudaFree.  For them the library offers
pw_propagate_gsm_fresnel_noalloc, which keeps its scratch in a fixed array inside the library.
This test calls it through the C ABI twice in a row with different inputs (the array keeps the
previous call's contents, so the second call must not depend on them) and compares each output
with the handle path, within the parity tolerance.  It lives in its own file so that it is
collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DXI, LAM, SS, SM = 20e-6, 633e-9, 0.1e-3, 0.05e-3
TOL = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _handle_path(pw, torch, N, z, A, aperture, lens_f, mask):
    c = pw.CSD(N, DXI, LAM)
    c.source_gsm(SS, SM, A)
    if aperture > 0:
        c.source_aperture(aperture)
    if lens_f:
        c.source_lens(lens_f)
    if mask is not None:
        c.source_mask(mask)
    c.propagate_fresnel(z)
    S = c.spectral_density()
    torch.cuda.synchronize()
    W = c.W.cpu().numpy()
    S = S.cpu().numpy()
    c.close()
    return W, S


def test_noalloc_matches_handle_path_on_two_calls():
    import torch
    import paper_2203_02734_gb300 as pw
    import workloads as WL

    N = 32
    stream = torch.cuda.current_stream().cuda_stream
    phase = torch.from_numpy(WL.to_c64(WL.phase_screen(N, seed=WL.SEED, corr_px=2.0))).cuda()
    cases = [
        dict(z=0.3, A=1.7, aperture=0.25e-3, lens_f=0.25, mask=phase),
        dict(z=0.5, A=1.0, aperture=0.0, lens_f=0.0, mask=None),
    ]
    W_out = torch.empty((N,) * 4, dtype=torch.complex64, device="cuda")
    S_out = torch.empty((N, N), dtype=torch.float32, device="cuda")
    for k in cases:
        W_out.fill_(float("nan"))
        S_out.fill_(float("nan"))
        pw.pw_propagate_gsm_fresnel_noalloc(
            N, DXI, LAM, k["z"], SS, SM, k["A"], k["aperture"], k["lens_f"],
            0 if k["mask"] is None else k["mask"].data_ptr(), W_out.data_ptr(), W_out.numel() * 8,
            S_out.data_ptr(), stream)
        torch.cuda.synchronize()
        W_ref, S_ref = _handle_path(pw, torch, N, **k)
        assert _rel(W_out.cpu().numpy(), W_ref) < TOL
        assert _rel(S_out.cpu().numpy(), S_ref) < TOL


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    import paper_2203_02734_gb300 as pw

    W_out = torch.empty(8, dtype=torch.complex64, device="cuda")
    with pytest.raises(pw.PwError) as e:
        pw.pw_propagate_gsm_fresnel_noalloc(64, DXI, LAM, 0.5, SS, SM, 1.0, 0.0, 0.0, 0, W_out.data_ptr(),
                                            64 ** 4 * 8, W_out.data_ptr(), 0)
    assert "PW_EINVAL" in str(e.value) and "maximum N = 32" in str(e.value)


def test_noalloc_rejects_misaligned_pointers():
    # W is written by bulk copies (16-byte aligned addresses), S as floats, the mask as 8-byte
    # complex values: misaligned pointers return PW_EINVAL on the host, before any launch.
    import torch
    import paper_2203_02734_gb300 as pw

    N = 8
    W_out = torch.empty(N ** 4 + 2, dtype=torch.complex64, device="cuda")
    S_out = torch.empty(N * N + 1, dtype=torch.float32, device="cuda")
    mask = torch.ones(N * N + 1, dtype=torch.complex64, device="cuda")
    nb = N ** 4 * 8
    bad = [(W_out.data_ptr() + 8, S_out.data_ptr(), 0, "dev_W_out must be 16-byte aligned"),
           (W_out.data_ptr(), S_out.data_ptr() + 2, 0, "dev_S_out must be 4-byte aligned"),
           (W_out.data_ptr(), S_out.data_ptr(), mask.data_ptr() + 4, "dev_mask must be 8-byte aligned")]
    for w, s, m, msg in bad:
        with pytest.raises(pw.PwError) as e:
            pw.pw_propagate_gsm_fresnel_noalloc(N, DXI, LAM, 0.5, SS, SM, 1.0, 0.0, 0.0, m, w, nb, s, 0)
        assert "PW_EINVAL" in str(e.value) and msg in str(e.value)
