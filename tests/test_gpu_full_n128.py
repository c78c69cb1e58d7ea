"""The N = 128 workload of GSM x 0.8 mm aperture x thin lens (Sec. 5.4, Eq. circle, Sec. 2.2) over
the whole output array: W, S and mu of the CUDA path against the FP64 oracle's full Algorithm 2
route (complex128 on the host), element by element, for Fresnel propagation behind the lens at
z = f = 0.3 m (Eq. W_fresnel) and far-field propagation of the aperture alone at z = 0.3 m
(Eq. W_farfield).  The two must also agree with each other (Eq. qprop3: the lens cancels the
input propagator at z = f).

Bar: relative L2 error <= 1e-5 for W (all 128^4 elements), S (all 128^2 points) and mu
(where S >= 1e-4 max S), and the stated bound in the region S >= 1e-6 max S."""
import numpy as np
import pytest

import workloads as WL
from gpu_cases import check_s_mu, gpu_run, oracle_run, record, rel

pytestmark = pytest.mark.gpu

TOL = 1e-5
CASES = [(WL.GSM_APERTURE_LENS_N128, "fresnel"), (WL.GSM_APERTURE_FARFIELD_N128, "farfield")]


@pytest.mark.parametrize("cfg,kind", CASES, ids=["fresnel_lens", "farfield"])
def test_full_array_n128(cfg, kind):
    N = cfg["N"]
    src = dict(gsm=(cfg["sigma_S"], cfg["sigma_mu"], cfg["A"]), aperture=cfg["aperture"], lens_f=cfg["lens_f"])
    steps = [(kind, cfg["z"])]
    out = gpu_run(N, cfg["dxi"], cfg["lam"], steps, P1=cfg["P1"], **src)
    ref, dx = oracle_run(N, cfg["dxi"], cfg["lam"], steps, **src)
    assert abs(out["dx"] - dx) <= 1e-15 * dx
    eW = rel(out["W"], ref)
    assert eW < TOL, "W rel-L2 %.3e" % eW
    check_s_mu(out, ref, cfg["P1"], tol=TOL, name="full_n128_" + kind)
    # the output is Hermitian to FP32 rounding over the whole array
    M = out["W"].reshape(N * N, N * N)
    eH = np.linalg.norm(M - M.conj().T) / np.linalg.norm(M)
    record("full_n128_" + kind + "_hermiticity", H=eH)
    assert eH < 1e-6


def test_lens_identity_full_array_n128():
    """Fresnel behind the f = 0.3 m lens at z = f equals the far field of the aperture alone
    (Eq. qprop3), over the whole array, up to FP32 rounding."""
    cfg = WL.GSM_APERTURE_LENS_N128
    N = cfg["N"]
    gsm = (cfg["sigma_S"], cfg["sigma_mu"], cfg["A"])
    a = gpu_run(N, cfg["dxi"], cfg["lam"], [("fresnel", cfg["z"])], gsm=gsm, aperture=cfg["aperture"],
                lens_f=cfg["lens_f"])
    b = gpu_run(N, cfg["dxi"], cfg["lam"], [("farfield", cfg["z"])], gsm=gsm, aperture=cfg["aperture"])
    e = rel(a["W"], b["W"])
    record("full_n128_lens_identity", W=e)
    assert e < 1e-6
