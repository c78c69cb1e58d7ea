"""C-ABI library on the CPU: it builds, loads, exports every symbol the header declares, and
rejects invalid arguments on the host before any device work (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pywolf_gb.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pw_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g._load_build_module().build()
    from paper_2203_02734_gb300 import abi
    return abi


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["pw_csd_create", "pw_csd_destroy", "pw_source_gsm", "pw_source_array", "pw_source_mask",
              "pw_propagate_fresnel", "pw_propagate_farfield", "pw_spectral_density",
              "pw_degree_of_coherence", "pw_get_sampling", "pw_last_error"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    for n in names:
        assert hasattr(lib.LIB, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pw_\w+)", out))
    assert set(names) <= exported
    assert set(names) == set(lib.SIGNATURES)


def test_sizes_and_plans(lib):
    assert lib.pw_csda_bytes(128) == 128 ** 4 * 8
    assert lib.pw_csda_bytes(256) == 256 ** 4 * 8
    for N in (2, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128):
        assert lib.pw_supported_n(N)
    for N in (0, 1, 3, 7, 10, 200, 1024):
        assert not lib.pw_supported_n(N)
    assert lib.LIB.pw_status_string(lib.PW_ETIMEOUT).decode() == "PW_ETIMEOUT"


FAKE_W, FAKE_WORK = 0x100000000, 0x900000000  # never dereferenced: validation comes first


@pytest.mark.parametrize("args,status,msg", [
    ((7, 20e-6, 633e-9), "PW_EINVAL", "even"),
    ((0, 20e-6, 633e-9), "PW_EINVAL", "even"),
    ((32, float("nan"), 633e-9), "PW_EINVAL", "sampling"),
    ((32, 20e-6, -1.0), "PW_EINVAL", "wavelength"),
    ((32, 20e-6, float("inf")), "PW_EINVAL", "wavelength"),
    ((514, 20e-6, 633e-9), "PW_EUNSUPPORTED", "N = 514"),
])
def test_create_rejects_bad_arguments(lib, args, status, msg):
    N = args[0]
    nb = max(lib.pw_csda_bytes(max(N, 2)), 8)
    with pytest.raises(lib.PwError) as e:
        lib.pw_csd_create(*args, FAKE_W, nb, FAKE_WORK, nb)
    assert status in str(e.value) and msg in str(e.value)


def test_create_rejects_small_and_overlapping_buffers(lib):
    nb = lib.pw_csda_bytes(32)
    with pytest.raises(lib.PwError, match="PW_ESIZE"):
        lib.pw_csd_create(32, 20e-6, 633e-9, FAKE_W, nb - 8, FAKE_WORK, nb)
    with pytest.raises(lib.PwError, match="PW_ESIZE"):
        lib.pw_csd_create(32, 20e-6, 633e-9, FAKE_W, nb, FAKE_WORK, 1)
    with pytest.raises(lib.PwError, match="overlap"):
        lib.pw_csd_create(32, 20e-6, 633e-9, FAKE_W, nb, FAKE_W + 8, nb)
    with pytest.raises(lib.PwError, match="non-null"):
        lib.pw_csd_create(32, 20e-6, 633e-9, 0, nb, FAKE_WORK, nb)
    # the CSDA buffers are moved by 16-byte bulk and tensor copies
    with pytest.raises(lib.PwError, match="16-byte aligned"):
        lib.pw_csd_create(32, 20e-6, 633e-9, FAKE_W + 8, nb, FAKE_WORK, nb)
    with pytest.raises(lib.PwError, match="16-byte aligned"):
        lib.pw_csd_create(32, 20e-6, 633e-9, FAKE_W, nb, FAKE_WORK + 4, nb)


def test_null_handle_is_rejected(lib):
    for f, args in [(lib.pw_source_gsm, (1e-4, 5e-5, 1.0)), (lib.pw_propagate_fresnel, (0.5,)),
                    (lib.pw_propagate_farfield, (0.5,)), (lib.pw_source_lens, (0.3,)),
                    (lib.pw_source_aperture, (1e-3,)), (lib.pw_get_sampling, ())]:
        with pytest.raises(lib.PwError, match="PW_EINVAL"):
            f(None, *args)
    lib.pw_csd_destroy(None)  # accepted


def test_no_device_reports_cuda_error(lib):
    """Valid arguments on a machine without a GPU: the first CUDA call fails and the status
    says so (host-side failure path; nothing is enqueued)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    nb = lib.pw_csda_bytes(32)
    with pytest.raises(lib.PwError, match="PW_ECUDA"):
        lib.pw_csd_create(32, 20e-6, 633e-9, FAKE_W, nb, FAKE_WORK, nb)
    assert "cudaMalloc" in lib.pw_last_error()
