"""Host-side checks of the run-control part of the C ABI (no GPU needed): checkpoint
headers are read and checked without a context, error codes have messages, and the
allocation-failure hook validates its argument without touching CUDA."""
import struct

import pytest

from paper_2012_05537_gb300 import build as B
from paper_2012_05537_gb300 import sllbm as S


@pytest.fixture(scope="module")
def lib():
    B.build()
    return S.load()


def header(storage=1, p=3, cells=(2, 3, 4), steps=17, payload=None, magic=b"SLLBMCK1", version=1):
    elem = {0: 8, 1: 4, 2: 2, 3: 2}[storage]
    nodes = cells[0] * cells[1] * cells[2] * p ** 3
    if payload is None:
        payload = 2 * 45 * nodes * elem
    h = magic + struct.pack("<I", version) + struct.pack("<7i", storage, p, 0, *cells, 1)
    h += struct.pack("<7d", 6.0, 6.1, 6.2, 0.05, 3e-4, 1.0, 1.0) + struct.pack("<qQ", steps, payload)
    h += bytes(16)
    assert len(h) == 128
    return h, 2 * 45 * nodes * elem


def test_error_codes_have_messages(lib):
    for code in (S.EABORTED, S.EIO):
        assert S.strerror(code) != "unknown error"


def test_checkpoint_info_reads_a_valid_header(lib, tmp_path):
    h, n = header()
    f = tmp_path / "ok.ckpt"
    f.write_bytes(h + bytes(n))
    c = S.sllbm_checkpoint_info(str(f))
    assert (c.storage, c.p, c.velset, tuple(c.cells), c.pr_correction) == (1, 3, 0, (2, 3, 4), 1)
    assert (tuple(c.L), c.dt, c.mu_inf, c.rho0, c.T0) == ((6.0, 6.1, 6.2), 0.05, 3e-4, 1.0, 1.0)
    assert c.steps == 17 and c.payload_bytes == n


@pytest.mark.parametrize("what", ["magic", "version", "payload_field", "truncated", "long", "order"])
def test_checkpoint_info_rejects_bad_files(lib, tmp_path, what):
    h, n = header()
    body = bytes(n)
    if what == "magic":
        h, n = header(magic=b"SLLBMCK0")
    elif what == "version":
        h, n = header(version=2)
    elif what == "payload_field":
        h, _ = header(payload=n + 2)
    elif what == "truncated":
        body = bytes(n - 1)
    elif what == "long":
        body = bytes(n + 8)
    elif what == "order":
        h, n = header(p=5)
        body = bytes(n)
    f = tmp_path / "bad.ckpt"
    f.write_bytes(h + body)
    with pytest.raises(S.SllbmError) as e:
        S.sllbm_checkpoint_info(str(f))
    assert e.value.code == S.EINVAL


def test_checkpoint_info_missing_file(lib, tmp_path):
    with pytest.raises(S.SllbmError) as e:
        S.sllbm_checkpoint_info(str(tmp_path / "none.ckpt"))
    assert e.value.code == S.EIO


def test_fail_allocs_hook_arguments(lib):
    with pytest.raises(S.SllbmError) as e:
        S.sllbm_debug_fail_allocs(-2)
    assert e.value.code == S.EINVAL
    S.sllbm_debug_fail_allocs(-1)  # disarmed; no CUDA call is made
    assert lib.sllbm_set_wait_limit(None, 1.0) == S.EINVAL
    assert lib.sllbm_request_abort(None, 1) == S.EINVAL
    assert lib.sllbm_save(None, b"x") == S.EINVAL and lib.sllbm_load(None, b"x") == S.EINVAL
    assert S.load().sllbm_fma_peak(3, 1, None, None, None) == S.EINVAL
