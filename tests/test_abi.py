"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/ctqr.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ctqr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(ct_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ct_build_system", "ct_qr_factor", "ct_apply_qt", "ct_trsm_solve",
                     "ct_reconstruct_batch", "ct_factor_destroy", "ct_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1907_01891_gb300 import ctqr
    lib = ctqr.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in ctqr.SIGNATURES, f"binding lacks {name}"
    assert set(ctqr.SIGNATURES) <= set(declared_functions())


def test_status_strings_and_version_without_gpu():
    from paper_1907_01891_gb300 import ctqr
    lib = ctqr.load()
    assert lib.ct_status_str(0) == b"CT_OK"
    assert lib.ct_status_str(4) == b"CT_ERR_RANK"
    assert b"sm_103a" in lib.ct_version()


def test_system_size_validation_without_gpu():
    from paper_1907_01891_gb300 import ctqr
    from paper_1907_01891_gb300 import inputs as I
    assert ctqr.system_size(I.CONFIG1["geom"]) == (2700, 1024)
    assert ctqr.system_size(I.CONFIG1["geom"], 1e-3) == (2700 + 1024, 1024)
    assert ctqr.system_size(I.CONFIG2["geom"]) == (23168, 16384)
    assert ctqr.system_size(I.CONFIG3["geom"]) == (69696, 65536)
    bad = I.ScanGeometry(1, 8, 8, 1.0, 4, 5, 0.0, 6.28, 2.0, 0.5)  # source inside the image
    with pytest.raises(ctqr.CtError) as e:
        ctqr.system_size(bad)
    assert e.value.status == ctqr.CT_ERR_INVALID


def test_null_arguments_rejected_without_gpu():
    from paper_1907_01891_gb300 import ctqr
    lib = ctqr.load()
    out = ctypes.c_void_p()
    assert lib.ct_qr_factor(None, 0, 10, 5, 10, 0, None, ctypes.byref(out), None) == ctqr.CT_ERR_INVALID
    assert lib.ct_apply_qt(None, None, 1, 1, None) == ctqr.CT_ERR_INVALID
    assert lib.ct_apply_qt_f32(None, None, 1, 1, None) == ctqr.CT_ERR_INVALID
    assert lib.ct_trsm_solve(None, None, 1, 1, None) == ctqr.CT_ERR_INVALID
    lib.ct_factor_destroy(None)


def test_factor_file_header_is_read_without_gpu(tmp_path):
    """The factor file's header format (ct_factor_save): magic, version,
    header size, m, n, nb, prec, storage type, block flag, tag, payload size,
    checksum; ct_factor_file_info reads it without touching a GPU and refuses
    a malformed one."""
    import struct
    from paper_1907_01891_gb300 import ctqr
    m, n, nb = 10, 4, 2
    payload = m * n * 8 + n * 8 + 2 * nb * nb * 8
    hdr = struct.pack("<8sII qq iiii QQQ", b"CTQRFAC1", 1, 128, m, n, nb, 0, 0, 0, 77, payload, 0)
    hdr += b"\0" * (128 - len(hdr))
    good = tmp_path / "good.ctqr"
    good.write_bytes(hdr + b"\0" * payload)
    assert ctqr.factor_file_info(str(good)) == dict(m=m, n=n, nb=nb, prec=ctqr.Prec.F64, tag=77)
    for name, blob in [("magic", b"CTQRFAC2" + hdr[8:]), ("short", hdr[:100]),
                       ("m_lt_n", hdr[:16] + struct.pack("<qq", 3, 4) + hdr[32:]),
                       ("store", hdr[:40] + struct.pack("<i", 1) + hdr[44:])]:
        p = tmp_path / f"{name}.ctqr"
        p.write_bytes(blob)
        with pytest.raises(ctqr.CtError) as e:
            ctqr.factor_file_info(str(p))
        assert e.value.status == ctqr.CT_ERR_INVALID, name
    out, tag = ctypes.c_void_p(), ctypes.c_uint64()
    lib = ctqr.load()
    assert lib.ct_factor_load(str(tmp_path / "missing.ctqr").encode(), ctypes.byref(out), ctypes.byref(tag),
                              None) == ctqr.CT_ERR_INVALID
    assert lib.ct_factor_load(str(tmp_path / "magic.ctqr").encode(), ctypes.byref(out), ctypes.byref(tag),
                              None) == ctqr.CT_ERR_INVALID
    assert not out.value


def test_geometry_hash_distinguishes_scans_without_gpu():
    from paper_1907_01891_gb300 import ctqr
    from paper_1907_01891_gb300 import inputs as I
    g = I.CONFIG2["geom"]
    h = ctqr.geometry_hash(g)
    assert h != 0 and h == ctqr.geometry_hash(g, 0.0) == ctqr.geometry_hash(g, -0.0)
    assert h != ctqr.geometry_hash(g, 1e-3)
    assert h != ctqr.geometry_hash(I.CONFIG3["geom"])
    assert h != ctqr.geometry_hash(I.fan_geometry(128, 128, 183))
