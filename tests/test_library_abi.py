"""The C ABI library builds, loads and exports every symbol include/*.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(inc, fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(hif_[a-z_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1607_00346_gb300 import build
    path = build.build_library()
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "hif_factor" in names and "hif_apply" in names and "hif_solve" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_lists_every_symbol():
    from paper_1607_00346_gb300 import hif
    assert sorted(hif.EXPORTS) == sorted(n for n in _declared())


def test_host_only_entry_points(lib):
    from paper_1607_00346_gb300 import hif
    hif.load()
    o = hif.default_options()
    assert o.eps == 1e-6 and o.pcg_tol == 1e-10 and o.max_iter == 200
    assert o.tensor_cores == 1 and o.use_graphs == 1 and o.precision == hif.PREC_FP64
    assert hif.predict_bytes(64, 4) > 0
    assert hif.predict_bytes(60, 4) == 0        # 60 is not 4 * 2^L
    assert hif.load().hif_version().startswith(b"hif-gb300")


def test_predicted_footprint_follows_eps_and_precision(lib):
    # a larger eps keeps fewer skeletons, so the predicted peak shrinks; it
    # stays above the operator (32 B per DOF) and above the peaks measured on
    # the GPU for the same configurations (FP32 factor)
    from paper_1607_00346_gb300 import hif
    hif.load()
    p = {e: hif.predict_bytes(64, 4, eps=e, precision=hif.PREC_FP32) for e in (0.0, 1e-6, 1e-5, 1e-4)}
    assert p[0.0] == p[1e-6] > p[1e-5] > p[1e-4] > 32 * 64 ** 3
    assert hif.predict_bytes(64, 4, eps=1e-6, precision=hif.PREC_FP64) > p[1e-6]
    measured = {(64, 1e-6): 2.11e9, (64, 1e-5): 1.2e9, (64, 1e-4): 0.7e9,
                (128, 1e-6): 24.9e9, (256, 1e-4): 74.3e9}
    for (n, e), peak in measured.items():
        assert hif.predict_bytes(n, 4, eps=e, precision=hif.PREC_FP32) > peak


def test_load_rejects_bad_files(tmp_path):
    from paper_1607_00346_gb300 import hif
    hif.load()
    with pytest.raises(hif.HifError) as e:
        hif.load_factor(str(tmp_path / "missing.hiff"))
    assert e.value.status == 1
    bad = tmp_path / "bad.hiff"
    bad.write_bytes(b"NOTAFACTORFILE")
    with pytest.raises(hif.HifError) as e:
        hif.load_factor(str(bad))
    assert e.value.status == 1
    trunc = tmp_path / "trunc.hiff"
    trunc.write_bytes(b"HIFF\x01\x00\x00\x00")
    with pytest.raises(hif.HifError) as e:
        hif.load_factor(str(trunc))
    assert e.value.status == 1


def test_invalid_grid_rejected_before_any_device_work():
    from paper_1607_00346_gb300 import hif
    import numpy as np
    with pytest.raises(hif.HifError) as e:
        hif.factor(20, 4, np.ones(20 ** 3))
    assert e.value.status == 1
    with pytest.raises(hif.HifError) as e:
        hif.factor(16, 4, np.ones(16 ** 3), eps=-1.0)
    assert e.value.status == 1
    o = hif.default_options(tensor_cores=2)
    g = hif.Grid(16, 4, 0)
    out = ctypes.c_void_p()
    a = np.ones(16 ** 3)
    st = hif.load().hif_factor(ctypes.byref(g), a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               None, 0.0, ctypes.byref(o), None, ctypes.byref(out))
    assert st == 1 and not out.value


def test_autotune_table_files(tmp_path):
    # the tuning table is text: a device line and one line per bucket; files
    # that are malformed or were written for another device are refused and
    # leave the table as it was
    from paper_1607_00346_gb300 import hif
    hif.load()
    hif.autotune_clear()
    text = hif.autotune_table()
    assert text.startswith("#") and "\ndevice " in text
    for bad in ("gemm 0 0 1\n", "device other_gpu\ngemm 0 0 1\n",
                "device " + text.split("device ")[1].split()[0] + "\ngemm 9 0 1\n",
                "device " + text.split("device ")[1].split()[0] + "\nid 0 0 17 0\n"):
        p = tmp_path / "t.txt"
        p.write_text(bad)
        with pytest.raises(hif.HifError) as e:
            hif.autotune_load(str(p))
        assert e.value.status == 1
    assert hif.autotune_table() == text
    good = tmp_path / "good.txt"
    tag = text.split("device ")[1].split()[0]
    # shape classes 0-2 (rows/width), 3-5 the same for shallow batches (K <= 256)
    good.write_text(f"device {tag}\ngemm 2 1 0\ngemm 5 2 1\nid 1 2 16 12\n")
    hif.autotune_load(str(good))
    t2 = hif.autotune_table()
    assert "gemm 2 1 0" in t2 and "gemm 5 2 1" in t2 and "id 1 2 16 12" in t2
    hif.autotune_clear()
    assert "gemm" not in hif.autotune_table().replace("# ", "")
