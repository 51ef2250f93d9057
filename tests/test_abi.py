"""The C-ABI library builds, loads and exports every function that
include/qslab.h declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qslab.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qslab_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2403_01521_gb300 as qslab
    return qslab.load()


def test_declarations_found():
    names = _declared()
    assert "qslab_compute" in names and "qslab_create" in names
    assert len(names) >= 18


def test_every_declared_symbol_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_strerror_without_gpu(lib):
    import paper_2403_01521_gb300 as qslab
    assert qslab.qslab_strerror(0) == "success"
    for code in range(-10, 0):
        assert qslab.qslab_strerror(code) not in ("", "unknown error")
    assert qslab.qslab_strerror(-99) == "unknown error"


def test_null_context_is_rejected(lib):
    # host-side argument checks run before any CUDA call
    assert lib.qslab_set_box(None, 1.0, 1.0, 1.0) == -1
    assert lib.qslab_compute(None, 10, None, None, None, None, None, None) == -1
    assert lib.qslab_num_modes(None) == -1
    assert lib.qslab_compute_virial(None, 10, None, None, None, None, None, None, None) == -1
    assert lib.qslab_compute_batched_virial(None, 1, None, None, None, None, None, None, None,
                                            None, None) == -1
    assert lib.qslab_compute_realspace_virial(None, 10, None, None, None, None, None, None,
                                              None) == -1
    assert lib.qslab_compute_energy(None, 10, None, None, None, None) == -1
    assert lib.qslab_compute_batched_energy(None, 1, None, None, None, None, None, None) == -1
    assert lib.qslab_compute_adjoint(None, None, None, None) == -1
    assert lib.qslab_measure_peaks(0, None, None) == -1


def test_library_is_in_tree():
    import paper_2403_01521_gb300 as qslab
    path = qslab.library_path()
    assert path.startswith(os.path.join(ROOT, "paper_2403_01521_gb300"))
    assert os.path.exists(path)


def test_status_codes_match_header():
    import paper_2403_01521_gb300 as qslab
    src = open(os.path.join(ROOT, "include", "qslab.h")).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"#define (QSLAB_(?:OK|ERR_[A-Z_]+))\s+\(?(-?\d+)\)?", src))
    assert len(codes) >= 10
    for name, value in codes.items():
        assert getattr(qslab, name) == value, name


def test_walls_null_context_is_rejected(lib):
    assert lib.qslab_set_walls(None, 0.0, 0.0, 0, None, None, None) == -1
    assert lib.qslab_clear_walls(None) == -1
