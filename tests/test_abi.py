"""The C ABI library loads and exports every symbol include/brmppi.h
declares; host-side argument checks that need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "brmppi.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300 as pkg
    return pkg.load()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(brmppi_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_functions():
    names = _declared_functions()
    assert "brmppi_create" in names and "brmppi_solve" in names and "brmppi_solve_device" in names


def test_exports_every_declared_symbol(lib):
    import paper_2508_05773_gb300 as pkg
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in pkg.EXPORTS, name
    for name in pkg.EXPORTS:
        assert name in _declared_functions(), name


def test_binding_has_every_entry_point_by_its_c_name():
    # the Python binding mirrors the C ABI name for name (argument marshalling only)
    import paper_2508_05773_gb300 as pkg
    for name in _declared_functions():
        assert callable(getattr(pkg, name, None)), name


def test_params_struct_layout_matches(lib):
    import paper_2508_05773_gb300 as pkg
    p = pkg.brmppi_default_params()
    assert p.abi_version == pkg.BRMPPI_ABI_VERSION
    assert (p.S, p.H) == (256, 30)
    assert abs(p.Ts - 0.05) < 1e-7 and abs(p.lambda_ - 1.0) < 1e-7
    assert list(p.z_lo) == [-2.0, pytest.approx(-0.6), 0.0]
    assert list(p.sigma) == [0.5, pytest.approx(0.3), 0.5]
    # last fields: a shifted layout would scramble these
    assert abs(p.rho - 0.01) < 1e-9 and abs(p.h_floor - 1e-6) < 1e-12
    assert p.q_coll == 100.0 and p.alpha_stab == 0.5 and list(p.q_stab) == [1.0, 1.0]
    assert p.q_abuf == 10.0 and p.h_buf == 0.5
    # the library checks the same sizes at compile time
    assert p.n_discs == 1 and p.disc_trailer_mask == 0 and list(p.disc_off) == [0.0] * 8
    assert ctypes.sizeof(pkg.brmppi_params) == 4 * 16 + 4 * 41 + 4 * 10
    assert ctypes.sizeof(pkg.brmppi_instance) == 8 * 4 + 4 * 5 + 4 + 8 * 2 + 8 * 9


@pytest.mark.parametrize("field,value", [
    ("S", 0), ("H", 0), ("H", 5000), ("max_obstacles", -1), ("max_obstacles", 125),
    ("max_path_pts", 1), ("max_path_pts", 8193), ("threads_per_sample", 3), ("block_threads", 48), ("Ts", 0.0),
    ("lambda_", -1.0), ("h_floor", 0.0), ("flags", 0x40), ("abi_version", 99),
    ("max_batch", -1), ("batch_threads_per_sample", 5), ("batch_block_threads", 1000),
    ("max_vehicles", -2), ("serve_lanes", 99), ("serve_max_batch", -1), ("serve_queue", -5),
    ("q_coll", -1.0), ("alpha_stab", 0.0), ("alpha_stab", 1.5), ("q_abuf", -1.0), ("h_buf", 0.0),
    ("n_discs", 0), ("n_discs", 9), ("disc_trailer_mask", 2),
])
def test_create_rejects_bad_params_without_gpu(lib, field, value):
    import paper_2508_05773_gb300 as pkg
    p = pkg.brmppi_default_params()
    setattr(p, field, value)
    with pytest.raises(pkg.BrmppiError) as ei:
        pkg.brmppi_create(p, 0)
    assert ei.value.status == pkg.BRMPPI_EINVAL
    assert pkg.brmppi_last_error(None)


def test_create_rejects_inverted_bounds(lib):
    import paper_2508_05773_gb300 as pkg
    p = pkg.brmppi_default_params()
    p.z_lo[1] = 1.0
    with pytest.raises(pkg.BrmppiError) as ei:
        pkg.brmppi_create(p, 0)
    assert ei.value.status == pkg.BRMPPI_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2508_05773_gb300 import _native
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(_native.NativeLibraryMissing):
        _native.load()


def test_product_package_never_imports_oracle():
    pkg_dir = os.path.join(ROOT, "paper_2508_05773_gb300")
    for dirpath, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "brmppi_oracle" not in text, f


def test_third_order_needs_the_rear_axle_disc(lib):
    import paper_2508_05773_gb300 as pkg
    p = pkg.brmppi_default_params()
    p.flags = pkg.BRMPPI_FLAG_THIRD_ORDER
    p.n_discs = 2
    with pytest.raises(pkg.BrmppiError) as ei:
        pkg.brmppi_create(p, 0)
    assert ei.value.status == pkg.BRMPPI_EINVAL
    assert "third-order" in pkg.brmppi_last_error(None)


def test_jerk_model_needs_the_rear_axle_disc(lib):
    import paper_2508_05773_gb300 as pkg
    p = pkg.brmppi_default_params()
    p.flags = pkg.BRMPPI_FLAG_JERK_MODEL
    p.n_discs = 3
    with pytest.raises(pkg.BrmppiError) as ei:
        pkg.brmppi_create(p, 0)
    assert ei.value.status == pkg.BRMPPI_EINVAL
    assert "jerk" in pkg.brmppi_last_error(None)

