"""Host-only checks of the C ABI: the library builds and loads, exports every
function include/*.h declares, and the ctypes mirrors have the C layout.
No compute call is made (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1910_12214_b300 import build
    return build.build()


def declared_functions():
    src = "".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tpc_[a-z_]+)\s*\(", src)))


def test_header_declares_the_four_call_boundary():
    names = declared_functions()
    for n in ("tpc_init", "tpc_load_clusters", "tpc_track", "tpc_get_tracks", "tpc_destroy", "tpc_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (tpc_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_names_match_header(lib_path):
    from paper_1910_12214_b300 import tpc
    assert set(tpc.EXPORTED) == set(declared_functions())


def test_struct_layouts_match_c(tmp_path, lib_path):
    from paper_1910_12214_b300 import tpc
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "tpc.h"\nint main(void){'
                    'printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(tpc_config), sizeof(tpc_clusters), '
                    'sizeof(tpc_track_t), offsetof(tpc_track_t, chi2), offsetof(tpc_config, allocator), '
                    'offsetof(tpc_clusters, on_device), sizeof(tpc_tuning), offsetof(tpc_tuning, merge_sort_cap));'
                    ' return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(tpc.tpc_config), ctypes.sizeof(tpc.tpc_clusters), tpc.TRACK_DTYPE.itemsize,
                    tpc.TRACK_DTYPE.fields["chi2"][1], tpc.tpc_config.allocator.offset,
                    tpc.tpc_clusters.on_device.offset, ctypes.sizeof(tpc.tpc_tuning),
                    tpc.tpc_tuning.merge_sort_cap.offset]


def test_init_rejects_invalid_config_without_touching_the_gpu(lib_path):
    from paper_1910_12214_b300 import tpc
    cfg = tpc.tpc_config(0, None, 0.5, 2, 85.0, 246.0, 10.0, 0.1, 0.1, 0, 0, 0, 0, None, 0)  # 2 rows: invalid
    h = ctypes.c_void_p()
    assert tpc._lib.tpc_init(ctypes.byref(cfg), ctypes.byref(h)) == 1
    assert not h.value
    assert tpc._lib.tpc_init(None, ctypes.byref(h)) == 1
    assert tpc._lib.tpc_last_error(None) == b"null context"


def test_oracle_library_loads():
    import oracle
    oracle.build_oracle()
    assert os.path.exists(oracle.oracle.LIB)


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1910_12214_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "tpc_oracle" not in txt, f


def test_reduce_struct_layouts_match_c(tmp_path, lib_path):
    from paper_1910_12214_b300 import tpc
    prog = tmp_path / "rz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "tpc_reduce.h"\nint main(void){'
                    'printf("%zu %zu %zu %zu\\n", sizeof(tpc_cluster_props), sizeof(tpc_cluster_codes), '
                    'offsetof(tpc_cluster_props, n), sizeof(tpc_mask_params) + 100 * sizeof(tpc_cluster_charges)); return 0;}\n')
    exe = tmp_path / "rz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(tpc.tpc_cluster_props), ctypes.sizeof(tpc.tpc_cluster_codes),
                    tpc.tpc_cluster_props.n.offset,
                    ctypes.sizeof(tpc.tpc_mask_params) + 100 * ctypes.sizeof(tpc.tpc_cluster_charges)]
