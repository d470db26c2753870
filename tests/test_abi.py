"""The C ABI library builds, loads and exports every symbol include/dri.h declares
(no GPU needed: no CUDA call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:int|const char\*)\s+(dri_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2207_10940_gb300 import build
    try:
        build.build()
    except RuntimeError as exc:         # no toolkit: nothing to check here
        pytest.skip(str(exc))
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("dri_create_stream", "dri_upload_frame", "dri_push_imu", "dri_track",
              "dri_get_state", "dri_set_state", "dri_destroy_stream", "dri_linearise"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points_run_without_a_gpu(lib):
    from paper_2207_10940_gb300 import dri
    cfg = dri.dri_config_default(640, 480)
    assert cfg.levels == 3 and list(cfg.iters)[:3] == [10, 5, 4]
    assert cfg.fx == pytest.approx(554.0)
    n = dri.dri_stream_workspace_bytes(cfg)
    assert n > 640 * 480 * 4 * 2
    cfg.levels = 9
    with pytest.raises(dri.DriError) as e:
        dri.dri_stream_workspace_bytes(cfg)
    assert e.value.code == dri.DRI_EINVAL
    assert dri.status_string(dri.DRI_ELOST) == "tracking lost"


def test_fp16_maps_shrink_the_workspace(lib):
    from paper_2207_10940_gb300 import dri
    a = dri.dri_config_default(640, 480)
    b = dri.dri_config_default(640, 480)
    b.precision_flags = dri.DRI_FP16_MAPS
    assert dri.dri_stream_workspace_bytes(b) < dri.dri_stream_workspace_bytes(a)


STRUCTS = ("dri_stream_config", "dri_imu_sample", "dri_state", "dri_track_result", "dri_linearisation",
           "dri_profile", "dri_batch_options", "dri_server_stats", "dri_server_tick")


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors in dri.py have the C header's size and field offsets
    (a small C program compiled against include/dri.h prints them)."""
    import shutil
    import subprocess
    from paper_2207_10940_gb300 import dri
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "dri.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(dri, name)._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    c_layout = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        *key, value = line.split()
        c_layout[tuple(key)] = int(value)
    for name in STRUCTS:
        cls = getattr(dri, name)
        assert c_layout[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert c_layout[(name, field)] == getattr(cls, field).offset, (name, field)
