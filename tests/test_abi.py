"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point declared in include/glmb.h (no compute calls here)."""
import ctypes
import re

import paper_2512_06230_gb300 as glmb


def test_library_exports_every_declared_symbol():
    glmb.build()
    lib = ctypes.CDLL(glmb.LIB_PATH)
    names = glmb.declared_functions()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's sizes and offsets."""
    import subprocess
    structs = {"glmb_config": glmb.GlmbConfig, "glmb_birth": glmb.GlmbBirth,
               "glmb_track": glmb.GlmbTrack, "glmb_info": glmb.GlmbInfo,
               "glmb_tuning": glmb.GlmbTuning, "glmb_frame_in": glmb.GlmbFrameIn}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{glmb.HEADER}"',
             'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    for line in filter(None, out):
        cname, field, val = line.split()
        py = structs[cname]
        want = ctypes.sizeof(py) if field == "size" else getattr(py, field).offset
        assert int(val) == want, (cname, field, int(val), want)


def test_state_buffer_round_trip_in_python():
    import numpy as np
    tracks = [[(1, 0, np.arange(4.0), np.eye(4))], []]
    buf = glmb.pack_state(3, [-0.1, -2.3], [5, 7], tracks, 4)
    fr, lw, uid, tr = glmb.unpack_state(buf)
    assert fr == 3 and list(uid) == [5, 7] and len(tr[1]) == 0
    assert np.array_equal(tr[0][0][2], np.arange(4.0))


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(glmb, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(glmb, "_lib", None)
    try:
        glmb.load()
    except RuntimeError as e:
        assert "no fallback" in str(e)
    else:
        raise AssertionError("load() must raise without the CUDA library")
