"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point declared in include/glmb.h (no compute calls here)."""
import ctypes
import re

import pytest

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


def test_device_detections_are_checked_before_the_call():
    """Detections passed as device memory must be a contiguous float32 CUDA
    tensor of shape (M, dim_z); the binding refuses anything else before a
    kernel could read it (host logic, checked with stand-in tensors)."""
    import types

    import paper_2512_06230_gb300 as g

    def fake(**kw):
        a = dict(is_cuda=True, dtype="float32", shape=(3, 2), data_ptr=lambda: 4096,
                 is_floating_point=lambda: True, is_complex=lambda: False, element_size=lambda: 4,
                 dim=lambda: len(a["shape"]), is_contiguous=lambda: True)
        a.update(kw)
        return types.SimpleNamespace(**a)

    f = types.SimpleNamespace(dz=2)
    ptr, M = g.Filter._dev_z(f, fake())
    assert M == 3 and ptr.value == 4096
    assert g.Filter._dev_z(f, fake(shape=(0, 3)))[1] == 0      # empty: any width
    bad = [(fake(is_cuda=False), TypeError), (fake(element_size=lambda: 8), TypeError),
           (fake(is_floating_point=lambda: False), TypeError), (fake(shape=(3, 3)), ValueError),
           (fake(shape=(6,)), ValueError), (fake(is_contiguous=lambda: False), ValueError)]
    for z, err in bad:
        with pytest.raises(err):
            g.Filter._dev_z(f, z)
    import numpy as np
    with pytest.raises(TypeError):
        g.Filter._dev_z(f, np.zeros((3, 2), np.float32))
