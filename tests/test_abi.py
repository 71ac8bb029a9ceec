"""The C ABI library builds, loads on a CPU-only host and exports every symbol of include/pic.h."""
import ctypes
import os
import re

from paper_1009_2727_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z0-9_]+)\s*\(", src)) - {"pic_alloc_fn", "pic_free_fn"})


def test_library_exports_every_declared_symbol():
    L = capi.load()
    names = declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(capi.EXPORTS)


def test_struct_layouts_match_header_sizes():
    # field counts of the ctypes mirrors track the header declarations
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    assert "PIC_API_VERSION 1" in src and capi.API_VERSION == 1
    assert ctypes.sizeof(capi.PicConfig) % 8 == 0
    assert ctypes.sizeof(capi.PicStats) > 100


def test_init_rejects_bad_config_without_gpu_work():
    L = capi.load()
    c = capi.PicConfig()
    c.struct_size = 3        # wrong size: rejected before any CUDA call
    c.version = capi.API_VERSION
    h = ctypes.c_void_p()
    r = L.pic_init(ctypes.byref(c), capi.ALLOC_FN(), capi.FREE_FN(), None, None, ctypes.byref(h))
    assert r == capi.PIC_EINVAL and not h.value
    assert L.pic_free(None) == capi.PIC_OK


def test_ctypes_mirrors_match_c_layout(tmp_path):
    """every field offset and struct size of the ctypes mirrors equals the C compiler's for include/pic.h"""
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"pic_config": capi.PicConfig, "pic_plasma": capi.PicPlasma, "pic_laser": capi.PicLaser,
               "pic_btd_req": capi.PicBtdReq, "pic_btd_out": capi.PicBtdOut, "pic_stats": capi.PicStats,
               "pic_tune_result": capi.PicTuneResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pic.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])


def _cfg(**over):
    from paper_1009_2727_gb300 import workloads as W
    from paper_1009_2727_gb300.pic import make_config
    w = W.parity_2d()
    w.update(over)
    return make_config(w, capi.PIC_MIXED)


def test_init_validates_filter_gather_and_dim_before_gpu_work():
    """configurations the host rejects before any CUDA call: an unknown dimension or gather scheme, a stride
    set with a gap or a negative entry, a filter halo wider than 40 cells, more than 16 passes per stride"""
    L = capi.load()
    bad = [
        _cfg(dim=4),
        _cfg(gather="energy"),
        _cfg(filter_passes=4, filter_compensate=1, filter_strides=[1, 2, 4, 8]),   # halo 75
        _cfg(filter_passes=17),
    ]
    bad[1].gather_scheme = 2
    gap = _cfg(filter_passes=1, filter_strides=[1, 0, 2])
    neg = _cfg(filter_passes=1)
    neg.filter_stride_set[0] = -1
    bad += [gap, neg]
    for c in bad:
        h = ctypes.c_void_p()
        r = L.pic_init(ctypes.byref(c), capi.ALLOC_FN(), capi.FREE_FN(), None, None, ctypes.byref(h))
        assert r == capi.PIC_EINVAL and not h.value
