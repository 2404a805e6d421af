"""The ctypes structures of the binding and the structured arrays of the input generator
have the C layout include/jt.h declares: a small C program built with the host compiler
prints every field's offset and every structure's size, which must equal what Python uses.
No GPU needed."""

import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# structure -> the C field names, in order (a field name may cover an array)
STRUCTS = {
    "jt_block_index": ["bit_offset", "dc_pred"],
    "jt_huff_spec": ["bits", "vals"],
    "jt_gbuffer": ["uv", "tex_id", "mip", "width", "height"],
    "jt_view": ["g", "out_rgba"],
    "jt_tuning": ["decode_mcus_per_warp", "decode_warps", "decode_ctas_per_sm", "pixel_threads",
                  "pixel_ctas_per_sm", "decode_short_lists"],
    "jt_scene_quad": ["cx", "cy", "ex", "ey", "h", "rep", "cs", "sn", "ou", "ov", "tex", "x0", "y0", "x1", "y1"],
    "jt_scene": ["width", "height", "cam", "rot", "ax", "ay", "tan_x", "tan_y", "max_t", "kx", "ky", "shift",
                 "cell_seed", "ntex", "use_mips", "tex_w", "tex_h", "tex_levels", "quads", "nquads", "reserved"],
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "jt.h"', "int main(void) {"]
    for s, fields in STRUCTS.items():
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines.append("  return 0;\n}")
    src = d / "abi.c"
    src.write_text("\n".join(lines))
    exe = d / "abi"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        s, f, v = ln.split()
        out[(s, f)] = int(v)
    return out


def test_binding_structures_match_the_header(c_layout):
    import paper_2510_08166_gb300 as jt
    for s, fields in STRUCTS.items():
        if s == "jt_scene_quad":
            continue
        cls = getattr(jt, s)
        assert ctypes.sizeof(cls) == c_layout[(s, "size")], s
        for f in fields:
            assert getattr(cls, f).offset == c_layout[(s, f)], (s, f)


def test_generator_records_match_the_header(c_layout):
    import synth
    dt = synth.QUAD_DTYPE
    assert dt.itemsize == c_layout[("jt_scene_quad", "size")]
    for f in STRUCTS["jt_scene_quad"]:
        assert dt.fields[f][1] == c_layout[("jt_scene_quad", f)], f
    assert synth.INDEX_DTYPE.itemsize == c_layout[("jt_block_index", "size")]
    assert synth.INDEX_DTYPE.fields["dc_pred"][1] == c_layout[("jt_block_index", "dc_pred")]
