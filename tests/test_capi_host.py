"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point declared in include/vpl.h, and the
ctypes structures have the C layout."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vpl.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2203_11484_gb300 import build
    path = build.build_library()
    return C.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"VPL_API[^;(]*?\b(vpl_\w+)\s*\(", text)))


def test_header_declares_the_pipeline():
    names = declared_functions()
    for n in ("vpl_scene_upload", "vpl_generate", "vpl_gather", "vpl_render", "vpl_create", "vpl_sync"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    # nothing but the C ABI is exported
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported == set(names)


def test_binding_signatures_cover_header():
    from paper_2203_11484_gb300 import vpl
    assert set(vpl._SIGS) == set(declared_functions())


def test_struct_layout_matches_c(tmp_path):
    from paper_2203_11484_gb300 import vpl
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "vpl.h"\nint main(void){\n'
                   'printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(vpl_light), sizeof(vpl_camera),'
                   ' sizeof(vpl_gen_params), sizeof(vpl_gather_params), sizeof(vpl_vpl_set), sizeof(vpl_gbuffer),'
                   ' sizeof(vpl_scene_info), sizeof(vpl_gen_info), offsetof(vpl_gen_params, ir_max_paths),'
                   ' offsetof(vpl_gen_params, seed));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [C.sizeof(vpl.vpl_light), C.sizeof(vpl.vpl_camera), C.sizeof(vpl.vpl_gen_params),
            C.sizeof(vpl.vpl_gather_params), C.sizeof(vpl.vpl_vpl_set), C.sizeof(vpl.vpl_gbuffer),
            C.sizeof(vpl.vpl_scene_info), C.sizeof(vpl.vpl_gen_info),
            vpl.vpl_gen_params.ir_max_paths.offset, vpl.vpl_gen_params.seed.offset]
    assert got == want


def test_null_arguments_rejected_without_device(lib):
    """Argument checks run on the host before any CUDA call."""
    from paper_2203_11484_gb300 import vpl
    L = vpl.load()
    assert L.vpl_create(None, 0) == 1            # out == NULL
    assert L.vpl_sync(None, None) == 1           # ctx == NULL
    assert L.vpl_launch_count(None) == -1
    assert L.vpl_last_error(None) == b"no context"


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2203_11484_gb300 import vpl
    saved = vpl._L
    try:
        vpl._L = None
        with pytest.raises(RuntimeError, match="libvpl.so not found"):
            vpl.load(str(tmp_path / "missing.so"))
    finally:
        vpl._L = saved


def test_gather_params_marshal_every_field(tmp_path):
    """make_gather copies every GatherParams field into the ctypes struct, and
    each field of vpl_gather_params sits at the offset the C compiler gives it
    (the speed-only knobs included: a slip would silently run the default)."""
    from paper_2203_11484_gb300 import vpl, workloads as W
    p = W.GatherParams(d2_min=0.25, ray_eps=0.5, precision=2, visibility=1, tile_w=16, blocks_per_sm=3,
                       vpl_tile=32, walk=1, tile_order=2)
    s = vpl.make_gather(p)
    assert (s.d2_min, s.ray_eps) == (0.25, 0.5)
    assert (s.precision, s.visibility, s.tile_w, s.blocks_per_sm, s.vpl_tile, s.walk, s.tile_order) == \
        (2, 1, 16, 3, 32, 1, 2)
    names = [f for f, _ in vpl.vpl_gather_params._fields_]
    src = tmp_path / "off.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "vpl.h"\nint main(void){\n'
                   + "".join(f'printf("%zu\\n", offsetof(vpl_gather_params, {n}));' for n in names)
                   + "return 0;}\n")
    exe = tmp_path / "off"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [getattr(vpl.vpl_gather_params, n).offset for n in names]
