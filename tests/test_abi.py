"""The C-ABI library builds, loads and exports every call of include/tsim.h.

CPU only: nothing here launches a kernel.  Struct layouts of the ctypes
binding are checked against the C header compiled with gcc.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2405_02914_gb300 import tsim
from paper_2405_02914_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tsim.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tsim_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_loads():
    path = B.build()
    assert os.path.exists(path)
    tsim.load()


def test_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 19
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (tsim_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(names) == set(tsim.EXPORTS)


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "tsim.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(tsim_gel_desc),'
                    'sizeof(tsim_material), sizeof(tsim_indenter_desc), sizeof(tsim_keyframe),'
                    'sizeof(tsim_solver_desc), sizeof(tsim_stats_t), offsetof(tsim_indenter_desc, perm));'
                    'printf("%zu %zu\\n", sizeof(tsim_tuning_t), offsetof(tsim_tuning_t, us_per_mupdate));'
                    'printf("%zu %zu\\n", sizeof(tsim_render_desc), offsetof(tsim_render_desc, seed));'
                    'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    got = [int(a) for a in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(tsim.GelDesc), C.sizeof(tsim.MaterialDesc), C.sizeof(tsim.IndenterDesc),
            C.sizeof(tsim.Keyframe), C.sizeof(tsim.SolverDesc), C.sizeof(tsim.Stats),
            tsim.IndenterDesc.perm.offset, C.sizeof(tsim.Tuning), tsim.Tuning.us_per_mupdate.offset,
            C.sizeof(tsim.RenderDesc), tsim.RenderDesc.seed.offset]
    assert got == want


def test_invalid_arguments_rejected_without_gpu():
    L = tsim.load()
    out = C.c_void_p()
    g = tsim.GelDesc()
    m = tsim.MaterialDesc()
    assert L.tsim_create(0, C.byref(g), C.byref(m), None, C.byref(out)) == 1
    assert out.value is None
    assert "instances" in L.tsim_last_error().decode()
    assert L.tsim_step(None, 1) == 1
    assert L.tsim_sync(None) == 1
    assert L.tsim_read_log(None, 0, None, None, 1) == 1
    # a node box that is not a multiple of 4 is rejected before any allocation
    g.cx, g.cy, g.cz, g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.ppc, g.dx = 4, 4, 4, 13, 12, 16, 4, 4, 4, 8, 1e-3
    m.E, m.nu, m.rho = 1e5, 0.4, 1000.0
    assert L.tsim_create(1, C.byref(g), C.byref(m), None, C.byref(out)) == 1
    t = tsim.Tuning(256, 0, 20, 0.0)
    assert L.tsim_set_tuning(None, C.byref(t)) == 1
    assert L.tsim_get_tuning(None, C.byref(t)) == 1
    assert L.tsim_autotune(None, 600, None) == 1
    L.tsim_destroy(None)
    # the block capacity: 1.25x the 512 particles of a full block at 8 per cell
    assert tsim.tsim_block_slots() == 640
    # object particles, sensor image and metrics: bad arguments are refused before any GPU work
    assert L.tsim_set_object_particles(None, 0, None, 0, C.c_float(0.0), 0) == 1
    assert L.tsim_render(None, None, 8, 8, C.c_float(1e-3), None, None, None) == 1
    d = tsim.render_desc([], spp=0, max_bounces=1)
    assert L.tsim_render(None, None, 8, 8, C.c_float(1e-3), C.byref(d), None, None) == 1
    out = (C.c_double * 3)()
    assert L.tsim_image_metrics(None, None, 10, 10, 3, C.c_float(1.0), out, None) == 1      # below 11 x 11
    assert "11 x 11" in L.tsim_last_error().decode()


def test_descriptors_from_inputs():
    from paper_2405_02914_gb300 import inputs as I
    sc = I.scene_pad4m(seed=1)
    g = tsim.gel_desc(sc.gel)
    assert (g.nx, g.ny, g.nz) == (136, 136, 44) and g.cx == 128
    ind = tsim.indenter_desc(sc.ind)
    assert ind.kind == I.CYLINDER and abs(ind.tip_offset - 5e-3) < 1e-9
    kf = tsim.keyframes(sc.keyframes)
    assert len(kf) == 4 and kf[3].substep == 20000
    for cx in (5, 13, 31):
        nx, ny, nz = I.Gel(cx, cx + 2, 3, 1e-3).nodes
        assert nx % 4 == 0 and ny % 4 == 0 and nz % 4 == 0 and nx >= cx + 8


def test_surrogate_header_symbols_exported():
    from paper_2405_02914_gb300 import tsurr
    src = open(os.path.join(ROOT, "include", "tsurr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = sorted(set(re.findall(r"\b(tsurr_[a-z0-9_]+)\s*\(", src)))
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (tsurr_[a-z0-9_]+)$", out, flags=re.M))
    assert names and not [n for n in names if n not in exported]
    assert set(names) == set(tsurr.EXPORTS)
    tsurr.load()


def test_surrogate_invalid_arguments_rejected_without_gpu():
    from paper_2405_02914_gb300 import tsurr
    L = tsurr.load()
    out = C.c_void_p()
    assert L.tsurr_create(4, 12, 16, None, C.byref(out)) == 1          # not a multiple of 8
    assert out.value is None
    assert L.tsurr_create(0, 16, 16, None, C.byref(out)) == 1
    assert L.tsurr_forward(None, None, 1, None, 1) == 1
    assert L.tsurr_backward(None, None, None, None, 1, None, 1) == 1
    assert L.tsurr_adam(None, 1e-3, 0.9, 0.999, 1e-8, 1) == 1
    assert L.tsurr_num_params(None) == 0
    L.tsurr_destroy(None)


def test_surrogate_layer_table_matches_inputs():
    from paper_2405_02914_gb300 import inputs as I
    from paper_2405_02914_gb300 import tsurr
    assert [(a, b) for a, b, *_ in tsurr.LAYERS] == I.SURR_CONVS
    assert tsurr.num_params() == I.surrogate_params(0).size == 1374160
