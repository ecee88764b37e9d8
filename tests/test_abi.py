"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/sph.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2511_11425_gb300 import build
    return build.build()


def test_header_declares_the_paper_calls():
    names = _declared()
    for n in ("sph_build_cells", "sph_density_h", "sph_forces", "sph_kdk_step",
              "sph_reduce_conserved", "sph_create", "sph_destroy", "sph_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    import paper_2511_11425_gb300 as sph
    for n in _declared():
        assert callable(getattr(sph, n)), n
    assert sph.sph_version().startswith("libsph")


def test_struct_layouts_match_header(libpath):
    # sph_particles: n + 21 pointers; sph_params as laid out by a C compiler
    import paper_2511_11425_gb300 as sph
    assert ctypes.sizeof(sph.c_particles) == 8 + 22 * 8
    assert ctypes.sizeof(sph.c_params) == 224
    assert sph.c_params.h_rel_tol.offset == 128 and sph.c_params.list_margin.offset == 136
    assert sph.c_params.curve.offset == 144 and sph.c_params.group_log.offset == 148
    assert ctypes.sizeof(sph.c_stats) == 112 + 16 * 8 + 16 * 8


def test_struct_offsets_agree_with_the_c_compiler(tmp_path):
    """Every member offset of the ctypes mirrors equals the one gcc gives the
    header's structs (catches a member added to one side only)."""
    import shutil
    import subprocess
    import paper_2511_11425_gb300 as sph
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    mirrors = {"sph_params": sph.c_params, "sph_particles": sph.c_particles,
               "sph_stats": sph.c_stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", "#include \"sph.h\"",
             "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "off.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "off"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            c, f, v = line.split()
            got[(c, f)] = int(v)
    for cname, cls in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_create_rejects_bad_parameters_without_touching_the_gpu(libpath):
    import paper_2511_11425_gb300 as sph
    with pytest.raises(sph.SphError):
        sph.sph_create(sph.Params(gamma=1.0), 10)
    with pytest.raises(sph.SphError):
        sph.sph_create(sph.Params(box_hi=(0.0, 1.0, 1.0)), 10)
    with pytest.raises(sph.SphError):
        sph.sph_create(sph.Params(max_newton=0), 10)
    with pytest.raises(sph.SphError):
        sph.sph_create(sph.Params(group_log=4), 10)
    with pytest.raises(sph.SphError):
        sph.sph_create(sph.Params(bucket_cell=0.5), 10)
    with pytest.raises(sph.SphError):
        sph.sph_create(sph.Params(bucket_cell=4.0, group_cell=3.0), 10)
    with pytest.raises(sph.SphError):
        sph.sph_create(sph.Params(resort_period=65), 10)


def test_noalloc_binding_refuses_unusable_out_buffers():
    """The allocation-free totals write 9 doubles through a raw device
    pointer: the binding refuses anything else before calling the library."""
    import numpy as np
    import torch

    import paper_2511_11425_gb300 as sph
    from paper_2511_11425_gb300 import inputs
    prob = inputs.uniform(n=4, seed=1)
    parts = sph.Particles.from_problem(prob, "cpu")
    for bad in (np.zeros(9), torch.zeros(9, dtype=torch.float64)):
        with pytest.raises(ValueError):
            sph.sph_reduce_conserved_noalloc(parts, bad)
