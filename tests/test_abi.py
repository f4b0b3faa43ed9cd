"""The C-ABI library loads and exports every function declared in
include/dmrt.h; argument validation needs no GPU."""

import ctypes

import pytest

from paper_1511_04633_gb300 import build, dmrt


def test_library_builds_and_loads():
    path = build.build()
    assert path.endswith("libdmrt.so")
    lib = dmrt.load()
    assert lib is not None


def test_every_declared_function_is_exported():
    names = dmrt.declared_functions()
    assert len(names) >= 20
    raw = ctypes.CDLL(dmrt.library_path())
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_status_strings_and_version():
    assert dmrt.dmrt_status_string(0) == "DMRT_OK"
    assert dmrt.dmrt_status_string(4) == "DMRT_ERR_DIVERGED"
    assert dmrt.dmrt_status_string(99) == "DMRT_UNKNOWN"
    assert "sm_103a" in dmrt.dmrt_version()


@pytest.mark.parametrize("grid,Ra,Pr,Ma,wall", [
    ((1, 8, 8), 1e4, 0.71, 0.1, 1),     # wall box thinner than 2 cells
    ((8, 8, 8), -1.0, 0.71, 0.1, 1),    # Ra <= 0
    ((8, 8, 8), 1e4, 0.0, 0.1, 1),      # Pr <= 0
    ((8, 8, 8), 1e4, 0.71, 0.35, 1),    # Ma >= 0.3
    ((8, 8, 8), 1e4, 0.71, 0.1, 7),     # unknown wall type
    ((2000, 2000, 2000), 1e4, 0.71, 0.1, 1),  # more than 2^31 cells
])
def test_create_rejects_bad_arguments_without_touching_the_gpu(grid, Ra, Pr, Ma, wall):
    with pytest.raises(dmrt.DmrtError) as ei:
        dmrt.dmrt_create(grid, Ra, Pr, Ma, wall)
    assert ei.value.status == dmrt.ERR_ARG


def test_cells_per_thread_out_of_range_is_rejected_without_touching_the_gpu():
    for cpt in (-1, 3):
        with pytest.raises(dmrt.DmrtError) as ei:
            dmrt.dmrt_create((8, 8, 8), 1e4, cells_per_thread=cpt)
        assert ei.value.status == dmrt.ERR_ARG


def test_create_lattice_rejects_nonpositive_transport():
    for nu, alpha in ((0.0, 0.1), (0.1, -1.0), (float("nan"), 0.1)):
        with pytest.raises(dmrt.DmrtError) as ei:
            dmrt.dmrt_create_lattice((8, 8, 8), nu, alpha, 0.0, 1)
        assert ei.value.status == dmrt.ERR_ARG


def test_null_handle_calls_are_rejected():
    lib = dmrt.load()
    assert lib.dmrt_step(None, 1) == dmrt.ERR_ARG
    assert lib.dmrt_sync(None) == dmrt.ERR_ARG
    assert lib.dmrt_last_error(None) == b"null handle"
    lib.dmrt_destroy(None)


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding passes across the ABI has the size and field
    offsets that a C compiler gives the header's declaration."""
    import os
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [dmrt.dmrt_opts, dmrt.dmrt_params, dmrt.dmrt_stats, dmrt.dmrt_cavity_desc,
               dmrt.dmrt_surrogate_cfg]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dmrt.h"', "int main(void) {"]
    for s in structs:
        name = s.__name__
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in s._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", include, str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                          text=True).stdout.split("\n") if l)
    for s in structs:
        name = s.__name__
        assert int(got[name]) == ctypes.sizeof(s), name
        for f, _ in s._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(s, f).offset, (name, f)
