"""The C-ABI library loads and exports every function include/kairos.h declares.  CPU
only: no call here touches a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2401_02563_gb300 as kx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(kairos_[a-z0-9_]+)\s*\(",
                                    text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def library():
    try:
        return kx.lib()
    except Exception as e:  # nvcc missing here means the build check fails elsewhere too
        pytest.fail(f"libkairos.so failed to build or load: {e}")


def test_every_declared_symbol_is_exported(library):
    names = declared_functions()
    assert {"kairos_graph_build", "kairos_index_build", "kairos_earliest_arrival", "kairos_latest_departure",
            "kairos_batch_query", "kairos_serve_submit", "kairos_serve_poll"} <= names
    for name in sorted(names):
        assert hasattr(library, name), name


def test_binding_covers_the_header():
    assert declared_functions() == set(kx.SIGNATURES)


def test_status_strings(library):
    assert library.kairos_status_string(kx.KAIROS_ERR_BUSY) == b"KAIROS_ERR_BUSY"
    assert library.kairos_status_string(kx.KAIROS_OK) == b"KAIROS_OK"


STRUCTS = ["kairos_edge_list", "kairos_graph_opts", "kairos_query", "kairos_query_stats", "kairos_tuning",
           "kairos_graph_info", "kairos_serve_opts", "kairos_result_info", "kairos_fastest_stats",
           "kairos_duration_stats"]


def test_binding_struct_layouts_match_the_c_compiler(tmp_path):
    """sizeof and every field offset of the binding's ctypes structs equal gcc's."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "kairos.h"', "int main(void){"]
    for name in STRUCTS:
        cls = getattr(kx, name)
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            cname = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {cname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name in STRUCTS:
        cls = getattr(kx, name)
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


def test_null_arguments_are_rejected_without_a_device(library):
    h = ctypes.c_void_p()
    assert library.kairos_graph_build(None, None, ctypes.byref(h)) == kx.KAIROS_ERR_INVALID_ARG
    assert library.kairos_index_build(None, 16) == kx.KAIROS_ERR_INVALID_ARG
    assert library.kairos_earliest_arrival(None, 0, 0, 1, None) == kx.KAIROS_ERR_INVALID_ARG
    for fn in (library.kairos_fastest_path, library.kairos_shortest_duration, library.kairos_temporal_bfs):
        assert fn(None, 0, 0, 1, 0, None, None) == kx.KAIROS_ERR_INVALID_ARG
    assert b"NULL" in library.kairos_last_error()
    library.kairos_graph_free(None)
    library.kairos_serve_destroy(None)


def test_readme_c_example_compiles_and_links(tmp_path, library):
    """The C example of the README builds against the header and links against the library
    (running it needs a GPU)."""
    import re
    text = open(os.path.join(ROOT, "README.md")).read()
    code = re.search(r"```c\n(.*?)```", text, re.S).group(1)
    src = tmp_path / "example.c"
    src.write_text(code)
    libdir = os.path.dirname(kx.library_path())
    subprocess.check_call(["gcc", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                           str(tmp_path / "example"), "-L", libdir, "-lkairos", f"-Wl,-rpath,{libdir}"])
