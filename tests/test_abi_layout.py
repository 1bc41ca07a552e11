"""The Python binding's ctypes structures have the layout of the C structures
of include/tpc.h: a small C program compiled with the host compiler prints
every field's offset and every structure's size (no GPU needed)."""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def pairs():
    from paper_2601_20569_gb300 import tpc

    return [(tpc.Geometry, "tpc_geometry"), (tpc.Map, "tpc_map"), (tpc.Options, "tpc_options"),
            (tpc.Clusters, "tpc_clusters"), (tpc.Tracks, "tpc_tracks"),
            (tpc.RemovalOptions, "tpc_removal_options"), (tpc.Removal, "tpc_removal")]


def test_ctypes_structures_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "tpc.h"', "int main(void) {"]
    want = {}
    for cls, cname in pairs():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        want[f"{cname} size"] = ctypes.sizeof(cls)
        for name, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{name} %zu\\n", offsetof({cname}, {name}));')
            want[f"{cname}.{name}"] = getattr(cls, name).offset
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                           str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        key, val = line.rsplit(" ", 1)
        got[key] = int(val)
    assert got == want


def test_oracle_option_structure_matches_its_binding(tmp_path):
    """The oracle's option struct (plain C++, in oracle.cpp) against the
    oracle binding's ctypes structure."""
    import oracle

    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    lines = ["#include <cstddef>", "#include <cstdio>", '#include "oracle.cpp"', "int main() {",
             '  std::printf("size %zu\\n", sizeof(orc_options));']
    want = {"size": ctypes.sizeof(oracle._Opt)}
    for name, _ in oracle._Opt._fields_:
        lines.append(f'  std::printf("{name} %zu\\n", offsetof(orc_options, {name}));')
        want[name] = getattr(oracle._Opt, name).offset
    lines += ["  return 0;", "}"]
    src = tmp_path / "olayout.cpp"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "olayout"
    subprocess.check_call([cxx, "-std=c++17", "-O0", "-I", os.path.join(ROOT, "oracle"), str(src),
                           "-o", str(exe)])
    got = dict((k, int(v)) for k, v in (l.rsplit(" ", 1) for l in
                                         subprocess.check_output([str(exe)], text=True).splitlines()))
    assert got == want
