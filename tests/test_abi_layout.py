"""The ctypes mirrors of the C ABI's structs (paper_2211_04045_gb300/cch.py)
have the C header's layout: every field at the offset and of the size the C
compiler gives it, and the same total size (no GPU; compiles a probe with
the host C compiler against include/cch.h).  The same holds for the
oracle's own structs and their mirrors in oracle/__init__.py."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2211_04045_gb300 import cch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"cch_params": cch.Params, "cch_topology": cch.Topology, "cch_step_stats": cch.StepStats,
           "cch_tune_result": cch.TuneResult}


def c_layout(tmp_path, structs=STRUCTS, header="cch.h", incdir=os.path.join(ROOT, "include")):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{header}"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu %zu\\n", offsetof({cname}, {f}), sizeof((({cname}*)0)->{f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c11", "-I", incdir, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        parts = line.split()
        if parts[1] == "size":
            layout[(parts[0], None)] = int(parts[2])
        else:
            layout[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    return layout


def test_ctypes_structs_match_the_header(tmp_path):
    layout = c_layout(tmp_path)
    for cname, py in STRUCTS.items():
        assert C.sizeof(py) == layout[(cname, None)], cname
        for f, _ in py._fields_:
            fd = getattr(py, f)
            assert (fd.offset, fd.size) == layout[(cname, f)], (cname, f)


def test_oracle_structs_match_its_header(tmp_path):
    import oracle
    structs = {"orc_topology": oracle.Topology, "orc_params": oracle.Params, "orc_stats": oracle.Stats,
               "orc_trace": oracle.Trace}
    layout = c_layout(tmp_path, structs, "cch_oracle.h", os.path.join(ROOT, "oracle"))
    for cname, py in structs.items():
        assert C.sizeof(py) == layout[(cname, None)], cname
        for f, _ in py._fields_:
            fd = getattr(py, f)
            assert (fd.offset, fd.size) == layout[(cname, f)], (cname, f)
