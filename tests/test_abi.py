"""C ABI checks that need no GPU: the library builds, loads and exports every
function the public header declares, and the ctypes mirrors of the structs
have the C layout."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fdc.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


@pytest.fixture(scope="module")
def libfdc():
    from paper_1011_2188_gb300 import build, fdc
    build.build()
    return fdc.lib()


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdc_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fdc_load_database", "fdc_load_phantom", "fdc_run", "fdc_run_ex", "fdc_sync",
                     "fdc_create", "fdc_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libfdc):
    from paper_1011_2188_gb300 import fdc
    for name in declared_functions():
        assert hasattr(libfdc, name), name
        assert name in fdc.SIGNATURES, f"binding lacks {name}"
    out = subprocess.run(["nm", "-D", "--defined-only", fdc.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(fdc_\w+)", out))
    assert set(declared_functions()) <= exported


def test_struct_layouts_match_c():
    from paper_1011_2188_gb300 import fdc
    from paper_1011_2188_gb300.denoise import Conv3d
    structs = {
        "fdc_conv3d": Conv3d,
        "fdc_database": fdc.Database, "fdc_phantom": fdc.Phantom, "fdc_spot": fdc.Spot,
        "fdc_beam": fdc.Beam, "fdc_schedule": fdc.Schedule, "fdc_run_opts": fdc.RunOpts,
        "fdc_outputs": fdc.Outputs, "fdc_counters": fdc.Counters,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>'] + [f'#include "{h}"' for h in HEADERS] + ["int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c11", "-o", exe, src], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(l.split() for l in out.strip().splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"


def test_loading_without_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1011_2188_gb300 import fdc
    monkeypatch.setattr(fdc, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(fdc, "_lib", None)
    with pytest.raises(RuntimeError):
        fdc.lib()
