"""The C-ABI library builds, loads without a GPU and exports every function
that include/*.h declares (no compute call is made here)."""
import glob
import os
import re

from paper_2004_11040_gb300 import build, ecmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ecmc_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    build.build()
    lib = ecmc.load()
    names = declared_functions()
    assert {"ecmc_create", "ecmc_run_to_breakpoint", "ecmc_positions", "ecmc_stats"} <= names
    for name in sorted(names):
        assert hasattr(lib, name), name
    assert set(ecmc.EXPORTS) <= names


def test_binding_structs_match_header_sizes(tmp_path):
    """The ctypes structs have the sizes and field offsets a C compiler gives
    the header's structs."""
    import ctypes as C
    import subprocess
    structs = {"ecmc_params": ecmc.ecmc_params, "ecmc_stats_t": ecmc.ecmc_stats_t,
               "ecmc_profile_t": ecmc.ecmc_profile_t}
    lines = []
    for name, cls in structs.items():
        lines.append(f'printf("%zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({name}, {f[0]}));')
    lines.append('printf("%zu\\n", sizeof(ecmc_lift_t));')
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ecmc.h"\n'
                   'int main(void) {\n' + "\n".join(lines) + '\nreturn 0; }\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = []
    for cls in structs.values():
        want.append(C.sizeof(cls))
        want.extend(getattr(cls, f[0]).offset for f in cls._fields_)
    want.append(ecmc.LIFT_DTYPE.itemsize)
    assert got == want


def test_create_rejects_bad_parameters_without_gpu():
    import numpy as np
    import pytest
    x = np.array([0.5, 2.0, 3.5])
    y = np.array([0.5, 0.5, 0.5])
    # box too small for three cells of side > d: rejected before any CUDA call
    with pytest.raises(ecmc.EcmcError) as e:
        ecmc.System(x, y, [0], box=2.5, ell=1.0)
    assert e.value.code == ecmc.ECMC_EINVAL
