"""The C ABI without a GPU: the library builds, loads and exports every symbol include/ovs.h declares; the
ctypes structs match the header's layout (checked by compiling a C probe of the header with gcc); sizing
calls work on the host; and a context on a machine without a usable GPU fails with OVS_ERR_NO_DEVICE
(there is no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1910_09315_gb300 import build, ovs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ovs.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ovs.load()


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(ovs_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    assert sorted(names) == sorted(ovs.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", ovs.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", out, flags=re.M), n


def test_struct_layout_matches_header(tmp_path):
    structs = {"ovs_grid_desc": ovs.ovs_grid_desc, "ovs_fringe_set": ovs.ovs_fringe_set, "ovs_donors": ovs.ovs_donors,
               "ovs_fields": ovs.ovs_fields, "ovs_fields_out": ovs.ovs_fields_out, "ovs_options": ovs.ovs_options,
               "ovs_stats": ovs.ovs_stats, "ovs_train_desc": ovs.ovs_train_desc, "ovs_tuning": ovs.ovs_tuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ovs.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    for macro in ("OVS_MAX_GRIDS", "OVS_MAX_SETS", "OVS_MAX_DONORS", "OVS_STATUS_FALLBACK", "OVS_STATUS_REFINED",
                  "OVS_ERR_NO_DEVICE", "OVS_GUESS_MLP", "OVS_GUESS_MLP_ONLY", "OVS_VEL_NONE", "OVS_LAUNCH_DIRECT",
                  "OVS_LAUNCH_GRAPH"):
        lines.append(f'printf("{macro} %d\\n", (int)({macro}));')
    lines.append("return 0;}")
    c = tmp_path / "probe.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), "-o", str(exe), str(c)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)
    for macro in ("OVS_MAX_GRIDS", "OVS_MAX_SETS", "OVS_MAX_DONORS", "OVS_STATUS_FALLBACK", "OVS_STATUS_REFINED",
                  "OVS_ERR_NO_DEVICE", "OVS_GUESS_MLP", "OVS_GUESS_MLP_ONLY", "OVS_VEL_NONE", "OVS_LAUNCH_DIRECT",
                  "OVS_LAUNCH_GRAPH"):
        assert int(got[macro]) == getattr(ovs, macro), macro


def test_grid_workspace_size_on_host(lib):
    d = ovs.ovs_grid_desc()
    d.n[0], d.n[1], d.n[2] = 33, 17, 9
    dummy = ctypes.c_double(0)
    d.x = d.y = d.z = ctypes.addressof(dummy)
    d.role = 1
    nbytes = ovs.ovs_grid_workspace_size(d)
    cells = 32 * 16 * 8
    assert nbytes >= 128 * cells + 4 * 33 * 17 * 9
    d.n[0] = 1
    with pytest.raises(ovs.OvsError):
        ovs.ovs_grid_workspace_size(d)
    d.n[0] = 2
    d.periodic[0] = 1
    with pytest.raises(ovs.OvsError):
        ovs.ovs_grid_workspace_size(d)


def test_no_device_is_an_error_not_a_fallback(lib, cuda_available):
    if cuda_available:
        pytest.skip("a GPU is present")
    ctx = ctypes.c_void_p()
    rc = lib.ovs_ctx_create(ctypes.byref(ctx), 0, None)
    assert rc == ovs.OVS_ERR_NO_DEVICE
    assert not ctx.value
    with pytest.raises(RuntimeError):
        ovs.Context()


def test_null_arguments_rejected(lib):
    assert lib.ovs_ctx_create(None, 0, None) == ovs.OVS_ERR_ARG
    assert lib.ovs_assemble(None, None, 0, None) == ovs.OVS_ERR_ARG
    assert lib.ovs_sync(None) == ovs.OVS_ERR_ARG
    assert lib.ovs_last_error(None) == b"null context"
