"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
and exports every entry point that include/voxcap.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "voxcap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(voxcap_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2004_02609_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (voxcap_[a-z_0-9]+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing


def test_binding_loads_and_lists_all_symbols(libpath):
    from paper_2004_02609_gb300 import voxcap as V
    L = V.lib()
    assert sorted(V.SYMBOLS) == sorted(s for s in _declared() if s in V.SYMBOLS)
    for s in _declared():
        assert hasattr(L, s), s


def test_default_options(libpath):
    from paper_2004_02609_gb300 import voxcap as V
    o = V.default_opts()
    assert o.restart == 35 and list(o.nv) == [10, 10, 10]
    assert o.precision == V.FP32_REFINE and o.precond == V.PRECOND["bdd"]
    o = V.default_opts(nv=5, precond="diag", precision="fp64")
    assert list(o.nv) == [5, 5, 5] and o.precond == 2 and o.precision == 0


def test_errors_are_status_codes_without_gpu(libpath):
    """Argument errors come back as status codes with a message; nothing aborts."""
    import ctypes
    from paper_2004_02609_gb300 import voxcap as V
    L = V.lib()
    rc = L.voxcap_num_panels(None, 0, None, None, None, None, None)
    assert rc == -1
    assert b"NULL" in L.voxcap_last_error()
    rc = L.voxcap_entries(-1, None, None, None, None, None)
    assert rc == -1
    h = ctypes.c_void_p()
    rc = L.voxcap_setup(None, 1, 1, 1, 1, None, None, 1, 1.0, None, None, ctypes.byref(h))
    assert rc == -1 and not h.value


def test_struct_layouts_match_header(tmp_path, libpath):
    """The ctypes mirrors of voxcap_opts / voxcap_stats / voxcap_tucker have
    the sizes and field offsets the C compiler gives the header's structs."""
    import ctypes
    from paper_2004_02609_gb300 import voxcap as V
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "voxcap.h"\n'
                   'int main(){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(voxcap_opts), '
                   'sizeof(voxcap_stats), sizeof(voxcap_tucker), offsetof(voxcap_opts, tucker), '
                   'offsetof(voxcap_opts, pad_mode), offsetof(voxcap_opts, entries), '
                   'offsetof(voxcap_tucker, factor));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(V.Opts), ctypes.sizeof(V.Stats), ctypes.sizeof(V.Tucker),
            V.Opts.tucker.offset, V.Opts.pad_mode.offset, V.Opts.entries.offset, V.Tucker.factor.offset]
    assert got == want


def test_argument_checks_before_any_device_work(libpath):
    """Invalid arguments of every entry point that takes a handle, a size or a
    table are rejected with VOXCAP_ERR_ARG (-1) and a message, before any CUDA
    call (so this runs without a GPU)."""
    import ctypes
    import numpy as np
    from paper_2004_02609_gb300 import voxcap as V
    L = V.lib()
    lab = np.zeros(8, np.int32)
    cid = np.array([-1, 0], np.int32)
    eps = np.array([1.0, 1.0])
    h = ctypes.c_void_p()
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    cases = {
        "non-positive grid": lambda: L.voxcap_setup(P(lab), 0, 2, 2, 1, P(cid), P(eps), 2, 1e-6, None, None,
                                                    ctypes.byref(h)),
        "non-positive voxel": lambda: L.voxcap_setup(P(lab), 2, 2, 2, 1, P(cid), P(eps), 2, 0.0, None, None,
                                                     ctypes.byref(h)),
        "bad conductor id": lambda: L.voxcap_setup(P(lab), 2, 2, 2, 1, P(np.array([-2, 0], np.int32)), P(eps),
                                                   2, 1e-6, None, None, ctypes.byref(h)),
        "bad permittivity": lambda: L.voxcap_setup(P(lab), 2, 2, 2, 1, P(cid), P(np.array([-1.0, 1.0])), 2,
                                                   1e-6, None, None, ctypes.byref(h)),
        "NULL out": lambda: L.voxcap_setup(P(lab), 2, 2, 2, 1, P(cid), P(eps), 2, 1e-6, None, None, None),
        "matvec NULL handle": lambda: L.voxcap_matvec(None, None, None, 1, 0, 0),
        "solve NULL handle": lambda: L.voxcap_solve(None, None, 1, 1e-6, None, None),
        "capacitance NULL handle": lambda: L.voxcap_capacitance(None, 1e-6, None, None, None),
        "gradient NULL handle": lambda: L.voxcap_capacitance_grad(None, None, 1e-6, None, None),
        "update_eps NULL handle": lambda: L.voxcap_update_eps(None, None),
        "panel map NULL handle": lambda: L.voxcap_panel_map(None, 0, None, None, None, None, None, None),
        "toeplitz NULL handle": lambda: L.voxcap_toeplitz(None, 0, None, None),
        "product tiles NULL handle": lambda: L.voxcap_set_product_tiles(None, 0, 4, -1, -1, None),
    }
    for name, call in cases.items():
        rc = call()
        assert rc == -1, (name, rc)
        assert L.voxcap_last_error(), name
    assert not h.value
    o = V.default_opts(entries="fp64")
    assert o.entries == V.ENTRIES["fp64"]
