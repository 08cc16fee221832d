"""The C ABI: the library builds, loads and exports every function include/hpac.h
declares, and the binding's ctypes structures match the header's layout
(checked by compiling a probe against the header with gcc). No GPU needed."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hpac.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(hpac_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("hpac_region_create", "hpac_region_destroy", "hpac_run_exact", "hpac_run_perfo",
              "hpac_run_taf", "hpac_run_iact", "hpac_quality", "hpac_last_error"):
        assert f in names


def test_library_exports_every_declared_symbol():
    from paper_2308_16877_gb300 import build, hpac
    build.build()
    lib = C.CDLL(build.LIB)
    for f in declared_functions():
        assert hasattr(lib, f), f
        assert f in hpac.SIGNATURES, f
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (hpac_\w+)", out))
    assert set(declared_functions()) <= exported


def test_no_compute_symbol_without_gpu_is_called_here():
    # only metadata calls: version and last_error work without a device
    from paper_2308_16877_gb300 import hpac
    assert "sm_103a" in hpac.hpac_version()
    assert isinstance(hpac.hpac_last_error(), str)


def test_struct_layouts_match_header(tmp_path):
    from paper_2308_16877_gb300 import hpac
    probe = tmp_path / "probe.c"
    structs = ["hpac_region_desc", "hpac_perfo_knobs", "hpac_taf_knobs", "hpac_iact_knobs",
               "hpac_stats", "hpac_quality_result", "hpac_hydro_state", "hpac_sweep_config",
               "hpac_sweep_region", "hpac_sweep_stats", "hpac_mlp_desc", "hpac_lavamd_desc"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hpac.h"', "int main(void){"]
    for s in structs:
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for fname, _ in getattr(hpac, s)._fields_:
            lines.append(f'printf("{s}.{fname} %zu\\n", offsetof({s}, {fname}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n") if l)
    for s in structs:
        cls = getattr(hpac, s)
        assert int(got[s]) == C.sizeof(cls), s
        for fname, _ in cls._fields_:
            assert int(got[f"{s}.{fname}"]) == getattr(cls, fname).offset, (s, fname)


def test_enum_values_match_header():
    from paper_2308_16877_gb300 import hpac
    src = open(HEADER).read()
    for name in ("HPAC_OK", "HPAC_EINVAL", "HPAC_EUNSUPPORTED", "HPAC_F64", "HPAC_LEVEL_BLOCK",
                 "HPAC_REGION_IDENTITY", "HPAC_REGION_BINOMIAL", "HPAC_PERFO_RANDOM", "HPAC_MASK_SKIPPED", "HPAC_METRIC_MCR"):
        m = re.search(rf"\b{name}\s*=\s*(\d+)", src)
        assert m and int(m.group(1)) == getattr(hpac, name), name


def test_invalid_arguments_are_rejected_before_any_device_work():
    """NULL handles and out-of-range arguments return HPAC_EINVAL with a
    message, without a device (every check precedes the first CUDA call)."""
    from paper_2308_16877_gb300 import hpac
    L = hpac.load()
    EINVAL = hpac.HPAC_EINVAL
    calls = [
        ("hpac_run_exact", (None, None, None)),
        ("hpac_region_adjoint", (None, None, None)),
        ("hpac_region_vjp", (None, None, None, None)),
        ("hpac_mlp_vjp", (None, 10, None, 10, 0.0, None, None, None)),
        ("hpac_mlp_set_params_device", (None, None)),
        ("hpac_mlp_input_grad", (None, 10, None, 10, 0.0, None)),
        ("hpac_kmeans_update", (10, 0, None, 10, None, None, None, None, None, None)),
        ("hpac_hydro_step", (None, None, 0, None, None, None)),
    ]
    for name, args in calls:
        status = getattr(L, name)(*args)
        assert status == EINVAL, (name, status)
        assert hpac.hpac_last_error(), name
    # destroying NULL is a no-op, as free(NULL)
    assert L.hpac_region_destroy(None) == hpac.HPAC_OK
    # LavaMD: descriptor, technique, knobs and pointers are checked first; an
    # empty grid is a no-op
    D = hpac.hpac_lavamd_desc
    taf = hpac.hpac_taf_knobs(4, 8, 0.01, 0, 0)
    bad_taf = hpac.hpac_taf_knobs(0, 8, 0.01, 0, 0)
    bad_iact = hpac.hpac_iact_knobs(8, 3, 0.01, 0, 0, None)
    lavamd_calls = [
        (None, 0, None, None, None),
        (C.byref(D(2, 0, 0.5)), 0, None, None, None),
        (C.byref(D(2, 1025, 0.5)), 0, None, None, None),
        (C.byref(D(2, 4, -1.0)), 0, None, None, None),
        (C.byref(D(2, 4, 0.5)), 3, None, None, None),
        (C.byref(D(2, 4, 0.5)), 1, None, None, None),
        (C.byref(D(2, 4, 0.5)), 1, C.byref(bad_taf), None, None),
        (C.byref(D(2, 4, 0.5)), 2, C.byref(bad_iact), None, None),
        (C.byref(D(2, 4, 0.5)), 1, C.byref(taf), None, None),       # NULL arrays
        (C.byref(D(2, 4, 0.5)), 0, None, 8 + 4, 16),                 # misaligned
    ]
    for desc, tech, kn, rq, fv in lavamd_calls:
        status = L.hpac_lavamd_run(desc, tech, kn, rq, fv, None, None, None)
        assert status == EINVAL, (tech, status)
    st = hpac.hpac_stats(7, 7, 7, 7)
    assert L.hpac_lavamd_run(C.byref(D(0, 4, 0.5)), 0, None, None, None, None, C.byref(st), None) == hpac.HPAC_OK
    assert (st.invocations, st.approximated) == (0, 0)


def test_lavamd_binding_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    from paper_2308_16877_gb300 import hpac
    with pytest.raises(ValueError):
        hpac.lavamd(torch.zeros(4, 8, dtype=torch.float64), 1, 8)
    with pytest.raises(ValueError):
        hpac.lavamd(torch.zeros(4, 9, dtype=torch.float64), 1, 8)
