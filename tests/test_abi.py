"""The C-ABI library loads and exports every function include/grt.h declares; the
Python structures match the C layouts (CPU only, no compute calls)."""
import ctypes
import os
import re

import pytest

import paper_2603_00292_gb300 as grt
from paper_2603_00292_gb300 import build as grt_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^grtError\s+(grt\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    grt_build.build()
    return grt.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    names = _declared()
    assert set(names) <= set(grt._SIGS), sorted(set(names) - set(grt._SIGS))
    for n in names:
        assert callable(getattr(grt, n, None)), n


def test_struct_layouts():
    assert ctypes.sizeof(grt.grtTriangleMeshPrimitive) == 32
    assert ctypes.sizeof(grt.grtAABBListPrimitive) == 16
    assert ctypes.sizeof(grt.grtGeometryBuildInput) == 8 + 32 + 16
    assert ctypes.sizeof(grt.grtSceneBuildInput) == 24
    assert ctypes.sizeof(grt.grtFuncDataSet) == 24
    assert ctypes.sizeof(grt.grtCamera) == 36
    assert ctypes.sizeof(grt.grtTraceOptions) == 48
    assert grt.RAY_BYTES == 32 and grt.HIT_BYTES == 20
    assert ctypes.sizeof(grt.grtBatchScene) == 8 + 56 + 8 + 8 + 8
    assert ctypes.sizeof(grt.grtBatchOptions) == 44
    assert ctypes.sizeof(grt.grtBatchInfo) == 32
    assert ctypes.sizeof(grt.grtBatchItemRecord) == 40
    assert ctypes.sizeof(grt.grtDeviceTarget) == 7 * 8 + 6 * 4
    assert ctypes.sizeof(grt.grtBvhInfo) == 3 * 8 + 4 * 4 + 3 * 8 + 2 * 4
    assert ctypes.sizeof(grt.grtBuildOptions) == 12
    assert ctypes.sizeof(grt.grtPathTraceInput) == 4 * 8 + 4 * 4 + 8 + 4 * 4


def test_host_only_queries_without_a_device(lib):
    # size/layout queries need no GPU
    k, v, b = grt.grtGetBuildTemporaryLayout(1000, 30)
    assert k % 256 == 0 and v % 256 == 0 and b % 256 == 0 and len({k, v, b}) == 3
    assert grt.grtSortTemporaryBufferSize(1 << 20, 64) > 8 * (1 << 20)
    with pytest.raises(grt.GrtError) as e:
        grt.grtSortTemporaryBufferSize(10, 16)
    assert e.value.code == grt.GRT_ERROR_INVALID_PARAMETER


def test_constants_match_the_header():
    """Every enumerator and numeric #define of include/grt.h that the binding exports has
    the header's value (the build flags, errors, primitive types, trace and batch flags)."""
    txt = open(os.path.join(ROOT, "include", "grt.h")).read()
    code = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    values = {}
    for body in re.findall(r"typedef\s+enum\s+\w*\s*\{(.*?)\}", code, flags=re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            if "=" in item:
                name, val = (x.strip() for x in item.split("=", 1))
                nxt = int(val, 0)
            else:
                name = item
            values[name] = nxt
            nxt += 1
    for name, val in re.findall(r"^#define\s+(GRT_\w+)\s+\(?([0-9xXa-fA-Fu<> ]+)\)?\s*$", code, flags=re.M):
        try:
            values[name] = int(eval(val.replace("u", "")))  # literals such as 1u or (1u << 3)
        except Exception:
            pass
    exported = {k: v for k, v in values.items() if hasattr(grt, k)}
    assert len(exported) >= 20, sorted(exported)
    wrong = {k: (getattr(grt, k), v) for k, v in exported.items() if getattr(grt, k) != v}
    assert not wrong, wrong
    for k in ("GRT_BUILD_PREFER_FAST", "GRT_BUILD_PREFER_BALANCED", "GRT_BUILD_PREFER_HIGH_QUALITY"):
        assert k in exported
