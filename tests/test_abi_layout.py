"""The ctypes structures of the Python binding against the C header: every
structure's size and every field's offset as a C compiler lays them out.
A mismatch would pass wrong values through the boundary without an error."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2606_31764_b300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {
    "ns_curves": B.NsCurves,
    "ns_sample_params": B.NsSampleParams,
    "ns_raster_params": B.NsRasterParams,
    "ns_capacity": B.NsCapacity,
    "ns_gaussians": B.NsGaussians,
    "ns_curve_grads": B.NsCurveGrads,
    "ns_report": B.NsReport,
    "ns_geometry_params": B.NsGeometryParams,
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_ctypes_structures_match_the_header():
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nurbs_splat.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "layout.c")
        exe = os.path.join(tmp, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    seen = {}
    for line in out.splitlines():
        cname, what, value = line.split()
        seen[(cname, what)] = int(value)
    for cname, cls in STRUCTS.items():
        assert seen[(cname, "size")] == C.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert seen[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
