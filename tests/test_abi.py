"""The C ABI library builds for sm_103a, loads, exports every entry point the
header declares, and the Python binding's struct layouts match the header.
No compute call is made (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2602_10761_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(tribo_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return C.CDLL(build.LIB)


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(_abi.exported_names()) | set()


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "tribo.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("tribo_grid %zu\n", sizeof(tribo_grid));
  printf("tribo_params %zu\n", sizeof(tribo_params));
  printf("tribo_fluid %zu\n", sizeof(tribo_fluid));
  printf("tribo_particles %zu\n", sizeof(tribo_particles));
  printf("tribo_modes %zu\n", sizeof(tribo_modes));
  printf("tribo_ssm %zu\n", sizeof(tribo_ssm));
  P(tribo_grid, lx) P(tribo_grid, y_faces)
  P(tribo_params, kappa_A) P(tribo_params, drag_law) P(tribo_params, sort_every) P(tribo_params, coulomb) P(tribo_params, collisions)
  P(tribo_particles, x) P(tribo_particles, q) P(tribo_particles, cell) P(tribo_particles, on_host)
  P(tribo_modes, nxi) P(tribo_modes, damp) P(tribo_modes, t0)
  P(tribo_ssm, c_sat) P(tribo_ssm, seed)
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.split("\n") if l)
    assert int(out["tribo_grid"]) == C.sizeof(_abi.tribo_grid)
    assert int(out["tribo_params"]) == C.sizeof(_abi.tribo_params)
    assert int(out["tribo_fluid"]) == C.sizeof(_abi.tribo_fluid)
    assert int(out["tribo_particles"]) == C.sizeof(_abi.tribo_particles)
    assert int(out["tribo_modes"]) == C.sizeof(_abi.tribo_modes)
    assert int(out["tribo_ssm"]) == C.sizeof(_abi.tribo_ssm)
    for key, val in out.items():
        if "." in key:
            st, f = key.split(".")
            assert getattr(getattr(_abi, st), f).offset == int(val), key


def test_error_strings(lib):
    lib.tribo_strerror.restype = C.c_char_p
    for s in range(7):
        assert lib.tribo_strerror(s)
    lib.tribo_init.restype = C.c_int32
    # a NULL output pointer is an argument error, reported without touching a GPU
    assert lib.tribo_init(None, None, None, None, C.c_int64(0), None) == _abi.TRIBO_ERR_ARG


def test_ssm_defaults_are_the_reference_impact_of_sec_3_1():
    """The binding's SSM defaults equal the oracle's (both restate Sec. 3.1)."""
    import dataclasses

    import paper_2602_10761_gb300 as T
    from oracle.ssm import SSM
    assert dataclasses.asdict(T.SSMParams()) == dataclasses.asdict(SSM())


def test_noalloc_binding_rejects_bad_arrays_before_the_call():
    """tribo_poisson_noalloc's binding checks dtype, shape, device and the
    face count before anything reaches the C side (which sees raw pointers)."""
    torch = pytest.importorskip("torch")
    import numpy as np
    from paper_2602_10761_gb300 import api
    nx, ny, nz = 8, 6, 4
    faces = np.linspace(0.0, 0.04, ny + 1)
    rho = torch.zeros((nz, ny, nx), dtype=torch.float64)
    E = torch.zeros((3, nz, ny + 2, nx), dtype=torch.float32)
    cases = [
        dict(y_faces=faces[:-1]),                                   # ny faces instead of ny + 1
        dict(rho=rho),                                              # host tensor
        dict(rho=rho.float()),                                      # wrong dtype
        dict(E=E[:, :, 1:-1]),                                      # no wall rows
        dict(E=E.double()),                                         # FP64 E in mixed mode
        dict(phi=torch.zeros((nz, ny, nx), dtype=torch.float32)),   # phi not FP64
        dict(rho=np.zeros((nz, ny, nx))),                           # not a tensor
    ]
    for kw in cases:
        args = dict(y_faces=faces, rho=rho, phi=None, E=E)
        args.update(kw)
        with pytest.raises(ValueError):
            api._check_noalloc_args(nx, ny, nz, args["y_faces"], _abi.TRIBO_MIXED, args["rho"], args["phi"],
                                    args["E"])
