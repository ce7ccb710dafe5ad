"""The C-ABI library loads and exports every symbol include/pint.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pint.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pint_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = _declared()
    for must in ("pint_create", "pint_operator_assemble", "pint_set_coupling",
                 "pint_apply_coupled", "pint_solve_block", "pint_newton_step", "pint_shift",
                 "pint_pipeline_run", "pint_coupling_from_dirk"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    lib_path = __graft_entry__._build_module().build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    import paper_2504_02117_gb300 as P
    missing = [n for n in _declared() if not hasattr(P, n)]
    assert not missing, missing


def test_host_only_calls_without_gpu():
    """Calls that touch no device: defaults, the DIRK coupling builder (theta
    example of Sec. 2.1 after elimination) and argument validation."""
    import numpy as np
    import paper_2504_02117_gb300 as P
    o = P.pint_opts_default()
    assert o.restart == 30 and o.tol == 1e-10
    th, tau = 0.3, 0.25
    A = np.array([[0.0, 0.0], [1 - th, th]])
    A1, A2, e = P.pint_coupling_from_dirk(A, 4, tau, eliminate_first=True)
    np.testing.assert_allclose(A1, (np.eye(4) - np.eye(4, k=-1)) / tau)
    np.testing.assert_allclose(A2, th * np.eye(4) + (1 - th) * np.eye(4, k=-1))
    np.testing.assert_allclose(e, [1 - th])
    with pytest.raises(P.PintError):
        P.pint_coupling_from_dirk(np.array([[1.0, 0.0], [0.5, 0.5]]), 2, tau, eliminate_first=True)
    with pytest.raises(P.PintError):
        P.pint_coupling_from_dirk(np.eye(3), 6, tau)        # 18 > 16 columns
    assert P.lib.pint_shift(None, 10, 2, None) == P.PINT_ERR_INVALID


def test_dirk_builder_matches_oracle():
    import numpy as np
    import paper_2504_02117_gb300 as P
    from oracle import coupling
    for tab in (coupling.implicit_euler(), coupling.sdirk2()):
        for steps in (1, 3):
            A1, A2, _ = P.pint_coupling_from_dirk(tab[0], steps, 0.1)
            R1, R2, _ = coupling.multistep_matrices(tab[0], steps, 0.1)
            np.testing.assert_array_equal(A1, R1)
            np.testing.assert_array_equal(A2, R2)


def test_vg_lipschitz_host_call_matches_oracle():
    """pint_vg_lipschitz (closed form) against the oracle's numerical
    supremum of theta', including the paper's silt loam (L = 4.501e-2)."""
    import paper_2504_02117_gb300 as P
    from oracle import fv
    for prm in [(1.0, 2.0, 0.05, 0.4), (0.423, 2.06, 0.131, 0.396), (3.0, 1.4, 0.0, 0.5)]:
        L = P.pint_vg_lipschitz(prm)
        assert abs(L - fv.VanGenuchten(*prm).lipschitz()) <= 1e-12 * L
    with pytest.raises(P.PintError):
        P.pint_vg_lipschitz((1.0, 1.0, 0.05, 0.4))


def test_struct_layout_matches_the_header(tmp_path):
    """pint_opts and pint_stats as the binding declares them have the C
    compiler's sizes and field offsets (a C program compiled against
    include/pint.h prints them)."""
    import shutil
    import subprocess
    import paper_2504_02117_gb300 as P
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = {"pint_opts": [f[0] for f in P.pint_opts._fields_],
              "pint_stats": [f[0] for f in P.pint_stats._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pint.h"', "int main(void) {"]
    for st, names in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for n in names:
            lines.append(f'  printf("{st} {n} %zu\\n", offsetof({st}, {n}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}
    for st, cls in (("pint_opts", P.pint_opts), ("pint_stats", P.pint_stats)):
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for n in fields[st]:
            assert got[(st, n)] == getattr(cls, n).offset, (st, n)


def test_plain_c_client_compiles_and_links(tmp_path):
    """The boundary is usable from C alone: tests/c/slab_client.c (a slab
    solve through the C ABI, device buffers from the CUDA runtime) compiles
    with a C compiler against include/pint.h and links against libpint.so."""
    import shutil
    import subprocess
    import __graft_entry__
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if cc is None or not os.path.isdir(os.path.join(cuda, "include")):
        pytest.skip("no C compiler or CUDA toolkit")
    lib_path = __graft_entry__._build_module().build()
    libdir = os.path.dirname(lib_path)
    cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                    if os.path.isdir(d)), None)
    if cudalib is None:
        pytest.skip("no CUDA runtime library directory")
    exe = tmp_path / "slab_client"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(cuda, "include"),
                        os.path.join(ROOT, "tests", "c", "slab_client.c"), "-o", str(exe),
                        "-L", libdir, "-lpint", "-L", cudalib, "-lcudart", "-lm",
                        f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert exe.exists()
