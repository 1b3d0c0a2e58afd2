"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every function include/hbpc.h declares, computes the basis like the oracle,
and rejects invalid arguments before touching the device."""
import os
import re

import numpy as np
import pytest

from oracle.basis import Basis, GAUSS, LOBATTO

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hbpc():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc as h
    return h


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hbpc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:hbpc_status|void|long long|int|const char\*)\s+(hbpc_\w+)\s*\(",
                                 text, re.M)))


def test_exports_every_declared_symbol(hbpc):
    import ctypes
    lib = ctypes.CDLL(hbpc.LIB_PATH)
    decl = declared_functions()
    assert len(decl) >= 18
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(hbpc.EXPORTED) == decl


@pytest.mark.parametrize("family,code", [(LOBATTO, 0), (GAUSS, 1)])
@pytest.mark.parametrize("N", range(1, 8))
def test_basis_matches_oracle(hbpc, N, family, code):
    b = hbpc.basis(N, code)
    o = Basis(N, family)
    np.testing.assert_allclose(b["nodes"], o.nodes, atol=2e-15)
    np.testing.assert_allclose(b["weights"], o.weights, rtol=1e-13)
    np.testing.assert_allclose(b["Dhat"], o.Dhat, atol=1e-12 * np.abs(o.Dhat).max())
    np.testing.assert_allclose(b["l_m"], o.l_m, atol=1e-13)
    np.testing.assert_allclose(b["l_p"], o.l_p, atol=1e-13)


@pytest.mark.parametrize("kw,code", [
    (dict(N=0), 1), (dict(N=8), 1), (dict(q=5), 1), (dict(dt=0.0), 1), (dict(dt=-1.0), 1),
    (dict(kmax=-1), 1), (dict(gmres_restart=0), 1), (dict(gmres_max_iter=0), 1),
    (dict(eps=0.0), 1), (dict(law=7), 1), (dict(nodes=3), 1), (dict(dim=4), 1),
    (dict(nu=-0.1), 1), (dict(nu=float("nan")), 1), (dict(nu=0.01, eta_br2=float("inf")), 1),
    (dict(nu=0.01, law=2), 7), (dict(law=3, nu=0.01, prandtl=float("nan")), 1),
    (dict(law=3, nu=0.01, gamma=1.0), 1), (dict(law=4), 1),
])
def test_invalid_arguments_rejected(hbpc, kw, code):
    args = dict(dim=2, n=(2, 2), lo=(0, 0), hi=(1, 1), N=3)
    args.update(kw)
    with pytest.raises(hbpc.HBPCError) as ei:
        hbpc.Context(**args)
    assert ei.value.status == code


@pytest.mark.parametrize("dim,N,nodes", [(1, 3, 0), (2, 1, 0), (2, 6, 0), (3, 6, 0), (2, 4, 1)])
def test_navier_stokes_outside_the_compiled_set_is_unsupported(hbpc, dim, N, nodes):
    """The Navier-Stokes kernels exist for dim 2 (N = 2-5 Lobatto, N = 2-3
    Gauss) and dim 3 (N = 2-5 Lobatto); anything else is HBPC_ERR_UNSUPPORTED
    before the device is touched."""
    n = (3,) * dim
    with pytest.raises(hbpc.HBPCError) as ei:
        hbpc.Context(dim, n, (0,) * dim, (1,) * dim, N, law=hbpc.LAW_NAVIER_STOKES, mu=0.01, nodes=nodes)
    assert ei.value.status == 7


def test_invalid_mesh_rejected(hbpc):
    with pytest.raises(hbpc.HBPCError):
        hbpc.Context(2, (0, 2), (0, 0), (1, 1), 3)
    with pytest.raises(hbpc.HBPCError):
        hbpc.Context(2, (2, 2), (0, 1), (1, 1), 3)


def test_batch_invalid_arguments_rejected(hbpc):
    """Batch creation checks its arguments before touching the device."""
    meshes = [((4, 4), (0, 0), (1, 1)), ((5, 3), (0, 0), (1, 1))]
    with pytest.raises(hbpc.HBPCError) as ei:          # a bad N in one instance
        hbpc.Batch(2, meshes, [3, 0], nus=[0.01, 0.02])
    assert ei.value.status == 1
    with pytest.raises(hbpc.HBPCError) as ei:          # negative viscosity
        hbpc.Batch(2, meshes, [3, 4], nus=[0.01, -0.02])
    assert ei.value.status == 1
    with pytest.raises(hbpc.HBPCError) as ei:          # the learned preconditioner
        hbpc.Batch(2, meshes, [3, 4], nus=[0.01, 0.02], pc=hbpc.PC_LEARNED)
    assert ei.value.status == 7
    with pytest.raises(hbpc.HBPCError) as ei:          # Navier-Stokes batches
        hbpc.Batch(2, meshes, [3, 4], nus=[0.01, 0.02], law=hbpc.LAW_NAVIER_STOKES)
    assert ei.value.status == 7


def test_non_periodic_mesh_is_unsupported(hbpc):
    """Only periodic meshes are implemented: periodic = 0 is
    HBPC_ERR_UNSUPPORTED and any other value HBPC_ERR_INVALID_ARG, both before
    the device is touched."""
    with pytest.raises(hbpc.HBPCError) as ei:
        hbpc.Context(2, (2, 2), (0, 0), (1, 1), 3, periodic=0)
    assert ei.value.status == 7
    with pytest.raises(hbpc.HBPCError) as ei:
        hbpc.Context(2, (2, 2), (0, 0), (1, 1), 3, periodic=2)
    assert ei.value.status == 1


@pytest.mark.parametrize("t_end", [-1.0, float("nan"), float("inf")])
def test_invalid_final_time_rejected(hbpc, t_end):
    with pytest.raises(hbpc.HBPCError) as ei:
        hbpc.Context(2, (2, 2), (0, 0), (1, 1), 3, t_end=t_end)
    assert ei.value.status == 1


def test_noalloc_rejects_overlapping_output(hbpc):
    """The allocation-free Jv reads X and dX while it writes out: an out that
    overlaps either is rejected before anything is launched (addresses only;
    no device memory is touched)."""
    import ctypes

    class FakeTensor:    # a device pointer the check compares but never dereferences
        def __init__(self, addr):
            self.addr = addr

        def is_contiguous(self):
            return True

        dtype = "torch.float64"

        def data_ptr(self):
            return self.addr

    n2 = 2 * 4 * 4 * 16         # 2 n_dof of a 4 x 4 mesh at N = 3
    base = 1 << 40
    X, dX = FakeTensor(base), FakeTensor(base + 8 * n2)
    for out in (FakeTensor(base), FakeTensor(base + 8 * n2 + 8), FakeTensor(base + 8 * (n2 - 1))):
        with pytest.raises(hbpc.HBPCError) as ei:
            hbpc.eval_Jv_noalloc(2, (4, 4), (0, 0), (1, 1), 3, 0.01, 0.5, 0.1, X, dX, out)
        assert ei.value.status == 1
        assert "overlap" in str(ei.value)
    assert ctypes.sizeof(hbpc.Mesh) == 4 + 12 + 48 + 4 + 4    # periodic field, padded to 8


def test_noalloc_rejects_viscous_law_on_the_host(hbpc):
    class FakeTensor:
        dtype = "torch.float64"

        def __init__(self, addr):
            self.addr = addr

        def is_contiguous(self):
            return True

        def data_ptr(self):
            return self.addr

    X, dX, out = FakeTensor(1 << 40), FakeTensor(1 << 41), FakeTensor(1 << 42)
    with pytest.raises(hbpc.HBPCError) as ei:
        hbpc.eval_Jv_noalloc(2, (4, 4), (0, 0), (1, 1), 3, 0.01, 0.5, 0.1, X, dX, out, nu=0.01)
    assert ei.value.status == 7


def test_bjext_h_preconditioner_checks(hbpc):
    """BJ^H_ext has no Navier-Stokes Hessian blocks (HBPC_ERR_UNSUPPORTED) and an
    unknown preconditioner code is HBPC_ERR_INVALID_ARG, both before the device
    is touched."""
    with pytest.raises(hbpc.HBPCError) as ei:
        hbpc.Context(2, (3, 3), (0, 0), (1, 1), 3, law=hbpc.LAW_NAVIER_STOKES, mu=0.01, pc=hbpc.PC_BJEXT_H)
    assert ei.value.status == 7
    with pytest.raises(hbpc.HBPCError) as ei:
        hbpc.Context(2, (3, 3), (0, 0), (1, 1), 3, pc=4)
    assert ei.value.status == 1


def test_binding_structs_match_the_header(hbpc, tmp_path):
    """The ctypes structures of the binding have the C compiler's layout of the
    header's structs: size and the offset of every field, in order (a field
    added on one side only would shift every later one)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = {"hbpc_mesh": hbpc.Mesh, "hbpc_physics": hbpc.Physics, "hbpc_solver": hbpc.Solver,
             "hbpc_stats": hbpc.Stats, "hbpc_tuning": hbpc.Tuning}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "hbpc.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                              text=True).stdout.splitlines())
    for cname, cls in pairs.items():
        assert int(out["%s size" % cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(out["%s.%s" % (cname, fname)]) == getattr(cls, fname).offset, (cname, fname)
