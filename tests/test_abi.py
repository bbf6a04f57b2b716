"""The C-ABI library loads and exports every entry point that
include/lbfsi.h declares; the ctypes structures match the C layouts; invalid
arguments are rejected before any CUDA call (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbfsi.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2107_01370_gb300 import build, lbfsi
    if not os.path.exists(lbfsi.LIB_PATH):
        build.build()
    return lbfsi.load()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbfsi_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbfsi_create_mesh", "lbfsi_blend_mesh", "lbfsi_init_fields", "lbfsi_step",
                     "lbfsi_body_forces", "lbfsi_advance_bodies"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True)
    exported = set(re.findall(r" T (lbfsi_\w+)", out.stdout))
    assert set(declared_functions()) <= exported


def test_binding_lists_every_declared_symbol():
    from paper_2107_01370_gb300 import lbfsi
    assert set(declared_functions()) == set(lbfsi.EXPORTED)


def test_struct_layouts_match_c(tmp_path):
    from paper_2107_01370_gb300 import lbfsi
    src = tmp_path / "sz.c"
    src.write_text('#include "lbfsi.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(lbfsi_body_desc),'
                   'sizeof(lbfsi_flow_params), sizeof(lbfsi_mesh_desc), sizeof(lbfsi_body_state),'
                   'offsetof(lbfsi_mesh_desc, bodies), offsetof(lbfsi_body_desc, wh_wa));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(lbfsi.BodyDesc), ctypes.sizeof(lbfsi.FlowParams),
                   ctypes.sizeof(lbfsi.MeshDesc), ctypes.sizeof(lbfsi.BodyState),
                   lbfsi.MeshDesc.bodies.offset, lbfsi.BodyDesc.wh_wa.offset]


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_2107_01370_gb300 import lbfsi
    h = ctypes.c_void_p()
    assert lib.lbfsi_create_mesh(None, None, ctypes.byref(h)) == lbfsi.EINVAL
    assert b"null" in lib.lbfsi_last_error()
    r = (ctypes.c_double * 8)(*range(1, 9))
    e = (ctypes.c_double * 14)()
    body = lbfsi.BodyDesc()
    d = lbfsi.MeshDesc(8, 7, r, e, 0.0, 0.0, 0, 1, ctypes.pointer(body))   # odd ntheta
    assert lib.lbfsi_create_mesh(ctypes.byref(d), None, ctypes.byref(h)) == lbfsi.EINVAL
    assert b"ntheta" in lib.lbfsi_last_error()
    d = lbfsi.MeshDesc(8, 8, r, e, 0.0, 0.0, 5, 1, ctypes.pointer(body))   # bad precision
    assert lib.lbfsi_create_mesh(ctypes.byref(d), None, ctypes.byref(h)) == lbfsi.EINVAL
    # the largest handle: 9 N nbatch population slots must stay within 2^31
    # (checked before the tables are read or the device is touched)
    big = (ctypes.c_double * (1 << 16))()
    d = lbfsi.MeshDesc(1 << 14, 1 << 14, big, big, 0.0, 0.0, 0, 1, ctypes.pointer(body))
    assert lib.lbfsi_create_mesh(ctypes.byref(d), None, ctypes.byref(h)) == lbfsi.EINVAL
    assert b"too large" in lib.lbfsi_last_error()
    bodies = (lbfsi.BodyDesc * 2000)()
    d = lbfsi.MeshDesc(512, 256, big, big, 0.0, 0.0, 0, 2000, bodies)     # 2000 solves of 131072 nodes
    assert lib.lbfsi_create_mesh(ctypes.byref(d), None, ctypes.byref(h)) == lbfsi.EINVAL
    assert b"too large" in lib.lbfsi_last_error()
    assert lib.lbfsi_step(None, 1) == lbfsi.EINVAL
    assert lib.lbfsi_launch_count(None) == -1
    ptr = ctypes.c_void_p()
    assert lib.lbfsi_field_ptr(None, lbfsi.FIELD_MOMENTS, ctypes.byref(ptr), None, None) == lbfsi.EINVAL


def test_xy_mesh_struct_layout_matches_c(tmp_path):
    from paper_2107_01370_gb300 import lbfsi
    src = tmp_path / "xy.c"
    src.write_text('#include "lbfsi.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(lbfsi_mesh_xy_desc),'
                   'offsetof(lbfsi_mesh_xy_desc, X), offsetof(lbfsi_mesh_xy_desc, bodies),'
                   'sizeof(lbfsi_solve_xy_desc), offsetof(lbfsi_solve_xy_desc, steps));return 0;}\n')
    exe = tmp_path / "xy"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(lbfsi.MeshXYDesc), lbfsi.MeshXYDesc.X.offset,
                   lbfsi.MeshXYDesc.bodies.offset, ctypes.sizeof(lbfsi.SolveXYDesc),
                   lbfsi.SolveXYDesc.steps.offset]


def test_general_mesh_validation_without_gpu(lib):
    """lbfsi_create_mesh_xy rejects, before touching the device, a mesh whose
    nodes are not subparametric and one that is not positively oriented."""
    import numpy as np
    from paper_2107_01370_gb300 import inputs, lbfsi
    wall = inputs.ellipse_wall(16, 0.6, 0.4)
    X = inputs.algebraic_ogrid(wall, 9, 4.0, 0.05)
    body = lbfsi.BodyDesc()
    h = ctypes.c_void_p()

    def create(Xa):
        Xa = np.ascontiguousarray(Xa)
        d = lbfsi.MeshXYDesc(Xa.shape[0], Xa.shape[1], Xa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             0.0, 0.0, 0, 1, ctypes.pointer(body))
        return lib.lbfsi_create_mesh_xy(ctypes.byref(d), None, ctypes.byref(h))

    bad = X.copy()
    bad[3, 5] += 1e-3                      # an odd node off its bilinear position
    assert create(bad) == lbfsi.EINVAL
    assert b"subparametric" in lib.lbfsi_last_error()
    assert create(np.roll(X[:, ::-1], 1, axis=1)) == lbfsi.EINVAL   # clockwise: j -> -j
    assert b"oriented" in lib.lbfsi_last_error()
    nan = X.copy()
    nan[0, 0, 0] = np.nan
    assert create(nan) == lbfsi.EINVAL


def test_cgrid_struct_layout_and_validation_without_gpu(tmp_path, lib):
    """lbfsi_mesh_cgrid_desc matches the binding; lbfsi_create_mesh_cgrid
    rejects, before touching the device, cut nodes that do not coincide, an
    even node count along the C, an odd or too long cut, and a mesh that is
    not subparametric."""
    import numpy as np
    from paper_2107_01370_gb300 import inputs, lbfsi
    src = tmp_path / "cg.c"
    src.write_text('#include "lbfsi.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(lbfsi_mesh_cgrid_desc),'
                   'offsetof(lbfsi_mesh_cgrid_desc, X), offsetof(lbfsi_mesh_cgrid_desc, xc),'
                   'offsetof(lbfsi_mesh_cgrid_desc, bodies), sizeof(lbfsi_solve_cgrid_desc),'
                   'offsetof(lbfsi_solve_cgrid_desc, steps));return 0;}\n')
    exe = tmp_path / "cg"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(lbfsi.MeshCGridDesc), lbfsi.MeshCGridDesc.X.offset,
                   lbfsi.MeshCGridDesc.xc.offset, lbfsi.MeshCGridDesc.bodies.offset,
                   ctypes.sizeof(lbfsi.SolveCGridDesc), lbfsi.SolveCGridDesc.steps.offset]
    X = inputs.cgrid_ellipse(17, 4, 9, 0.6, 0.35, r_far=4.0, wake=3.0)
    body = lbfsi.BodyDesc()
    h = ctypes.c_void_p()

    def create(Xa, n_cut):
        Xa = np.ascontiguousarray(Xa)
        d = lbfsi.MeshCGridDesc(Xa.shape[0], Xa.shape[1], n_cut,
                                Xa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0.0, 0.0, 0, 1,
                                ctypes.pointer(body))
        return lib.lbfsi_create_mesh_cgrid(ctypes.byref(d), None, ctypes.byref(h))

    bad = X.copy()
    bad[0, 1, 1] += 1e-3                   # an upper cut node off the lower one
    assert create(bad, 4) == lbfsi.EINVAL
    assert b"coincide" in lib.lbfsi_last_error()
    assert create(X[:, :-1], 4) == lbfsi.EINVAL
    assert create(X, 3) == lbfsi.EINVAL
    assert create(X, 8) == lbfsi.EINVAL     # leaves no wall
    bad = X.copy()
    bad[3, 9] += 1e-3
    assert create(bad, 4) == lbfsi.EINVAL
    assert b"subparametric" in lib.lbfsi_last_error()


def test_box_struct_layout_and_validation_without_gpu(tmp_path, lib):
    """lbfsi_mesh_box_desc matches the binding; lbfsi_create_mesh_box rejects,
    before touching the device, odd sizes, a moving body and a box that is not
    positively oriented."""
    import numpy as np
    from paper_2107_01370_gb300 import inputs, lbfsi
    src = tmp_path / "bx.c"
    src.write_text('#include "lbfsi.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(lbfsi_mesh_box_desc),'
                   'offsetof(lbfsi_mesh_box_desc, shift_i), offsetof(lbfsi_mesh_box_desc, precision),'
                   'offsetof(lbfsi_mesh_box_desc, bodies));return 0;}\n')
    exe = tmp_path / "bx"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(lbfsi.MeshBoxDesc), lbfsi.MeshBoxDesc.shift_i.offset,
                   lbfsi.MeshBoxDesc.precision.offset, lbfsi.MeshBoxDesc.bodies.offset]
    h = ctypes.c_void_p()

    def create(X, si, sj, dof=0):
        X = np.ascontiguousarray(X)
        body = lbfsi.BodyDesc()
        body.dof = dof
        body.r_in, body.r_out, body.length, body.m_star, body.v_r = 1.0, 2.0, 1.0, 1.0, 1.0
        d = lbfsi.MeshBoxDesc(X.shape[0], X.shape[1], X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              (ctypes.c_double * 2)(*si), (ctypes.c_double * 2)(*sj), 0, 1, ctypes.pointer(body))
        return lib.lbfsi_create_mesh_box(ctypes.byref(d), None, ctypes.byref(h))

    X, si, sj = inputs.box_mesh(8, 6, 8.0, 6.0, skew=0.2)
    assert create(X[:7], si, sj) == lbfsi.EINVAL                       # odd ni
    assert create(X, si, sj, dof=1) == lbfsi.EINVAL
    assert b"fixed" in lib.lbfsi_last_error()
    assert create(X, si, (0.0, -6.0)) == lbfsi.EINVAL                   # period against the node order


def test_cgrid_walls_struct_layout_and_independent_bodies_validation_without_gpu(tmp_path, lib):
    """lbfsi_mesh_cgrid_walls_desc matches the binding (nbody and wall_body
    appended); lbfsi_create_mesh_cgrid_walls rejects, before touching the
    device, a chain body out of range, a body without a chain, mirrored
    chains on different bodies, another body's wall inside a moving body's
    blended region and overlapping blended regions of two moving bodies."""
    from paper_2107_01370_gb300 import inputs, lbfsi
    src = tmp_path / "cw.c"
    src.write_text('#include "lbfsi.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(lbfsi_mesh_cgrid_walls_desc),'
                   'offsetof(lbfsi_mesh_cgrid_walls_desc, bodies), offsetof(lbfsi_mesh_cgrid_walls_desc, nbody),'
                   'offsetof(lbfsi_mesh_cgrid_walls_desc, wall_body));return 0;}\n')
    exe = tmp_path / "cw"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    D = lbfsi.MeshCGridWallsDesc
    assert got == [ctypes.sizeof(D), D.bodies.offset, D.nbody.offset, D.wall_body.offset]
    X, walls = inputs.tandem_cgrid(34, 17, 11, 16, 17)
    front = inputs.BodySpec(dof=1, xc=0.0, r_in=0.7, r_out=1.8)
    rear = inputs.BodySpec(dof=1, xc=4.0, r_in=0.7, r_out=1.8)

    def create(bodies, wall_body):
        try:
            lbfsi.Mesh.cgrid_walls(X, walls, bodies, wall_body=wall_body)
        except lbfsi.LbfsiError as e:
            return e.code, str(e)
        raise AssertionError("accepted")

    assert create([[front, rear]], [1, 0, 2])[0] == lbfsi.EINVAL
    assert create([[front, rear, rear]], [1, 0, 1])[0] == lbfsi.EINVAL     # body 2 owns no chain
    assert "symmetric" in create([[front, rear]], [1, 0, 0])[1]
    wide = inputs.BodySpec(dof=1, xc=0.0, r_in=0.7, r_out=3.6)
    assert "blended region" in create([[wide, inputs.BodySpec(dof=0)]], [1, 0, 1])[1]
    near = inputs.BodySpec(dof=1, xc=4.0, r_in=0.7, r_out=2.3)
    assert "overlap" in create([[inputs.BodySpec(dof=1, xc=0.0, r_in=0.7, r_out=1.9), near]], [1, 0, 1])[1]
    assert create([[rear, front]], [1, 0, 1])[0] == lbfsi.EINVAL               # bodies swapped
    small_front = inputs.BodySpec(dof=1, xc=0.0, r_in=0.45, r_out=1.8)
    assert "rigid zone" in create([[small_front, inputs.BodySpec(dof=0)]], [1, 0, 1])[1]


def test_element_mesh_layout_and_validation_without_a_gpu(lib, tmp_path):
    """The element-list descriptor matches its C layout, and a bad element
    list is refused before any CUDA call: an out-of-range node, a node in no
    element, an element whose mid nodes are off the bilinear positions, a
    chain of odd length, a node on both chains."""
    import numpy as np
    from paper_2107_01370_gb300 import inputs, lbfsi
    src = tmp_path / "el.c"
    src.write_text('#include "lbfsi.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu\\n", sizeof(lbfsi_mesh_elements_desc),'
                   'offsetof(lbfsi_mesh_elements_desc, bodies), offsetof(lbfsi_mesh_elements_desc, grid_ij));'
                   'return 0;}\n')
    exe = tmp_path / "el"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(lbfsi.MeshElementsDesc), lbfsi.MeshElementsDesc.bodies.offset,
                   lbfsi.MeshElementsDesc.grid_ij.offset]
    case = inputs.cylinder_case(9, 16, r_far=6.0)
    X = np.stack([case.r[:, None] * case.e[None, :, 0], case.r[:, None] * case.e[None, :, 1]], axis=-1)
    el = inputs.ogrid_element_list(X, seed=2)

    def make(X=el.X, E=el.elements, wall=el.wall, far=el.far):
        with pytest.raises(lbfsi.LbfsiError) as ei:
            lbfsi.ElementMesh(X, E, wall, far, case.bodies, precision=lbfsi.FP64)
        return ei.value.code, str(ei.value)

    E = el.elements.copy()
    E[0, 0, 0] = el.X.shape[0]
    assert make(E=E)[0] == lbfsi.EINVAL
    X2 = np.vstack([el.X, [[30.0, 30.0]]])
    code, msg = make(X=X2)
    assert code == lbfsi.EINVAL and "every node" in msg
    X3 = el.X.copy()
    X3[el.elements[3, 1, 1]] += 0.01
    code, msg = make(X=X3)
    assert code == lbfsi.EINVAL and "subparametric" in msg
    assert make(wall=el.wall[:-1])[0] == lbfsi.EINVAL
    far = el.far.copy()
    far[0] = el.wall[0]
    assert make(far=far)[0] == lbfsi.EINVAL
