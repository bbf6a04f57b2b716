"""The bounds-checked build (LBFSI_BOUNDS_CHECK, liblbfsi_bounds.so): every
shared-memory window the step reads and every global slot it writes
(second copies, mirrored rows) is checked, and a violation would be reported
as LBFSI_EBOUNDS with the access skipped — the substitute for a memory
checker on this GPU.  Every mesh kind and launch form runs clean: separable
O-grids (FP32 in the bench's tile shape, FP64), an O-grid given by
coordinates, a NACA 0012 C-grid, linked tandem cylinders, a periodic box,
the collide-only launch, and a batch mixing separable, general and C-grid
solves.  Run in a child process, which loads the checked library instead of
the normal one."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2107_01370_gb300 import build, inputs, lbfsi as L
L.load(build.LIB_BOUNDS)

def run(m, flow, M0, steps=6, post=False):
    m.init_fields(flow, np.ascontiguousarray(M0))
    m.step(steps)
    m.synchronize()
    if post:
        m.get_populations(1)
    m.close()

body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=3.0, v_r=4.0)
case = inputs.cylinder_case(40, 64, r_far=8.0, body=body)
M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=1)
for prec in (L.FP32, L.FP64):
    run(L.Mesh(case.r, case.e, case.bodies * 2, precision=prec), case.flow, np.stack([M0, M0]), post=True)
ell = inputs.xy_case(inputs.ellipse_wall(64, 0.6, 0.35), 40, r_far=8.0, length=1.2, body=body)
run(L.Mesh.xy(ell.X, ell.bodies, precision=L.FP32), ell.flow,
    inputs.initial_field(ell.nr, ell.ntheta, ell.flow, seed=2)[None])
nb = inputs.BodySpec(dof=2, xp=-1.0, r_in=0.6, r_out=2.0, m_star=100.0, v_r=0.5025, x_alpha=1.8,
                     r_alpha=1.87, wh_wa=0.3, length=1.0)
na = inputs.cgrid_case(97, 24, 32, 0.5, 0.06, r_far=6.0, wake=4.0, ma=0.8, t_inf=0.2, re=1e5, body=nb, naca=0.12)
for prec in (L.FP32, L.FP64):
    run(L.Mesh.cgrid(na.X, na.n_cut, na.bodies, precision=prec), na.flow,
        inputs.initial_field(na.nr, na.ntheta, na.flow, seed=3)[None], post=True)
lk = inputs.BodySpec(dof=1, xc=2.0, xp=2.0, r_in=2.7, r_out=4.5, m_star=4.0, v_r=5.0)
tc = inputs.tandem_case(34, 17, 11, 16, 33, body=lk)
run(L.Mesh.cgrid_walls(tc.X, tc.walls, tc.bodies, precision=L.FP32), tc.flow,
    inputs.initial_field(tc.nr, tc.ntheta, tc.flow, seed=4)[None])
X, si, sj = inputs.box_mesh(24, 16, 24.0, 16.0, skew=0.3)
bf = inputs.FlowSpec(ma=0.1, re=10.0, dt=0.5)
Mb = inputs.initial_field(24, 16, bf, seed=5)
run(L.Mesh.box(X, si, sj, precision=L.FP32), bf, Mb[None])
batch = L.Batch(256 << 20, precision=L.FP32)
batch.set_graph_steps(2)
batch.add(case.r, case.e, body, case.flow, 7, M0)
batch.add_xy(ell.X, body, ell.flow, 5, inputs.initial_field(ell.nr, ell.ntheta, ell.flow, seed=6))
batch.add_cgrid(na.X, na.n_cut, nb, na.flow, 6, inputs.initial_field(na.nr, na.ntheta, na.flow, seed=7))
while batch.step(3) > 0:
    pass
for s in range(3):
    batch.get(s)
batch.close()
print("clean")
'''


def test_bounds_checked_build_runs_clean():
    from paper_2107_01370_gb300 import build
    build.build(bounds=True)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "clean" in r.stdout
