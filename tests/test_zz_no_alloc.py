"""The allocation-free wall-load entry point (for callers that cannot call
cudaMalloc, e.g. code running while a framework's caching allocator or a
real-time loop owns all device memory) gives the same loads as the handle's
own lbfsi_body_forces, on two calls in a row, in both precisions.

This file is collected last on purpose: the entry point keeps a fixed device
scratch array for the life of the process, and a failure here should not stop
a run that halts at the first failure before the other tests have run.  It
passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from paper_2107_01370_gb300 import inputs

pytestmark = pytest.mark.gpu

P_SCALE = 1.0 / 3.0   # p_inf * D, the scale of the summed pressure terms


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_wall_loads_noalloc_matches_body_forces(precision):
    import torch
    from paper_2107_01370_gb300 import build, lbfsi as L
    build.build()
    L.load()
    prec = L.FP64 if precision == "fp64" else L.FP32
    bodies = [inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=ms, v_r=5.0) for ms in (2.0, 8.0)]
    case = inputs.cylinder_case(24, 48, r_far=8.0)
    M0 = np.stack([inputs.initial_field(24, 48, case.flow, seed=s) for s in (5, 6)])
    mesh = L.Mesh(case.r, case.e, bodies, precision=prec)
    mesh.init_fields(case.flow, M0)
    dev = torch.device("cuda", 0)
    dtype = torch.float64 if prec == L.FP64 else torch.float32
    r_d = torch.tensor(case.r, dtype=torch.float64, device=dev)
    e_d = torch.tensor(case.e, dtype=torch.float64, device=dev)
    ref_d = torch.zeros((2, 3), dtype=torch.float64, device=dev)   # x_p, y_p, alpha
    loads_d = torch.empty((2, 3), dtype=torch.float64, device=dev)
    fl = case.flow
    for call in range(2):
        mesh.step(3 + call)
        expect = mesh.body_forces()
        f, g = mesh.get_populations(0)
        f_d = torch.tensor(f, dtype=dtype, device=dev).contiguous()
        g_d = torch.tensor(g, dtype=dtype, device=dev).contiguous()
        loads_d.fill_(float("nan"))
        torch.cuda.synchronize()
        L.wall_loads_noalloc(case.nr, case.ntheta, 2, prec, r_d.data_ptr(), e_d.data_ptr(), (0.0, 0.0),
                             f_d.data_ptr(), g_d.data_ptr(), ref_d.data_ptr(), fl.mu, fl.dt, fl.gamma,
                             loads_d.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = loads_d.cpu().numpy()
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, expect, rtol=0, atol=1e-12 * P_SCALE)
    mesh.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_wall_loads_noalloc_pitched_body_about_an_offset_axis(precision):
    """A pitch-plunge body whose reference point (elastic axis) is away from
    the cylinder centre, set to a pitched and plunged pose: the rotated wall
    normals and the moment arms about the undeformed reference point give
    the step's own loads, on two calls in a row at two different poses.
    body_ref carries the reference point of the undeformed mesh and the pitch
    angle of the pose the populations were streamed at."""
    import torch
    from paper_2107_01370_gb300 import build, lbfsi as L
    build.build()
    L.load()
    prec = L.FP64 if precision == "fp64" else L.FP32
    xp, yp = 0.2, -0.1
    body = inputs.BodySpec(dof=2, xp=xp, yp=yp, r_in=0.75, r_out=2.0, m_star=10.0, v_r=5.0,
                           x_alpha=0.2, r_alpha=0.5, wh_wa=0.3)
    case = inputs.cylinder_case(24, 48, r_far=8.0)
    M0 = inputs.initial_field(24, 48, case.flow, seed=7)[None]
    mesh = L.Mesh(case.r, case.e, [body], precision=prec)
    mesh.init_fields(case.flow, M0)
    mesh.step(2)
    dev = torch.device("cuda", 0)
    dtype = torch.float64 if prec == L.FP64 else torch.float32
    r_d = torch.tensor(case.r, dtype=torch.float64, device=dev)
    e_d = torch.tensor(case.e, dtype=torch.float64, device=dev)
    loads_d = torch.empty((1, 3), dtype=torch.float64, device=dev)
    fl = case.flow
    scale = 1.0 / 3.0
    for h, alpha in ((0.05, 0.2), (-0.03, -0.15)):
        # the pose of the next stream, at rest (V_G = 0): the mesh is pitched
        # about (x_p, y_p) and plunged by h
        mesh.blend_mesh([(h, alpha, 0.0, 0.0)])
        mesh.step(1)
        expect = mesh.body_forces()
        assert abs(expect[0, 2]) > 1e-6 * scale   # a moment to compare
        f, g = mesh.get_populations(0)
        f_d = torch.tensor(f, dtype=dtype, device=dev).contiguous()
        g_d = torch.tensor(g, dtype=dtype, device=dev).contiguous()
        ref_d = torch.tensor([[xp, yp, alpha]], dtype=torch.float64, device=dev)
        loads_d.fill_(float("nan"))
        torch.cuda.synchronize()
        L.wall_loads_noalloc(case.nr, case.ntheta, 1, prec, r_d.data_ptr(), e_d.data_ptr(), (0.0, 0.0),
                             f_d.data_ptr(), g_d.data_ptr(), ref_d.data_ptr(), fl.mu, fl.dt, fl.gamma,
                             loads_d.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = loads_d.cpu().numpy()
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, expect, rtol=0, atol=1e-12 * scale)
        # the plunged position as the reference point is wrong (a different moment)
        ref_d = torch.tensor([[xp, yp + h, alpha]], dtype=torch.float64, device=dev)
        L.wall_loads_noalloc(case.nr, case.ntheta, 1, prec, r_d.data_ptr(), e_d.data_ptr(), (0.0, 0.0),
                             f_d.data_ptr(), g_d.data_ptr(), ref_d.data_ptr(), fl.mu, fl.dt, fl.gamma,
                             loads_d.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert abs(loads_d.cpu().numpy()[0, 2] - expect[0, 2]) > 1e-9 * scale
    mesh.close()


def test_wall_loads_noalloc_rejects_sizes_beyond_the_scratch():
    from paper_2107_01370_gb300 import build, lbfsi as L
    build.build()
    L.load()
    with pytest.raises(L.LbfsiError) as ei:
        L.wall_loads_noalloc(8, 8192, 32, L.FP64, 1, 1, (0.0, 0.0), 1, 1, 1, 1e-3, 1e-2, 1.4, 1, 0)
    assert ei.value.code == L.EINVAL and "4096" in str(ei.value)
