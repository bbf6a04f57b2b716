"""lbfsi_field_ptr: the handle's current moment field and populations as a
torch tensor over the same device memory (no copy), equal to what the
synchronising host accessors return, on a separable O-grid (FP64) and on a
C-grid with its mirrored rows (FP32)."""
import numpy as np
import pytest

from paper_2107_01370_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2107_01370_gb300 import build, lbfsi
    build.build()
    lbfsi.load()
    return lbfsi


def _check_views(L, m, nr, nt, nb):
    import torch
    m.synchronize()
    N = nr * nt
    mv = m.field_view(L.FIELD_MOMENTS)
    Mt = torch.as_tensor(mv, device="cuda")
    assert Mt.data_ptr() == m.field_ptr(L.FIELD_MOMENTS)[0]      # a view, not a copy
    got = Mt[:, :, mv.row0:mv.row0 + N].double().cpu().numpy().reshape(nb, 4, nr, nt)
    assert np.array_equal(got, m.get_fields())
    pv = m.field_view(L.FIELD_POPULATIONS)
    Pt = torch.as_tensor(pv, device="cuda")
    pairs = Pt[:, :, pv.row0:pv.row0 + N, :].double().cpu().numpy()
    f, g = m.get_populations(0)
    assert np.array_equal(pairs[..., 0].reshape(f.shape), f)
    assert np.array_equal(pairs[..., 1].reshape(g.shape), g)
    # the pointer follows the current buffer of the ping-pong pair
    p0 = m.field_ptr(L.FIELD_MOMENTS)[0]
    m.step(1)
    m.synchronize()
    assert m.field_ptr(L.FIELD_MOMENTS)[0] != p0


def test_field_views_separable_fp64(L):
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=3.0, v_r=4.0)
    case = inputs.cylinder_case(32, 64, r_far=8.0, body=body)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=5)
    m = L.Mesh(case.r, case.e, case.bodies * 2, precision=L.FP64)
    m.init_fields(case.flow, np.ascontiguousarray(np.broadcast_to(M0, (2,) + M0.shape)))
    m.step(3)
    _check_views(L, m, case.nr, case.ntheta, 2)
    m.close()


def test_field_views_cgrid_fp32(L):
    case = inputs.cgrid_case(33, 8, 24, 0.6, 0.35, r_far=6.0, wake=4.0, length=1.2)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=6)
    m = L.Mesh.cgrid(case.X, case.n_cut, case.bodies, precision=L.FP32)
    m.init_fields(case.flow, M0[None])
    m.step(3)
    assert m.field_ptr(L.FIELD_MOMENTS)[1:] == (case.nodes + 4 * case.ntheta, 4 * case.ntheta)
    _check_views(L, m, case.nr, case.ntheta, 1)
    m.close()
