"""The one loose physical check of the whole coupled run (the oracle is
pinned part by part; there is no printed worked example): a fixed circular
cylinder at Re 100, Ma 0.2 sheds vortices periodically at a Strouhal number
of about 0.16-0.17.  The run starts from the seeded free stream (noise 1e-3
U_inf) on a 256 x 128 O-grid to 20 D and takes 300k steps (about 335
convective times, ten seconds on a GB300); the shedding is measured over the
last 150k.  Measured: St 0.163, mean C_D 1.43, C_L amplitude 0.40."""
import numpy as np
import pytest

from paper_2107_01370_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_fixed_cylinder_sheds_at_the_strouhal_number_of_re_100():
    from paper_2107_01370_gb300 import build, lbfsi as L
    build.build()
    L.load()
    case = inputs.cylinder_case(256, 128)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    m = L.Mesh(case.r, case.e, case.bodies, precision=L.FP32)
    m.init_fields(case.flow, M0[None])
    qd = 0.5 * case.flow.rho_inf * case.flow.u_inf ** 2 * case.flow.length
    hist = np.concatenate([m.step_record(50000)[:, 0] / qd for _ in range(6)])
    m.synchronize()   # raises if the run turned non-physical
    M = m.get_fields()[0]
    m.close()
    assert 0.9 < M[0].min() and M[0].max() < 1.2 and 0.3 < M[3].min() and M[3].max() < 0.37
    tail = hist[-150000:]
    cl = tail[:, 1]
    up = np.nonzero((cl[:-1] < 0) & (cl[1:] >= 0))[0]
    periods = (up[-1] - up[0]) / (len(up) - 1) * case.flow.dt * case.flow.u_inf / case.flow.length
    st = 1.0 / periods
    assert 0.155 < st < 0.175, st
    amp = 0.5 * (cl.max() - cl.min())
    assert 0.2 < amp < 0.6, amp
    assert 1.2 < tail[:, 0].mean() < 1.6, tail[:, 0].mean()
