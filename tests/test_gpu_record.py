"""Per-step load and body-state histories (lbfsi_step_record): the records
copied behind every launch equal, bit for bit, what lbfsi_body_forces and
lbfsi_get_body_state return after each single step, and the run itself is
the same run."""
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


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_step_record_equals_single_steps(L, precision):
    prec = L.FP32 if precision == "fp32" else L.FP64
    bodies = [inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=2.0, v_r=4.0),
              inputs.BodySpec(dof=2, xp=-0.25, r_in=0.75, r_out=2.0, m_star=5.0, v_r=2.0,
                              x_alpha=0.3, r_alpha=0.6, wh_wa=0.5)]
    case = inputs.cylinder_case(40, 64, r_far=8.0)
    M0 = np.stack([inputs.initial_field(40, 64, case.flow, seed=s) for s in (2, 3)])
    runs = []
    for mode in ("record", "single"):
        m = L.Mesh(case.r, case.e, bodies, precision=prec)
        m.init_fields(case.flow, M0)
        m.blend_mesh([(0.01, 0.0, 0.002, 0.0), (-0.01, 0.02, 0.0, 0.005)])
        if mode == "record":
            loads, states = m.step_record(15, states=True)
        else:
            loads, states = [], []
            for _ in range(15):
                m.step(1)
                loads.append(m.body_forces().copy())
                states.append([[s["h"], s["alpha"], s["hdot"], s["adot"]] for s in m.body_state()])
            loads, states = np.array(loads), np.array(states)
        runs.append((loads, states, m.get_fields()))
        m.close()
    (la, sa, fa), (lb, sb, fb) = runs
    assert la.shape == (15, 2, 3) and sa.shape == (15, 2, 4)
    assert np.array_equal(la, lb)
    assert np.array_equal(sa, sb)
    assert np.array_equal(fa, fb)
