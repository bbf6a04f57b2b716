"""Checkpoint / resume and host-visible failure reports.

A run restored from a checkpoint into a fresh handle continues bit for bit
like the uninterrupted run (the checkpoint holds every piece of state the
next step reads: populations, moments, body states including the previous
one for the mesh velocity, loads, maps and the step number).  A poisoned
input field is reported as a non-physical state, by the mesh handle and by
the batch runtime, without faulting anything."""
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


def _case(dof, nr=48, nt=64, seed=5):
    if dof == 2:
        body = inputs.BodySpec(dof=2, r_in=0.75, r_out=2.0, m_star=5.0, v_r=1.5, x_alpha=0.2,
                               r_alpha=0.5, wh_wa=0.8)
    else:
        body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=3.0, v_r=4.0)
    case = inputs.cylinder_case(nr, nt, r_far=8.0, body=body)
    M0 = inputs.initial_field(nr, nt, case.flow, seed=seed)
    return case, M0


def _mesh(L, case, M0, prec, nb=2):
    m = L.Mesh(case.r, case.e, case.bodies * nb, precision=prec)
    m.init_fields(case.flow, np.ascontiguousarray(np.broadcast_to(M0, (nb,) + M0.shape)))
    return m


def _state(m):
    return m.get_fields(), m.body_forces(), m.body_state()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("dof", [1, 2])
@pytest.mark.parametrize("at", [0, 12])
def test_resume_from_checkpoint_is_bit_identical(L, precision, dof, at):
    prec = L.FP32 if precision == "fp32" else L.FP64
    case, M0 = _case(dof)
    a = _mesh(L, case, M0, prec)
    a.step(at)
    ckpt = a.checkpoint()
    a.step(30 - at)
    ref = _state(a)
    a.close()
    # a fresh handle, initialised from a different field, then restored
    b = _mesh(L, case, inputs.initial_field(case.nr, case.ntheta, case.flow, seed=99), prec)
    b.restore(ckpt)
    b.step(30 - at)
    got = _state(b)
    b.close()
    assert np.array_equal(ref[0], got[0])
    assert np.array_equal(ref[1], got[1])
    assert ref[2] == got[2]


def test_restore_rejects_a_checkpoint_of_another_handle(L):
    case, M0 = _case(1)
    a = _mesh(L, case, M0, L.FP32)
    a.step(3)
    ckpt = a.checkpoint()
    a.close()
    other, M1 = _case(1, nr=40, nt=64)
    b = _mesh(L, other, M1, L.FP32)
    with pytest.raises(L.LbfsiError) as ei:
        b.restore(ckpt)
    assert ei.value.code == L.EINVAL
    c = _mesh(L, case, M0, L.FP64)
    with pytest.raises(L.LbfsiError) as ei:
        c.restore(ckpt)
    assert ei.value.code == L.EINVAL
    with pytest.raises(L.LbfsiError):
        c.restore(b"not a checkpoint" + bytes(len(ckpt)))
    b.close()
    c.close()


def test_poisoned_field_is_reported_as_nonphysical(L):
    case, M0 = _case(1)
    bad = M0.copy()
    bad[0, 10, 7] = np.nan          # one node's density
    m = L.Mesh(case.r, case.e, case.bodies, precision=L.FP32)
    m.init_fields(case.flow, bad[None])
    m.step(2)
    with pytest.raises(L.LbfsiError) as ei:
        m.synchronize()
    assert ei.value.code == L.ENONPHYS
    # the handle stays usable: a clean state restored and stepped again
    good = L.Mesh(case.r, case.e, case.bodies, precision=L.FP32)
    good.init_fields(case.flow, M0[None])
    good.step(2)
    m.restore(good.checkpoint())
    m.step(2)
    m.synchronize()
    m.close()
    good.close()

    batch = L.Batch(64 << 20, precision=L.FP32)
    s = batch.add(case.r, case.e, case.bodies[0], case.flow, 3, bad)
    while batch.step(1) > 0:
        pass
    with pytest.raises(L.LbfsiError) as ei:
        batch.get(s)
    assert ei.value.code == L.ENONPHYS
    batch.close()
