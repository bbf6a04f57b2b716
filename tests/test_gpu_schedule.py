"""Execution schedule, CUDA-graph replay and the autotuner: none of them may
change a solve.  Every tile shape and CTA order, graph replay against plain
launches, and a run that spent its first steps tuning must give bit-identical
fields, loads and body states."""
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


def _case(nr=64, nt=96, v_r=5.0, m_star=4.0, seed=3):
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=m_star, v_r=v_r)
    case = inputs.cylinder_case(nr, nt, r_far=8.0, body=body)
    M0 = inputs.initial_field(nr, nt, case.flow, seed=seed)
    return case, M0


def _run_mesh(L, case, M0, steps, precision, nbatch=2, schedule=None, graph=0):
    m = L.Mesh(case.r, case.e, case.bodies * nbatch, precision=precision)
    if schedule is not None:
        m.set_schedule(*schedule)
    m.init_fields(case.flow, np.ascontiguousarray(np.broadcast_to(M0, (nbatch,) + M0.shape)))
    if graph:
        m.set_graph_steps(graph)
    m.step(steps)
    out = (m.get_fields(), m.body_forces(), m.body_state())
    m.close()
    return out


def _same(a, b):
    fa, la, sa = a
    fb, lb, sb = b
    assert np.array_equal(fa, fb)
    assert np.array_equal(la, lb)
    assert sa == sb


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_every_tile_shape_and_order_is_bit_identical(L, precision):
    prec = L.FP32 if precision == "fp32" else L.FP64
    case, M0 = _case()
    ref = _run_mesh(L, case, M0, 25, prec, schedule=(0, 0))
    assert L.step_variants(prec) == (5 if precision == "fp32" else 3)
    for v in range(L.step_variants(prec)):
        for o in (0, 1):
            _same(ref, _run_mesh(L, case, M0, 25, prec, schedule=(v, o)))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_graph_replay_equals_plain_launches(L, precision):
    prec = L.FP32 if precision == "fp32" else L.FP64
    case, M0 = _case(48, 64)
    plain = _run_mesh(L, case, M0, 23, prec)
    graphed = _run_mesh(L, case, M0, 23, prec, graph=7)     # 3 replays + 2 plain launches
    _same(plain, graphed)


def test_mesh_autotune_picks_a_schedule_and_keeps_the_trajectory(L):
    case, M0 = _case()
    nb = 2
    m = L.Mesh(case.r, case.e, case.bodies * nb, precision=L.FP32)
    m.init_fields(case.flow, np.ascontiguousarray(np.broadcast_to(M0, (nb,) + M0.shape)))
    v, o, ms = m.autotune(steps_per_trial=3)
    nv = L.step_variants(L.FP32)
    assert 0 <= v < nv and o in (0, 1)
    assert ms.shape == (nv, 2) and np.all(ms > 0)
    assert ms[v, o] == ms.min()
    assert m.schedule() == (v, o)
    m.step(5)
    tuned = (m.get_fields(), m.body_forces(), m.body_state())
    m.close()
    steps = nv * 2 * (1 + 3) + 5
    _same(tuned, _run_mesh(L, case, M0, steps, L.FP32, nbatch=nb))


SPECS = [(32, 32, 3.0, 2.0, 1, 40), (48, 64, 5.0, 10.0, 2, 55), (64, 96, 8.0, 20.0, 3, 47)]


def _batch_run(L, schedule=None, graph=0, tune=0):
    batch = L.Batch(256 << 20, precision=L.FP32)
    slots = []
    for nr, nt, vr, ms, seed, n in SPECS:
        case, M0 = _case(nr, nt, vr, ms, seed)
        slots.append(batch.add(case.r, case.e, case.bodies[0], case.flow, n, M0))
    if schedule is not None:
        batch.set_schedule(*schedule)
    if graph:
        batch.set_graph_steps(graph)
    info = batch.autotune(tune) if tune else None
    while batch.step(10) > 0:
        pass
    out = [batch.get(s) for s in slots]
    for s in slots:
        assert batch.poll(s)[1]
        batch.remove(s)
    batch.close()
    return out, info


def test_batch_schedule_graph_and_autotune_keep_every_result(L):
    ref, _ = _batch_run(L)
    for sched, graph in (((0, 1), 0), ((4, 0), 6), ((2, 1), 4)):
        got, _ = _batch_run(L, schedule=sched, graph=graph)
        for a, b in zip(ref, got):
            _same(a, b)
    got, (v, o, ns) = _batch_run(L, graph=5, tune=2)
    assert 0 <= v < L.step_variants(L.FP32) and o in (0, 1)
    assert np.all(ns > 0)
    for a, b in zip(ref, got):
        _same(a, b)


def test_tensor_copy_staging_is_bit_identical_to_per_thread_copies(L, monkeypatch):
    """The float kernel stages the populations and moments of a tile whose
    columns do not wrap by tensor copies (TMA); LBFSI_TMA=0 at handle creation
    stages every tile by per-thread copies.  Ntheta = 128 gives two such tiles
    of four per tile row; every float tile shape, with a moving body, must
    give the same bits either way."""
    case, M0 = _case(64, 128)
    for v in range(L.step_variants(L.FP32)):
        monkeypatch.setenv("LBFSI_TMA", "0")
        ref = _run_mesh(L, case, M0, 25, L.FP32, schedule=(v, 1))
        monkeypatch.delenv("LBFSI_TMA")
        _same(ref, _run_mesh(L, case, M0, 25, L.FP32, schedule=(v, 1)))
