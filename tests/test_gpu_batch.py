"""Batch runtime (continuous batching of uneven meshes): every solve gives the
same result alone and in the mix, FP64 batches match the oracle, and
admission is decided by the device memory pool."""
import numpy as np
import pytest

import oracle.mesh as OM
import oracle.solver as OS
from paper_2107_01370_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2107_01370_gb300 import build, lbfsi
    build.build()
    lbfsi.load()
    return lbfsi


def _case(nr, nt, v_r, m_star, seed):
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=m_star, v_r=v_r)
    case = inputs.cylinder_case(nr, nt, r_far=8.0, body=body)
    M0 = inputs.initial_field(nr, nt, case.flow, seed=seed)
    return case, M0


SPECS = [(32, 32, 3.0, 2.0, 1, 7), (48, 64, 5.0, 10.0, 2, 11), (64, 96, 8.0, 20.0, 3, 9)]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_each_solve_same_alone_and_in_the_mix(L, precision):
    """Three solves of different sizes and step counts, admitted at different
    times into one batch, give bit-identical fields, loads and body states to
    the same solves run alone through the single-mesh handle."""
    prec = L.FP32 if precision == "fp32" else L.FP64
    batch = L.Batch(256 << 20, precision=prec)
    cases = [_case(nr, nt, vr, ms, seed) for nr, nt, vr, ms, seed, _ in SPECS]
    steps = [s[5] for s in SPECS]
    slots = [batch.add(cases[0][0].r, cases[0][0].e, cases[0][0].bodies[0], cases[0][0].flow, steps[0],
                       cases[0][1])]
    batch.step(2)                                   # solve 0 runs alone for 2 steps
    slots.append(batch.add(cases[1][0].r, cases[1][0].e, cases[1][0].bodies[0], cases[1][0].flow,
                           steps[1], cases[1][1]))
    batch.step(3)
    slots.append(batch.add(cases[2][0].r, cases[2][0].e, cases[2][0].bodies[0], cases[2][0].flow,
                           steps[2], cases[2][1]))
    while batch.step(1) > 0:
        pass
    for k, (case, M0) in enumerate(cases):
        assert batch.poll(slots[k]) == (steps[k], True)
        fb, lb, sb = batch.get(slots[k])
        mesh = L.Mesh(case.r, case.e, case.bodies, precision=prec)
        mesh.init_fields(case.flow, M0[None])
        mesh.step(steps[k])
        fa = mesh.get_fields()[0]
        la = mesh.body_forces()[0]
        sa = mesh.body_state()[0]
        mesh.close()
        assert np.array_equal(fa, fb), k
        assert np.array_equal(la, lb), k
        assert sa == sb, k
    for s in slots:
        batch.remove(s)
    batch.close()


def test_fp64_batch_matches_oracle(L):
    batch = L.Batch(128 << 20, precision=L.FP64)
    got = []
    for nr, nt, vr, ms, seed, n in SPECS[:2]:
        case, M0 = _case(nr, nt, vr, ms, seed)
        got.append((batch.add(case.r, case.e, case.bodies[0], case.flow, n, M0), case, M0, n))
    while batch.step(1) > 0:
        pass
    for slot, case, M0, n in got:
        s = OS.Solver.from_case(OM.ogrid_mesh(case.r, case.e), case, M0)
        for _ in range(n):
            r = s.step()
        f, loads, st = batch.get(slot)
        err = max(np.abs(f[c] - r.M[c]).max() / np.abs(r.M[c]).max() for c in (0, 3))
        err = max(err, np.hypot(f[1] - r.M[1], f[2] - r.M[2]).max() / np.hypot(r.M[1], r.M[2]).max())
        assert err < 1e-12
        assert np.abs(loads - np.array(r.force)).max() < 1e-12 / 3.0
        assert abs(st["h"] - s.S[0]["h"]) < 1e-12
    batch.close()


def test_admission_by_device_memory(L):
    """A pool sized for about two solves admits two, refuses the third until
    one is removed, and returns all its memory at the end."""
    case, M0 = _case(64, 96, 5.0, 5.0, 4)
    probe = L.Batch(64 << 20, precision=L.FP32)
    free0, _ = probe.memory()
    s0 = probe.add(case.r, case.e, case.bodies[0], case.flow, 3, M0)
    per_solve = free0 - probe.memory()[0]
    probe.remove(s0)
    assert probe.memory()[0] == free0
    probe.close()
    batch = L.Batch(int(2.5 * per_solve), precision=L.FP32)
    free_start, _ = batch.memory()
    a = batch.add(case.r, case.e, case.bodies[0], case.flow, 3, M0)
    b = batch.add(case.r, case.e, case.bodies[0], case.flow, 3, M0)
    c = batch.add(case.r, case.e, case.bodies[0], case.flow, 3, M0)
    assert a is not None and b is not None and c is None
    batch.step(3)
    batch.remove(a)
    c = batch.add(case.r, case.e, case.bodies[0], case.flow, 3, M0)
    assert c is not None
    while batch.step(1) > 0:
        pass
    f1 = batch.get(b)[0]
    f2 = batch.get(c)[0]
    assert np.array_equal(f1, f2)        # same inputs, admitted at different times
    batch.remove(b)
    batch.remove(c)
    assert batch.memory()[0] == free_start
    batch.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_general_and_separable_meshes_in_one_batch(L, precision):
    """Solves on O-grids given by node coordinates (an elliptic cylinder)
    share the batch with separable O-grids: two launches per step, one per
    geometry kind.  Every solve, admitted at a different time, ends bit for
    bit like the same solve alone, also across a schedule change and with
    graph replay."""
    prec = L.FP32 if precision == "fp32" else L.FP64
    ell_body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=3.0, v_r=4.0, length=1.2)
    ell = inputs.xy_case(inputs.ellipse_wall(64, 0.6, 0.35), 40, r_far=8.0, length=1.2, body=ell_body)
    M_ell = inputs.initial_field(ell.nr, ell.ntheta, ell.flow, seed=31)
    sep = [_case(32, 32, 3.0, 2.0, 1), _case(48, 64, 5.0, 10.0, 2)]
    steps = {"e": 30, "s0": 25, "s1": 34}
    batch = L.Batch(256 << 20, precision=prec)
    batch.set_graph_steps(4)
    slots = {"s0": batch.add(sep[0][0].r, sep[0][0].e, sep[0][0].bodies[0], sep[0][0].flow, steps["s0"], sep[0][1])}
    batch.step(3)
    slots["e"] = batch.add_xy(ell.X, ell_body, ell.flow, steps["e"], M_ell, centre=ell.centre)
    batch.step(5)
    if prec == L.FP32:
        batch.set_schedule(0, 1)
    slots["s1"] = batch.add(sep[1][0].r, sep[1][0].e, sep[1][0].bodies[0], sep[1][0].flow, steps["s1"], sep[1][1])
    while batch.step(7) > 0:
        pass
    got = {k: batch.get(v) for k, v in slots.items()}
    batch.close()
    # alone
    m = L.Mesh.xy(ell.X, [ell_body], precision=prec, centre=ell.centre)
    m.init_fields(ell.flow, M_ell[None])
    m.step(steps["e"])
    alone = {"e": (m.get_fields()[0], m.body_forces()[0], m.body_state()[0])}
    m.close()
    for k, (case, M0) in (("s0", sep[0]), ("s1", sep[1])):
        m = L.Mesh(case.r, case.e, case.bodies, precision=prec)
        m.init_fields(case.flow, M0[None])
        m.step(steps[k])
        alone[k] = (m.get_fields()[0], m.body_forces()[0], m.body_state()[0])
        m.close()
    for k in slots:
        assert np.array_equal(got[k][0], alone[k][0]), k
        assert np.array_equal(got[k][1], alone[k][1]), k
        assert got[k][2] == alone[k][2], k


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cgrid_solves_in_the_batch(L, precision):
    """A C-grid solve (collide-only and stream table launches) shares the
    batch with a separable and a general O-grid solve, admitted at different
    times, with graph replay: each ends bit for bit like the same solve alone."""
    prec = L.FP32 if precision == "fp32" else L.FP64
    cb = inputs.BodySpec(dof=2, xp=-0.2, yp=0.0, r_in=0.75, r_out=2.0, m_star=5.0, v_r=2.0, x_alpha=0.3,
                         r_alpha=0.6, wh_wa=0.5, length=1.2)
    cgc = inputs.cgrid_case(49, 8, 32, 0.6, 0.35, r_far=6.0, wake=4.0, length=1.2, body=cb)
    M_c = inputs.initial_field(cgc.nr, cgc.ntheta, cgc.flow, seed=51)
    eb = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=3.0, v_r=4.0, length=1.2)
    ell = inputs.xy_case(inputs.ellipse_wall(64, 0.6, 0.35), 40, r_far=8.0, length=1.2, body=eb)
    M_e = inputs.initial_field(ell.nr, ell.ntheta, ell.flow, seed=52)
    sep = _case(48, 64, 5.0, 10.0, 2)
    steps = {"c": 27, "e": 22, "s": 31}
    batch = L.Batch(256 << 20, precision=prec)
    batch.set_graph_steps(3)
    slots = {"s": batch.add(sep[0].r, sep[0].e, sep[0].bodies[0], sep[0].flow, steps["s"], sep[1])}
    batch.step(4)
    slots["c"] = batch.add_cgrid(cgc.X, cgc.n_cut, cb, cgc.flow, steps["c"], M_c)
    batch.step(2)
    slots["e"] = batch.add_xy(ell.X, eb, ell.flow, steps["e"], M_e)
    while batch.step(5) > 0:
        pass
    got = {k: batch.get(v) for k, v in slots.items()}
    batch.close()
    alone = {}
    m = L.Mesh.cgrid(cgc.X, cgc.n_cut, [cb], precision=prec)
    m.init_fields(cgc.flow, M_c[None])
    m.step(steps["c"])
    alone["c"] = (m.get_fields()[0], m.body_forces()[0], m.body_state()[0])
    m.close()
    m = L.Mesh.xy(ell.X, [eb], precision=prec)
    m.init_fields(ell.flow, M_e[None])
    m.step(steps["e"])
    alone["e"] = (m.get_fields()[0], m.body_forces()[0], m.body_state()[0])
    m.close()
    m = L.Mesh(sep[0].r, sep[0].e, sep[0].bodies, precision=prec)
    m.init_fields(sep[0].flow, sep[1][None])
    m.step(steps["s"])
    alone["s"] = (m.get_fields()[0], m.body_forces()[0], m.body_state()[0])
    m.close()
    for k in slots:
        assert np.array_equal(got[k][0], alone[k][0]), k
        assert np.array_equal(got[k][1], alone[k][1]), k
        assert got[k][2] == alone[k][2], k


def test_batch_tensor_copy_staging_is_bit_identical(L, monkeypatch):
    """The batch's float table launch stages the populations and moments of a
    tile whose columns do not wrap by tensor copies, through per-solve tensor
    maps; LBFSI_TMA=0 stages every tile by per-thread copies.  Three solves
    with Ntheta 64, 128 and 256 (no, two and six such tiles per tile row)
    advanced together: the same bits either way, for every solve."""
    specs = [(32, 64, 3.0, 2.0, 1, 9), (48, 128, 5.0, 10.0, 2, 12), (40, 256, 8.0, 20.0, 3, 10)]

    def run():
        batch = L.Batch(256 << 20, precision=L.FP32)
        slots = []
        for nr, nt, vr, ms, seed, n in specs:
            case, M0 = _case(nr, nt, vr, ms, seed)
            slots.append(batch.add(case.r, case.e, case.bodies[0], case.flow, n, M0))
        while batch.step(1) > 0:
            pass
        out = [batch.get(s) for s in slots]
        for s in slots:
            batch.remove(s)
        batch.close()
        return out

    monkeypatch.setenv("LBFSI_TMA", "0")
    ref = run()
    monkeypatch.delenv("LBFSI_TMA")
    got = run()
    for k, ((fa, la, sa), (fb, lb, sb)) in enumerate(zip(ref, got)):
        assert np.array_equal(fa, fb), k
        assert np.array_equal(la, lb), k
        assert sa == sb, k
