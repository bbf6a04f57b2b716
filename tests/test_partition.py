"""One mesh split over ranks along the angular index (paper_2107_01370_gb300/
partition.py), tested on CPU ranks (gloo, world size 2): each rank steps its
own columns of the O-grid with the oracle's step, every column outside its
range and its halos set to NaN before every step (so a stencil reaching
further than the halo poisons the result), the halos filled from the
neighbours by the partition's point-to-point exchange, and the wall load
assembled from every rank's edge terms in the global order.  Every rank's
columns, every step's load and the body state must equal the one-rank
oracle run bit for bit: the fixed cylinder of the 128 x 64 workload, and a
1-DOF body whose redundant RK4 updates on both ranks must stay identical."""
import os
import socket

import numpy as np
import pytest

from paper_2107_01370_gb300 import partition as P

STEPS = 10


def test_ranges_cover_the_ring_in_whole_tiles():
    for nt in (64, 100, 256, 520):
        for nranks in range(1, -(-nt // 32) + 1):
            part = P.AngularPartition(nt, nranks)
            cols = []
            for r in range(nranks):
                j0, j1 = part.owned(r)
                assert j0 % 32 == 0 and (j1 % 32 == 0 or j1 == nt) and j1 > j0
                cols.extend(range(j0, j1))
            assert cols == list(range(nt))
    with pytest.raises(ValueError):
        P.AngularPartition(64, 3)


def test_halo_columns_wrap_and_come_from_the_adjacent_rank():
    part = P.AngularPartition(96, 3)
    assert part.owned(0) == (0, 32) and part.owned(2) == (64, 96)
    assert part.halo_columns(0, 4) == ([92, 93, 94, 95], [32, 33, 34, 35])
    assert part.halo_columns(2, 2) == ([62, 63], [0, 1])
    assert part.neighbours(0) == (2, 1)
    assert part.local_columns(1, 1) == [31] + list(range(32, 64)) + [64]
    with pytest.raises(ValueError):
        P.AngularPartition(70, 3).check_halo(8)   # the last range holds 6 columns


def test_one_rank_exchange_leaves_the_ring_unchanged():
    """With one rank the halo columns of the periodic ring are the rank's own
    end columns: the exchange copies each onto itself."""
    torch = pytest.importorskip("torch")
    part = P.AngularPartition(64, 1)
    a = torch.arange(2 * 64, dtype=torch.float64).reshape(2, 64)
    b = a.clone()
    P.exchange_halos(part, 0, [b], 4)
    assert torch.equal(a, b)
    assert part.halo_columns(0, 2) == ([62, 63], [0, 1])
    assert P.ordered_sum([0.1, 0.2, 0.3]) == (0.1 + 0.2) + 0.3


# ----- two gloo ranks stepping one mesh ---------------------------------------
def _cases():
    from paper_2107_01370_gb300 import inputs
    fixed = inputs.fixed_cylinder_128x64(steps=STEPS)
    body = inputs.BodySpec(dof=1, r_in=0.75, r_out=2.0, m_star=2.0, v_r=4.0)
    moving = inputs.cylinder_case(40, 64, r_far=8.0, body=body, steps=STEPS)
    state = {"h": 0.02, "alpha": 0.0, "hdot": 0.004, "adot": 0.0}
    prev = {"h": 0.0199, "alpha": 0.0, "hdot": 0.004, "adot": 0.0}
    return [("fixed", fixed, None, None), ("moving", moving, state, prev)]


def _solver(case, state, prev):
    import oracle.mesh as OM
    import oracle.solver as OS
    from paper_2107_01370_gb300 import inputs
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    s = OS.Solver.from_case(OM.ogrid_mesh(case.r, case.e), case, M0)
    if state is not None:
        s.S = [dict(state)]
        s.S_prev = [dict(prev)]
    return s


def _edge_terms(x_wall, sxx, sxy, syy, x_ref, edges):
    """The terms of the oracle's wall-load sum (Simpson shares of each
    straight wall edge, forces.wall_force) for the given edges, in the
    order that sum takes them: rows (F_x, F_y, M_z)."""
    Nj = x_wall.shape[0]
    out = []
    for k in edges:
        ids = (2 * k, 2 * k + 1, (2 * k + 2) % Nj)
        t = x_wall[ids[2]] - x_wall[ids[0]]
        ds = float(np.hypot(t[0], t[1]))
        n = np.array([t[1], -t[0]]) / ds
        for w, idx in zip((1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0), ids):
            tx = sxx[idx] * n[0] + sxy[idx] * n[1]
            ty = sxy[idx] * n[0] + syy[idx] * n[1]
            rx = x_wall[idx, 0] - x_ref[0]
            ry = x_wall[idx, 1] - x_ref[1]
            out.append((w * ds * tx, w * ds * ty, w * ds * (rx * ty - ry * tx)))
    return out


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    halo = P.HALO_POST_COLLISION    # the oracle keeps post-collision populations
    results = {}
    for name, case, state, prev in _cases():
        part = P.AngularPartition(case.ntheta, world)
        j0, j1 = part.owned(rank)
        keep_f = np.zeros(case.ntheta, dtype=bool)
        keep_f[part.local_columns(rank, halo["populations"])] = True
        keep_m = np.zeros(case.ntheta, dtype=bool)
        keep_m[part.local_columns(rank, halo["moments"])] = True
        own = np.zeros(case.ntheta, dtype=bool)
        own[j0:j1] = True
        edges = [k for k in range(case.ntheta // 2) if j0 <= 2 * k < j1]

        def reduce_loads(x_wall, sxx, sxy, syy, x_ref):
            mine = np.array(_edge_terms(x_wall, sxx, sxy, syy, x_ref, edges), dtype=np.float64)
            allt = P.gather_in_order(part, torch.from_numpy(mine.reshape(-1)), dist).numpy()
            allt = allt.reshape(-1, 3)
            return tuple(P.ordered_sum(allt[:, c]) for c in range(3))

        s = _solver(case, state, prev)
        s.load_reduction = reduce_loads
        loads, states = [], []
        for _ in range(STEPS):
            # nothing outside the own columns survives a step; halos come
            # from the neighbours
            s.f[..., ~own] = np.nan
            s.g[..., ~own] = np.nan
            s.M_prev[..., ~own] = np.nan
            P.exchange_halos(part, rank, [torch.from_numpy(s.f), torch.from_numpy(s.g)],
                             halo["populations"], dist)
            P.exchange_halos(part, rank, [torch.from_numpy(s.M_prev)], halo["moments"], dist)
            assert np.isnan(s.f[..., ~keep_f]).all() and not np.isnan(s.f[..., keep_f]).any()
            assert not np.isnan(s.M_prev[..., keep_m]).any()
            with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
                r = s.step()
            loads.append(r.force)
            states.append(dict(s.S[0]))
        results[name] = (j0, j1, s.f[..., j0:j1].copy(), s.g[..., j0:j1].copy(),
                         r.M[..., j0:j1].copy(), np.array(loads), states)
    q.put((rank, results))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_step_one_mesh_bit_identical_to_one_rank():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for name, case, state, prev in _cases():
        s = _solver(case, state, prev)
        loads = []
        for _ in range(STEPS):
            r = s.step()
            loads.append(r.force)
        for rank in (0, 1):
            j0, j1, f, g, M, gl, gs = got[rank][name]
            assert np.array_equal(f, s.f[..., j0:j1]), (name, rank)
            assert np.array_equal(g, s.g[..., j0:j1]), (name, rank)
            assert np.array_equal(M, r.M[..., j0:j1]), (name, rank)
            assert np.array_equal(gl, np.array(loads)), (name, rank)
            assert gs[-1] == s.S[0], (name, rank)
        if name == "moving":
            assert abs(s.S[0]["h"] - 0.02) > 1e-6      # the body did move


@pytest.mark.parametrize("pops,moms", [(4, 3), (3, 4)])
def test_a_narrower_halo_reaches_the_own_columns(pops, moms):
    """The halo widths are the least that work: one column less of either
    state and the NaN outside reaches the rank's own columns within a step
    (so the two-rank test above would see it)."""
    import oracle.mesh as OM
    import oracle.solver as OS
    from paper_2107_01370_gb300 import inputs
    case = inputs.fixed_cylinder_128x64(steps=1)
    M0 = inputs.initial_field(case.nr, case.ntheta, case.flow, seed=0)
    s = OS.Solver.from_case(OM.ogrid_mesh(case.r, case.e), case, M0)
    part = P.AngularPartition(case.ntheta, 2)
    j0, j1 = part.owned(0)
    kf = np.zeros(case.ntheta, dtype=bool)
    kf[part.local_columns(0, pops)] = True
    km = np.zeros(case.ntheta, dtype=bool)
    km[part.local_columns(0, moms)] = True
    s.f[..., ~kf] = np.nan
    s.g[..., ~kf] = np.nan
    s.M_prev[..., ~km] = np.nan
    s.load_reduction = lambda *a: (0.0, 0.0, 0.0)
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        r = s.step()
    assert np.isnan(r.f_post[..., j0:j1]).any()
    assert P.HALO_POST_COLLISION == {"populations": 4, "moments": 4}
