"""The z-slab decomposition of include/lbm_slabs.h, checked on the CPU.

The split comes from the library's host-only lbm_slabs_plan; every slab (its owned planes
plus halo planes) is advanced by the FP64 oracle as a grid of its own, and after every
step each slab's first and last owned planes are copied into its neighbours' halo planes,
as the library's exchange does: in one process, and over two gloo ranks holding one slab
each (the message pattern a multi-GPU run would use).  Pull streaming reads only the
planes z - 1, z, z + 1, so the owned planes must follow the undivided grid bit for bit.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from tests import inputs
from tests.test_gpu_parity import random_state as _random_state


def _slabs():
    from paper_1710_04751_gb300 import slabs
    return slabs


def _problem(nx, ny, nz, q, bc):
    om_f = [1.0] * 4 + list(inputs.random_rates(11, 40 + nz, 0.6, 1.95))
    om_g = [1.0] + list(inputs.random_rates(q - 1, 41 + nz, 0.6, 1.95)) + [1.0] * (15 - q)
    return oracle.Problem(nx, ny, nz, q_g=q, boundary=bc, omega_f=om_f, omega_g=om_g, gbeta=2e-3,
                          T_hot=0.6, T_cold=-0.4, U0=0.05,
                          ext_force=(1e-4, -2e-4, 5e-5) if bc == oracle.BC_PERIODIC else (0, 0, 0))


def _with_nz(p, nz):
    return oracle.Problem(p.nx, p.ny, nz, q_g=p.q_g, boundary=p.boundary, omega_f=p.omega_f,
                          omega_g=p.omega_g, gbeta=p.gbeta, T_hot=p.T_hot, T_cold=p.T_cold,
                          cs2_phi=p.cs2_phi, e4_mode=p.e4_mode, ext_force=p.ext_force, U0=p.U0,
                          adiabatic_mode=p.adiabatic_mode, heat_source=p.heat_source)


def _slab_planes(plan, k, nz):
    """Global plane of every local plane of slab k (wrapping when z is periodic)."""
    lo, own = plan["halo_lo"][k], plan["nz_owned"][k]
    nzb = lo + own + plan["halo_hi"][k]
    return [(plan["z0"][k] - lo + z) % nz for z in range(nzb)]


def _exchange(states, plan):
    S = len(states)
    lo, hi, own = plan["halo_lo"], plan["halo_hi"], plan["nz_owned"]
    for k in range(S):
        for i, X in enumerate(states[k]):  # i = 0: flow, 1: scalar populations
            if lo[k]:
                b = (k - 1) % S
                X[:, 0] = states[b][i][:, lo[b] + own[b] - 1]
            if hi[k]:
                a = (k + 1) % S
                X[:, lo[k] + own[k]] = states[a][i][:, lo[a]]


CASES = [  # (nx, ny, nz, q, boundary, nslabs, owned)
    (12, 10, 17, 15, oracle.BC_CAVITY, 3, [4, 9, 4]),
    (9, 8, 11, 7, oracle.BC_CAVITY, 2, None),
    (10, 8, 11, 15, 6, 2, None),                   # periodic y and z: the cuts wrap
    (8, 8, 9, 15, oracle.BC_PERIODIC, 4, None),
    (8, 6, 5, 15, oracle.BC_CAVITY, 5, None),      # one plane per slab
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}-q{c[3]}-bc{c[4]}-s{c[5]}" for c in CASES])
def test_decomposition_follows_the_whole_grid(case):
    nx, ny, nz, q, bc, nslabs, owned = case
    p = _problem(nx, ny, nz, q, bc)
    plan = _slabs().plan(nz, nslabs, bc, owned)
    F, G = _random_state(p, 9 + nz)
    parts = []
    for k in range(nslabs):
        zs = _slab_planes(plan, k, nz)
        parts.append([F[:, zs].copy(), G[:, zs].copy()])
    probs = [_with_nz(p, parts[k][0].shape[1]) for k in range(nslabs)]
    for _ in range(5):
        F, G = p.step(F, G)
        parts = [list(probs[k].step(*parts[k])) for k in range(nslabs)]
        _exchange(parts, plan)
    for k in range(nslabs):
        zs = _slab_planes(plan, k, nz)
        # every plane of the slab, halos included, equals the whole grid's
        assert np.array_equal(parts[k][0], F[:, zs]) and np.array_equal(parts[k][1], G[:, zs])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, case, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nx, ny, nz, q, bc = case
    p = _problem(nx, ny, nz, q, bc)
    plan = _slabs().plan(nz, world, bc)
    F, G = _random_state(p, 5)
    zs = _slab_planes(plan, rank, nz)
    mine = [F[:, zs].copy(), G[:, zs].copy()]
    prob = _with_nz(p, len(zs))
    lo, hi, own = plan["halo_lo"][rank], plan["halo_hi"][rank], plan["nz_owned"][rank]
    below, above = (rank - 1) % world, (rank + 1) % world
    for _ in range(steps):
        mine = list(prob.step(*mine))
        # tag 2i: a plane of population set i (0 flow, 1 scalar) for the receiver's halo
        # below; tag 2i + 1: for its halo above
        sends = []
        for i, X in enumerate(mine):
            if lo:  # my first owned plane goes to the halo above of the slab below
                sends.append(dist.isend(torch.from_numpy(np.ascontiguousarray(X[:, lo])), below, tag=2 * i + 1))
            if hi:  # my last owned plane goes to the halo below of the slab above
                sends.append(dist.isend(torch.from_numpy(np.ascontiguousarray(X[:, lo + own - 1])), above, tag=2 * i))
        for i, X in enumerate(mine):
            if lo:
                buf = torch.empty(X[:, 0].shape, dtype=torch.float64)
                dist.recv(buf, below, tag=2 * i)
                X[:, 0] = buf.numpy()
            if hi:
                buf = torch.empty(X[:, 0].shape, dtype=torch.float64)
                dist.recv(buf, above, tag=2 * i + 1)
                X[:, lo + own] = buf.numpy()
        for w in sends:
            w.wait()
    out[rank] = (zs[lo:lo + own], mine[0][:, lo:lo + own], mine[1][:, lo:lo + own])
    dist.destroy_process_group()


@pytest.mark.timeout(180)
@pytest.mark.parametrize("case", [(10, 8, 12, 15, oracle.BC_CAVITY), (9, 8, 10, 7, 6)],
                         ids=["cavity", "periodic-z"])
def test_two_gloo_ranks_exchange_halo_planes(case):
    world, steps = 2, 4
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, case, steps, out)) for r in range(world)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(150)
            assert pr.exitcode == 0
        res = dict(out)
    nx, ny, nz, q, bc = case
    p = _problem(nx, ny, nz, q, bc)
    F, G = p.run(*_random_state(p, 5), steps)
    seen = []
    for r in range(world):
        zs, f, g = res[r]
        assert np.array_equal(f, F[:, zs]) and np.array_equal(g, G[:, zs])
        seen += list(zs)
    assert sorted(seen) == list(range(nz))


def _rank_cut_messages(rank, world, port, case, steps, out):
    """As _rank, but each cut carries only the library's message: the populations whose
    e_z crosses it (lbm_slabs_pack_cut / lbm_slabs_unpack_cut)."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sl = _slabs()
    nx, ny, nz, q, bc = case
    p = _problem(nx, ny, nz, q, bc)
    plan = sl.plan(nz, world, bc)
    F, G = _random_state(p, 5)
    zs = _slab_planes(plan, rank, nz)
    f, g = F[:, zs].copy(), G[:, zs].copy()
    prob = _with_nz(p, len(zs))
    lo, hi, own = plan["halo_lo"][rank], plan["halo_hi"][rank], plan["nz_owned"][rank]
    below, above = (rank - 1) % world, (rank + 1) % world
    sizes = []
    for _ in range(steps):
        f, g = prob.step(f, g)
        sends = []
        if hi:  # upward set of my last owned plane, for the halo below of the slab above
            m = sl.pack_cut(f, g, q, lo + own - 1, +1)
            sizes.append(m.size)
            sends.append(dist.isend(torch.from_numpy(m), above, tag=0))
        if lo:  # downward set of my first owned plane, for the halo above of the slab below
            m = sl.pack_cut(f, g, q, lo, -1)
            sizes.append(m.size)
            sends.append(dist.isend(torch.from_numpy(m), below, tag=1))
        n = sl.pack_cut(f, g, q, 0, +1).size
        if lo:
            buf = torch.empty(n, dtype=torch.float64)
            dist.recv(buf, below, tag=0)
            sl.unpack_cut(buf.numpy(), f, g, q, 0, +1)
        if hi:
            buf = torch.empty(n, dtype=torch.float64)
            dist.recv(buf, above, tag=1)
            sl.unpack_cut(buf.numpy(), f, g, q, lo + own, -1)
        for w in sends:
            w.wait()
    out[rank] = (zs[lo:lo + own], f[:, lo:lo + own], g[:, lo:lo + own], sizes[:1])
    dist.destroy_process_group()


@pytest.mark.timeout(180)
@pytest.mark.parametrize("case", [(10, 8, 12, 15, oracle.BC_CAVITY), (9, 8, 10, 7, 6)],
                         ids=["cavity", "periodic-z"])
def test_two_gloo_ranks_exchange_the_library_cut_messages(case):
    world, steps = 2, 5
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_cut_messages, args=(r, world, port, case, steps, out))
                 for r in range(world)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(150)
            assert pr.exitcode == 0
        res = dict(out)
    nx, ny, nz, q, bc = case
    p = _problem(nx, ny, nz, q, bc)
    F, G = p.run(*_random_state(p, 5), steps)
    seen = []
    for r in range(world):
        zs, f, g, sizes = res[r]
        assert np.array_equal(f, F[:, zs]) and np.array_equal(g, G[:, zs])
        seen += list(zs)
        assert sizes == [(5 + (5 if q == 15 else 1)) * nx * ny]  # a third / a quarter of the plane
    assert sorted(seen) == list(range(nz))


@pytest.mark.parametrize("q", [15, 7])
def test_cut_message_sets_and_round_trip(q):
    sl = _slabs()
    up_f, up_g = sl.cut_populations(q, +1)
    dn_f, dn_g = sl.cut_populations(q, -1)
    ez = oracle.velocities(15)[:, 2]
    assert up_f == [a for a in range(15) if ez[a] == 1] and dn_f == [a for a in range(15) if ez[a] == -1]
    assert up_g == [a for a in up_f if a < q] and dn_g == [a for a in dn_f if a < q]
    rng = np.random.default_rng(2)
    f, g = rng.standard_normal((15, 4, 3, 5)), rng.standard_normal((q, 4, 3, 5))
    msg = sl.pack_cut(f, g, q, 2, -1)
    assert np.array_equal(msg[:15], f[dn_f[0], 2].ravel())
    f2, g2 = np.zeros_like(f), np.zeros_like(g)
    sl.unpack_cut(msg, f2, g2, q, 1, -1)
    assert np.array_equal(f2[dn_f][:, 1], f[dn_f][:, 2]) and np.array_equal(g2[dn_g][:, 1], g[dn_g][:, 2])
    others = [a for a in range(15) if a not in dn_f]
    assert not f2[others].any() and not f2[:, [0, 2, 3]].any()
    from paper_1710_04751_gb300.lbm import LBMError
    with pytest.raises(LBMError):
        sl.pack_cut(f, g, q, 4, +1)  # no plane 4 in a 4-plane slab

