"""The slab split of the finest level across ranks (paper_1903_10367_gb300/
partition.py; Sec. 4.3 and 5.5 "Parallel adAFAC") on CPU.

Two gloo processes (127.0.0.1) each own a slab of fine planes and keep every
coarser level in full.  Per cycle they exchange the halo planes of the
iterate once and sum their partial level-(L-1) vectors (the restricted
residual and the damping right-hand side) once; every other step runs on
the rank's own data.  The assembled iterate equals the oracle's cycle on the
whole grid (Alg. 1, Eq. 9) to rounding."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1903_10367_gb300 import partition  # noqa: E402

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def test_slabs_cover_the_interior_planes_once():
    for n, world in [(27, 2), (81, 3), (243, 8), (9, 8)]:
        slabs = partition.plan(n, world)
        planes = [z for s in slabs for z in s.planes]
        assert planes == list(range(1, n))
        for s in slabs:
            # the residual of plane z reads z - 1 .. z + 1: the halo holds the
            # neighbours' planes next to the slab, never a boundary plane
            assert set(s.halo) == {z for z in (s.z0 - 1, s.z1) if 1 <= z <= n - 1}
            # a coarse plane m is shared when its window 3m-2 .. 3m+2 meets
            # this slab and another one
            for m in range(1, n // 3):
                window = set(range(3 * m - 2, 3 * m + 3)) & set(range(1, n))
                mine = window & set(s.planes)
                others = window - set(s.planes)
                assert (m in s.coarse_shared) == (bool(mine) and bool(others))
    with pytest.raises(ValueError):
        partition.plan(28, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _slab_cycle(H, u, slab, exchange, allreduce):
    """One adAFAC-Jac cycle (CS form, truncated R~) computed by one rank from
    its slab: the oracle's level operations on arrays that hold the rank's
    planes (and the halo), the partial sums combined by `allreduce`."""
    from oracle import cycle as oc
    from oracle import fem
    L = H.L
    own = np.zeros(u.shape, dtype=bool)
    own[slab.z0:slab.z1] = True           # axis 0 is z
    local = np.where(own, u, 0.0)
    exchange(local)                       # halo planes from the neighbours
    r = np.where(own, oc.residual(H, L, local, H.b), 0.0)
    # partial restriction and damping right-hand side of level L - 1
    part = np.stack([oc.R(H, L, r), oc.Rtilde(H, L, r, oc.OMEGA, "truncated")])
    full = allreduce(part)
    rl = {L: r, L - 1: full[0]}
    for l in range(L - 2, 0, -1):
        rl[l] = oc.R(H, l + 1, rl[l + 1])
    c = {l: oc.jacobi_correction(H, l, rl[l], oc.OMEGA) for l in range(1, L + 1)}
    bt = {L - 1: full[1]}
    for l in range(L - 1, 1, -1):
        bt[l - 1] = oc.Rtilde(H, l, rl[l], oc.OMEGA, "truncated")
    du = c[L].copy()
    for l in range(1, L):
        du += oc.P_pow(H, l, L, c[l])
    for l in range(1, L):
        du -= oc.P_pow(H, l, L, oc.jacobi_correction(H, l, bt[l], oc.OMEGA_TILDE))
    return np.where(own, u + fem.zero_boundary(du), 0.0)


def _rank(rank, world, port, out):
    import workloads as wl
    from oracle import cycle as oc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d, L = 3, 3
        n = 3 ** L
        eps = np.random.default_rng(4).uniform(0.2, 3.0, size=(n,) * d)
        H = oc.build_hierarchy(d, L, eps, False, wl.manufactured_rhs(d, L))
        u0 = wl.random_vertex_field(d, L, 9)
        slabs = partition.plan(n, world)
        me = slabs[rank]
        owner = {z: s.rank for s in slabs for z in s.planes}
        sent = [0]

        def exchange(a):
            reqs = []
            recv = {}
            for s in slabs:
                for z in s.halo:
                    if owner[z] == rank:            # a neighbour needs my plane z
                        t = torch.from_numpy(np.ascontiguousarray(a[z]))
                        reqs.append(dist.isend(t, dst=s.rank))
                        sent[0] += t.numel() * 8
                    elif s.rank == rank:            # I need plane z
                        recv[z] = torch.empty(a.shape[1:], dtype=torch.float64)
                        reqs.append(dist.irecv(recv[z], src=owner[z]))
            for q in reqs:
                q.wait()
            for z, t in recv.items():
                a[z] = t.numpy()

        def allreduce(part):
            t = torch.from_numpy(np.ascontiguousarray(part))
            dist.all_reduce(t)
            return t.numpy()

        u = _slab_cycle(H, u0, me, exchange, allreduce)
        mine = torch.from_numpy(np.ascontiguousarray(u))
        dist.all_reduce(mine)                       # disjoint slabs: the sum assembles
        out.put((rank, mine.numpy(), oc.cycle(H, u0), sent[0], me.halo))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_one_oracle_cycle_of_the_whole_grid():
    import torch.multiprocessing as mp
    if not dist.is_gloo_available():
        pytest.skip("gloo backend not built")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, want, sent, halo in res:
        scale = np.abs(want).max()
        interior = got[1:-1, 1:-1, 1:-1]
        assert np.abs(interior - want[1:-1, 1:-1, 1:-1]).max() <= 1e-12 * scale, rank
        # one plane of (3^3 + 1)^2 values goes each way across the single cut
        assert halo and sent == 28 * 28 * 8
