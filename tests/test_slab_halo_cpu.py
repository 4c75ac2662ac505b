"""One solve split into x slabs over CPU ranks (gloo, world size 2) that
exchange halos every step: the result is bit-identical to the unsplit solve
(the per-cell update is the oracle's; only the crossing populations move).
A rank that dies between steps is detected by the survivor as a missing halo
within the process-group timeout -- failure detection on the host, no GPU.
"""
import os
import sys
import datetime

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _case(lattice):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1710_02065_gb300 import inputs
    if lattice == oracle.D2Q9:
        n = (40, 18)
    else:
        n = (24, 12, 10)
    P = oracle.Problem(lattice, n, 0.58)
    P.set_boundary(2, oracle.VELOCITY, (0.03, 0.0, 0.0))
    P.set_boundary(3, oracle.OUTFLOW)
    P.set_sponge(3, 4, 0.4, 1.0, (0.0, 0.0, 0.0))
    shape = tuple(reversed(P.n[:2 if lattice == oracle.D2Q9 else 3]))
    solid = np.zeros(shape, np.uint8)
    if lattice == oracle.D2Q9:
        solid[6:9, 18:23] = 1
    else:
        solid[4:6, 5:7, 9:13] = 1
    P.solid = solid.reshape(-1)
    _, _, _, w, _ = oracle.lattice(lattice)
    f0 = inputs.random_populations(w, P.ncell, 19, 0.06)
    return P, f0


def _rank(rank, world, port, lattice, steps, die_at, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1710_02065_gb300 import slabs
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=6))
    P, f = _case(lattice)
    nx = P.n[0]
    _, qn, xi, _, _ = oracle.lattice(lattice)
    x0, x1 = slabs.slab_ranges(nx, world)[rank]
    right, left = slabs.crossing_directions(xi)
    F = f.reshape(qn, -1, nx).copy()  # (q, rows, nx)
    rows = F.shape[1]
    owned = np.array([r * nx + x for r in range(rows) for x in range(x0, x1)], dtype=np.int64)
    nb_r, nb_l = (rank + 1) % world, (rank - 1) % world
    try:
        for t in range(steps):
            if rank == 1 and t == die_at:
                raise SystemExit(7)  # this rank leaves between steps
            # halo: my last column's right-movers to the right neighbour, my
            # first column's left-movers to the left neighbour
            send_r = torch.from_numpy(np.ascontiguousarray(F[right][:, :, x1 - 1]))
            send_l = torch.from_numpy(np.ascontiguousarray(F[left][:, :, x0]))
            recv_l = torch.empty_like(send_r)
            recv_r = torch.empty_like(send_l)
            reqs = [dist.isend(send_r, nb_r, tag=1), dist.isend(send_l, nb_l, tag=2),
                    dist.irecv(recv_l, nb_l, tag=1), dist.irecv(recv_r, nb_r, tag=2)]
            for rq in reqs:
                rq.wait()
            F[np.ix_(right, np.arange(rows), [(x0 - 1) % nx])] = recv_l.numpy()[:, :, None]
            F[np.ix_(left, np.arange(rows), [x1 % nx])] = recv_r.numpy()[:, :, None]
            out = P.update_cells(F.reshape(qn, -1), owned, step=t)  # (cells, q)
            Fn = F.reshape(qn, -1).copy()
            Fn[:, owned] = out.T
            F = Fn.reshape(qn, rows, nx)
        # gather the slabs on rank 0
        mine = torch.from_numpy(np.ascontiguousarray(F[:, :, x0:x1]))
        if rank == 0:
            parts = [mine.numpy()]
            for r in range(1, world):
                a, b = slabs.slab_ranges(nx, world)[r]
                buf = torch.empty((qn, rows, b - a), dtype=torch.float64)
                dist.recv(buf, r, tag=9)
                parts.append(buf.numpy())
            q.put((rank, "ok", np.concatenate(parts, axis=2).reshape(qn, -1)))
        else:
            dist.send(mine, 0, tag=9)
            q.put((rank, "ok", None))
    except RuntimeError as e:  # a halo or the gather did not arrive in time
        q.put((rank, "lost neighbour", str(e)[:200]))
        q.close()
        q.join_thread()  # deliver the message before leaving
        os._exit(3)
    dist.destroy_process_group()


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run(lattice, steps, die_at=-1):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, lattice, steps, die_at, q)) for r in range(2)]
    for p in procs:
        p.start()
    # drain the queue while the ranks run: a child cannot exit while its
    # large result still sits in the pipe
    import queue as _queue
    import time
    out, t0 = {}, time.time()
    while time.time() - t0 < 180:
        try:
            r, status, payload = q.get(timeout=0.5)
            out[r] = (status, payload)
        except _queue.Empty:
            if not any(p.is_alive() for p in procs):
                break
    for p in procs:
        p.join(30)
    codes = [p.exitcode for p in procs]
    return codes, out


@pytest.mark.parametrize("lattice", [0, 1])
def test_two_slabs_match_the_unsplit_solve_bit_for_bit(lattice):
    sys.path.insert(0, ROOT)
    P, f = _case(lattice)
    steps = 6
    ref = P.run(f, steps)
    codes, out = _run(lattice, steps)
    assert codes == [0, 0], codes
    assert out[0][0] == "ok"
    assert np.array_equal(out[0][1], ref)


def test_slab_plan():
    from paper_1710_02065_gb300 import slabs
    sys.path.insert(0, ROOT)
    import oracle
    assert slabs.slab_ranges(10, 3) == [(0, 3), (3, 6), (6, 10)]
    for lat, per_face in ((oracle.D2Q9, 3), (oracle.D3Q19, 5), (oracle.D3Q27, 9)):
        _, _, xi, _, _ = oracle.lattice(lat)
        right, left = slabs.crossing_directions(xi)
        assert len(right) == len(left) == per_face
    # the round jet split in two: 5 + 5 FP32 populations per face cell
    _, _, xi, _, _ = oracle.lattice(oracle.D3Q19)
    assert slabs.halo_bytes_per_step((384, 256, 256), xi, 4) == 10 * 256 * 256 * 4


def test_a_rank_that_leaves_is_detected_by_its_neighbour():
    codes, out = _run(0, 6, die_at=2)
    assert codes[1] == 7          # the leaving rank
    assert codes[0] == 3          # the survivor saw its halo missing and stopped
    assert out[0][0] == "lost neighbour"
