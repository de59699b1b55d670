"""The x-strip decomposition's bookkeeping on CPU ranks (gloo, world size 2
and 3): strip geometry (`decomp.split_columns`, `strip_case`), the rate
all-reduce and the halo send/receive of `decomp.exchange_dist`, driven with
stand-in strips that step their columns with the FP64 oracle (dt from the
exchanged rate, levels of their own columns).  The assembled owned columns
must equal the oracle's run of the undivided grid bit for bit: the stencil
reaches two columns, the levels of Eq. (Free_surf_detector) are column sums,
and dt is the largest signal rate over the grid (reading R-cfl)."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleStrip:
    """The strip protocol of decomp.Strip on host tensors, stepped by the
    oracle: test infrastructure only."""

    def __init__(self, case, a, b):
        from paper_1806_04960_gb300 import decomp
        self.grid_case = case
        self.lo, self.hi, self.own_lo, self.own_hi = decomp.strip_extent(case.nx, a, b)
        self.case = decomp.strip_case(case, a, b)
        self.q = self.case.q.copy()
        self.has_w = self.lo < a
        self.has_e = self.hi > b
        self.rate = None

    def halo_buffer(self):
        import torch
        return torch.zeros(4 * self.case.ny * 2, dtype=torch.float64)

    def own_rate(self, all_columns=False):
        """Largest (|u| + c)/dx + (|v| + c)/dy over the owned (or all) fluid
        cells, in the oracle's operation order."""
        c = self.case
        cols = slice(None) if all_columns else slice(self.own_lo, self.own_hi)
        q = self.q[:, :, cols]
        fl = c.solid[:, cols] == 0
        cs = math.sqrt(c.gamma * c.k0 / c.rho0)
        u = q[1][fl] / q[0][fl]
        v = q[2][fl] / q[0][fl]
        r = (np.abs(u) + cs) / c.dx + (np.abs(v) + cs) / c.dy
        return float(r.max()) if r.size else 0.0

    def rate_into(self, buf):
        buf[0] = self.own_rate(all_columns=self.rate is None)

    def set_rate(self, rates):
        self.rate = float(rates.max())

    def step(self, cfl):
        from oracle import oracle as O
        dt = cfl / self.rate
        _, K = O.dt_levels(self.case, q=self.q)
        self.q, _, _, _ = O.run_record(self.case, 1, [0], q=self.q, dt_fix=[dt], K_fix=[K])

    def pack(self, side, buf):
        c0 = self.own_lo if side == 0 else self.own_hi - 2
        buf.copy_(__import__("torch").from_numpy(np.ascontiguousarray(self.q[:, :, c0:c0 + 2]).ravel()))

    def unpack(self, side, buf):
        c0 = 0 if side == 0 else self.own_hi
        self.q[:, :, c0:c0 + 2] = buf.numpy().reshape(4, self.case.ny, 2)


def _rank_main(rank, world, port, out_path, steps, cfl):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_1806_04960_gb300 import cases, decomp
    dist.init_process_group("gloo", rank=rank, world_size=world)
    case = cases.perturbed(cases.c1(), 3)
    a, b = decomp.split_columns(case.nx, world)[rank]
    strip = OracleStrip(case, a, b)
    rate = torch.zeros(1, dtype=torch.float64)
    send = {k: strip.halo_buffer() for k in (0, 1) if (strip.has_w, strip.has_e)[k]}
    recv = {k: strip.halo_buffer() for k in send}
    # after loading the state: rates over all held columns (true values), once
    strip.rate_into(rate)
    dist.all_reduce(rate, op=dist.ReduceOp.MAX)
    strip.set_rate(rate)
    for _ in range(steps):
        strip.step(cfl)
        decomp.exchange_dist(strip, rank, world, dist, rate, send, recv)
    np.save(f"{out_path}.{rank}.npy", strip.q[:, :, strip.own_lo:strip.own_hi])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_strip_exchange_reproduces_the_undivided_grid(tmp_path, world):
    import socket
    import torch.multiprocessing as mp
    from oracle import oracle as O
    from paper_1806_04960_gb300 import cases
    steps, cfl = 12, 0.45
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "q")
    mp.start_processes(_rank_main, args=(world, port, out, steps, cfl), nprocs=world, join=True,
                       start_method="spawn")
    got = np.concatenate([np.load(f"{out}.{r}.npy") for r in range(world)], axis=2)
    case = cases.perturbed(cases.c1(), 3)
    ref, _, _, _ = O.run(case, steps, cfl=cfl)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)


def test_split_and_strip_geometry():
    from paper_1806_04960_gb300 import cases, decomp
    assert decomp.split_columns(10, 3) == [(0, 3), (3, 7), (7, 10)]
    with pytest.raises(ValueError):
        decomp.split_columns(5, 3)
    c = cases.c1()
    lo, hi, ol, oh = decomp.strip_extent(c.nx, 40, 90)
    assert (lo, hi, ol, oh) == (38, 92, 2, 52)
    s = decomp.strip_case(c, 40, 90)
    assert s.nx == 54 and s.x0 == c.x0 + 38 * c.dx and s.sides == (0, 0, 0, 0)
    assert np.array_equal(s.q, c.q[:, :, 38:92]) and np.array_equal(s.solid, c.solid[:, 38:92])
    t = decomp.strip_case(cases.dambreak(16, 8, sides=(1, 1, 0, 0)), 8, 16)
    assert t.sides == (0, 1, 0, 0) and t.nx == 10
