"""The partitioned (sharded) apply on CPU ranks: the driver
paper_2411_03029_gb300.sharded_apply over a gloo process group.

Steps 1 and 3 of Alg. 2 are independent per mid-level multi-set (Sec. 3.2):
rank g runs steps 1-2 for its range S_g of source multi-sets, the mid-level
tiles (t, s) move to the owner of t, and rank g runs step 3 for its range
T_g.  On a GPU the halves are tb_apply_src_part / tb_apply_tgt_part; here,
with no GPU, the step-by-step oracle's halves (oracle/butterfly.py
source_part / target_part) stand in for them behind the same interface, on a
synthetic butterfly in the export format, so that the partition plan
(tb_shard_plan), the layout of the exchanged tiles and the point-to-point
exchange are what is tested.  Every output point is computed by exactly one
rank with the same arithmetic as the single-rank apply, so the sum of the
ranks' outputs equals the single-rank result bit for bit.
"""
import os
import socket
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleHalves:
    """The interface sharded_apply uses (mid_shape, apply_src_part, apply_tgt_part),
    with the step-by-step oracle as the engine and the exchanged tensor in the
    layout of tb_apply_src_part: (nF, nF, prod padded ranks, nv), tile (t, s),
    entries C order over the padded target ranks, compact entries at the front
    of each mode."""

    def __init__(self, bf):
        from oracle import butterfly as O2
        self.O2, self.bf = O2, bf
        self.d, self.Lc = bf["d"], bf["Lc"]
        self.n = list(bf["n"])
        self.nF = 1 << (self.d * self.Lc)
        self.R = [bf["factors"][(1, self.Lc, k)]["blocks"].shape[1] for k in range(self.d)]

    def mid_shape(self, nv):
        return (self.nF, self.nF, int(np.prod(self.R)), nv)

    def apply_src_part(self, f, g_mid, s_range, precision=None):
        G = self.O2.source_part(self.bf, f.numpy(), s_range)
        for (t, s), X in G.items():
            tile = np.zeros(tuple(self.R) + (X.shape[-1],), dtype=np.complex128)
            tile[tuple(slice(0, r) for r in X.shape[:-1])] = X
            g_mid[t, s] = torch.from_numpy(tile.reshape(-1, X.shape[-1]))
        return g_mid

    def apply_tgt_part(self, g_mid, u, t_range, precision=None):
        G = {}
        dims = self.bf["core_dims"]
        for t in range(int(t_range[0]), int(t_range[1])):
            for s in range(self.nF):
                rt = [int(v) for v in dims[t * self.nF + s][: self.d]]
                tile = g_mid[t, s].numpy().reshape(tuple(self.R) + (g_mid.shape[-1],))
                G[(t, s)] = tile[tuple(slice(0, r) for r in rt)]
        out = u.numpy()
        self.O2.target_part(self.bf, G, t_range, out=out)
        return u


def _worker(rank, ws, port, q, case):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import paper_2411_03029_gb300 as tb
    from oracle import butterfly as O2
    from test_oracle_butterfly import synthetic
    d, L, cb, R = case
    bf = synthetic(d, L, cb, R, seed=31 + d + L)      # every rank builds the same butterfly
    n = cb << L
    rng = np.random.default_rng(5)
    f = rng.standard_normal((n,) * d + (2,)) + 1j * rng.standard_normal((n,) * d + (2,))
    u = tb.sharded_apply(OracleHalves(bf), torch.from_numpy(f))
    dist.all_reduce(torch.view_as_real(u))             # each target point is set on one rank only
    ref = O2.apply(bf, f)
    q.put((rank, bool(np.array_equal(u.numpy(), ref)), float(np.abs(u.numpy() - ref).max())))
    dist.destroy_process_group()


def _run(ws, case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q, case)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(ws))
    assert [r for r, _, _ in res] == list(range(ws))
    assert all(ok for _, ok, _ in res), res


def test_two_ranks_reproduce_the_single_rank_apply_bit_for_bit():
    _run(2, (2, 4, 1, 2))     # d = 2, L = 4: 16 mid-level multi-sets per side


def test_three_ranks_with_uneven_ranges():
    _run(3, (3, 2, 2, 2))     # d = 3, L = 2: 8 mid-level multi-sets, ranges 2/3/3


def test_shard_plan_covers_every_multiset_once():
    sys.path.insert(0, ROOT)
    import paper_2411_03029_gb300 as tb
    for nmid, nr in ((16, 2), (8, 3), (4096, 7), (5, 8)):
        plan = tb.shard_plan(nmid, nr)
        assert plan[0][0] == 0 and plan[-1][1] == nmid
        assert all(plan[g][1] == plan[g + 1][0] for g in range(nr - 1))
        sizes = [e - b for b, e in plan]
        assert max(sizes) - min(sizes) <= 1
