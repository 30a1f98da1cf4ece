"""tb_apply_src_part / tb_apply_tgt_part on one GPU: the ranks of a
partitioned apply run one after another (no kernel waits on another), each
with its own mid-level buffer, and the exchange of mid-level tiles is done
with device copies between the buffers.  Every unit is computed by the same
kernels with the same arithmetic as in the whole apply, so the assembled
result equals tb_apply bit for bit (per-mode level launches on both sides)."""
import pytest
import torch

import paper_2411_03029_gb300 as tb
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    tb.build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("name,w", [("helmholtz3d_n32", W.small("helmholtz3d_n64", 32, nv=3, L=2)),
                                    ("radon2d_n64_L4", W.small("radon2d_n256", 64, nv=1, L=4))])
@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_apply_equals_tb_apply(name, w, world):
    op = tb.from_workload(w, precisions=(1 << tb.PREC_C64) | (1 << tb.PREC_C128),
                          level_schedule=tb.LEVEL_PER_MODE)
    for prec in (tb.PREC_C64, tb.PREC_C128):
        f = W.rhs(w).to(tb.dtype_of(prec)).cuda()
        ref = op.apply(f, prec)
        shape = op.mid_shape(w.nv)
        plan = tb.shard_plan(shape[0], world)
        mids = [torch.zeros(shape, dtype=f.dtype, device="cuda") for _ in range(world)]
        for g in range(world):                       # steps 1-2 of each rank
            op.apply_src_part(f, mids[g], plan[g], prec)
        for g in range(world):                       # tile (t, s): owner of s -> owner of t
            for h in range(world):
                if g != h:
                    (t0, t1), (s0, s1) = plan[h], plan[g]
                    mids[h][t0:t1, s0:s1] = mids[g][t0:t1, s0:s1]
        u = torch.zeros_like(f)
        for g in range(world):                       # step 3 of each rank
            part = torch.zeros_like(f)
            op.apply_tgt_part(mids[g], part, plan[g], prec)
            u += part
        torch.cuda.synchronize()
        assert torch.equal(u, ref), (prec, (u - ref).abs().max().item())
    op.close()


def test_partitioned_apply_rejects_what_it_does_not_cover():
    w = W.small("helmholtz3d_n64", 16, nv=1, L=2)
    op = tb.from_workload(w, precisions=(1 << tb.PREC_C64) | (1 << tb.PREC_C64_SPLITBF16))
    f = W.rhs(w).to(torch.complex64).cuda()
    g = torch.zeros(op.mid_shape(1), dtype=torch.complex64, device="cuda")
    with pytest.raises(tb.TBError) as e:
        op.apply_src_part(f, g, (0, 2), tb.PREC_C64_SPLITBF16)
    assert e.value.status == 6
    with pytest.raises(tb.TBError) as e:
        op.apply_src_part(f, g, (0, 10 ** 6), tb.PREC_C64)
    assert e.value.status == 1
    op.close()
