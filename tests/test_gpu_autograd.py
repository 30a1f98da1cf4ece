"""Differentiation through the butterfly apply (GPU).

tb_apply is wrapped in a torch.autograd.Function whose backward is the adjoint
butterfly (the factorization of Eq. butterfly_tensor conjugate-transposed and
traversed in reverse).  For the loss L(f) = ||K f - b||^2 PyTorch's complex
convention gives grad = dL/dRe f + i dL/dIm f = 2 K^H (K f - b), and because L
is quadratic the central difference [L(f + h v) - L(f - h v)] / (2h) equals
Re<grad, v> up to rounding.

Rounding of the complex64 forward (~1e-6 relative per entry) enters the
difference through <error, residual>; along a random direction the derivative
itself is ~1/sqrt(N) of its largest value, so the direction mixes the
normalised gradient with a random part: the derivative is then O(1) and a
wrong backward (a missing conjugate, a transposed factor) still changes it.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_03029_gb300 as tb
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def radon():
    tb.build.build()
    oracle.build()
    torch.cuda.set_device(0)
    w = W.WORKLOADS["radon2d_n256"]
    op = tb.from_workload(w, precisions=(1 << tb.PREC_C64) | (1 << tb.PREC_C128))
    yield w, op
    op.close()


def _loss(op, x, b, precision):
    r = tb.apply(op, x, precision) - b
    return torch.sum(torch.abs(r.to(torch.complex128)) ** 2)


@pytest.mark.parametrize("precision,tol", [(tb.PREC_C64, 1e-4), (tb.PREC_C128, 1e-9)])
def test_central_difference_matches_backward(radon, precision, tol):
    w, op = radon
    dt = tb.dtype_of(precision)
    shape = (w.n,) * w.d + (1,)
    f_true = W.smooth_bumps(w).to(dt).cuda()
    b = op.apply(f_true, precision)
    f = (0.1 * W.complex_gaussian(shape, 5)).to(dt).cuda().requires_grad_()
    L = _loss(op, f, b, precision)
    L.backward()
    g = f.grad.detach()
    # backward == 2 K^H (K f - b) computed directly with the adjoint apply
    with torch.no_grad():
        direct = 2 * op.apply_adjoint(op.apply(f.detach(), precision) - b, precision)
    assert (torch.linalg.vector_norm(g - direct) / torch.linalg.vector_norm(direct)).item() < 1e-6
    rnd = W.random_directions(shape, 7).to(dt).cuda()
    ghat = g / torch.linalg.vector_norm(g)
    v = (ghat + 0.5 * rnd / torch.linalg.vector_norm(rnd)) * torch.linalg.vector_norm(f.detach())
    h = 1e-3
    with torch.no_grad():
        fd = ((_loss(op, f.detach() + h * v, b, precision) - _loss(op, f.detach() - h * v, b, precision))
              / (2 * h)).item()
    an = torch.sum((g.conj() * v).real.to(torch.float64)).item()
    assert abs(fd - an) <= tol * abs(an), f"fd {fd:.8e} analytic {an:.8e}"


def test_backward_is_oracle_adjoint(radon):
    w, op = radon
    shape = (w.n,) * w.d + (1,)
    x = W.complex_gaussian(shape, 11).to(torch.complex64).cuda().requires_grad_()
    u = tb.apply(op, x)
    gu = W.complex_gaussian(shape, 12)                    # seeded upstream gradient
    u.backward(gu.to(torch.complex64).cuda())
    cols = W.sample_targets(w, 512, seed=13)
    ref = oracle.workload_apply_adjoint(w, gu, cols)
    got = x.grad.detach().cpu().to(torch.complex128).numpy().reshape(-1, 1)[cols]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= w.bound


def test_least_squares_inversion_on_device(radon):
    # CGLS on K f = b with the forward and adjoint butterflies, all on the GPU
    w, op = radon
    f_true = W.smooth_bumps(w).to(torch.complex64).cuda()
    b = op.apply(f_true)
    x = torch.zeros_like(f_true)
    r = b.clone()
    s = op.apply_adjoint(r)
    p = s.clone()
    gamma = torch.sum(torch.abs(s) ** 2)
    r0 = torch.linalg.vector_norm(r).item()
    for _ in range(15):
        q = op.apply(p)
        alpha = gamma / torch.sum(torch.abs(q) ** 2)
        x = x + alpha * p
        r = r - alpha * q
        s = op.apply_adjoint(r)
        gnew = torch.sum(torch.abs(s) ** 2)
        p = s + (gnew / gamma) * p
        gamma = gnew
    assert torch.linalg.vector_norm(r).item() < 1e-2 * r0


def _cgls_state(op, b):
    x = torch.zeros_like(b)
    r = b.clone()
    s = op.apply_adjoint(r)
    return {"x": x, "r": r, "p": s.clone(), "gamma": torch.sum(torch.abs(s) ** 2)}


def _cgls_step(op, st):
    # one CGLS iteration on K f = b, in place on the state tensors
    q = op.apply(st["p"])
    alpha = st["gamma"] / torch.sum(torch.abs(q) ** 2)
    st["x"].add_(alpha * st["p"])
    st["r"].sub_(alpha * q)
    s = op.apply_adjoint(st["r"])
    gnew = torch.sum(torch.abs(s) ** 2)
    st["p"].mul_(gnew / st["gamma"]).add_(s)
    st["gamma"].copy_(gnew)


def test_least_squares_iterations_replay_as_one_cuda_graph(radon):
    """Device-resident inversion: one CGLS iteration (forward butterfly, adjoint
    butterfly and the vector updates) is captured once as a CUDA graph and
    replayed; it reproduces the eager iterations and reduces the residual."""
    w, op = radon
    f_true = W.smooth_bumps(w).to(torch.complex64).cuda()
    b = op.apply(f_true)
    iters = 15
    eager = _cgls_state(op, b)
    for _ in range(iters):
        _cgls_step(op, eager)
    st = _cgls_state(op, b)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        _cgls_step(op, st)                       # warm-up iteration (kernel attributes, workspaces)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        _cgls_step(op, st)
    for _ in range(iters - 1):                   # capturing does not execute the step
        g.replay()
    torch.cuda.synchronize()
    r0 = torch.linalg.vector_norm(b).item()
    assert torch.linalg.vector_norm(st["r"]).item() < 1e-2 * r0
    assert (torch.linalg.vector_norm(st["x"] - eager["x"]) / torch.linalg.vector_norm(eager["x"])).item() < 1e-4


def test_cgls_library_call_graph_and_eager(radon):
    """tb_cgls: the least-squares solve as one library call, device-resident.
    The graph-replayed and the eager iterations run the same kernels in the same
    order (bit-identical), agree with the torch-driven iterations above, and the
    recorded residual history starts at ||b||, never increases and ends below
    1e-2 ||b|| after 15 iterations."""
    w, op = radon
    f_true = W.smooth_bumps(w).to(torch.complex64).cuda()
    b = op.apply(f_true)
    iters = 15
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        xg, rg = op.cgls(b, iters, graph=True)
        xe, re_ = op.cgls(b, iters, graph=False)
    side.synchronize()
    assert torch.equal(xg, xe) and np.array_equal(rg, re_)
    ref = _cgls_state(op, b)
    for _ in range(iters):
        _cgls_step(op, ref)
    assert (torch.linalg.vector_norm(xg - ref["x"]) / torch.linalg.vector_norm(ref["x"])).item() < 1e-4
    bn = torch.linalg.vector_norm(b.to(torch.complex128)).item()
    assert abs(rg[0, 0] - bn) <= 1e-6 * bn
    assert np.all(np.diff(rg[:, 0]) <= 1e-6 * bn)
    assert rg[-1, 0] < 1e-2 * bn
    # the last recorded residual is the residual of the returned iterate
    true_r = torch.linalg.vector_norm((b - op.apply(xg)).to(torch.complex128)).item()
    assert abs(true_r - rg[-1, 0]) <= 1e-3 * rg[-1, 0] + 1e-6 * bn


def test_cgls_columns_are_independent(radon):
    """Several RHS columns solve independent systems: each column of a 3-column
    solve equals the 1-column solve of that column, and a zero column stays zero
    (alpha = beta = 0, no NaN)."""
    w, op = radon
    f_true = W.smooth_bumps(w).to(torch.complex64).cuda()
    b1 = op.apply(f_true)
    b3 = torch.cat([b1, 2.5j * b1, torch.zeros_like(b1)], dim=-1).contiguous()
    x3, r3 = op.cgls(b3, 8)
    x1, r1 = op.cgls(b1, 8)
    assert (torch.linalg.vector_norm(x3[..., :1] - x1) / torch.linalg.vector_norm(x1)).item() < 1e-5
    assert (torch.linalg.vector_norm(x3[..., 1:2] - 2.5j * x1) / torch.linalg.vector_norm(x1)).item() < 1e-5
    assert torch.count_nonzero(x3[..., 2]).item() == 0 and np.all(r3[:, 2] == 0)
    assert np.allclose(r3[:, 0], r1[:, 0], rtol=1e-5)
