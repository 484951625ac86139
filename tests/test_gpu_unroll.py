"""Unrolled PDHG and its adjoint on the GPU (pdlp_unroll / pdlp_grad) against
the oracle's unrolled map and reverse mode, central finite differences of
the oracle's forward map, the envelope gradients at an optimum, and the
torch.autograd.Function wrapper."""
import copy

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle
import paper_2106_04756_gb300 as P

pytestmark = pytest.mark.gpu


def _shifted(lp, seed):
    # c shifted off the planted optimum so no coordinate starts on a kink
    lp = copy.deepcopy(lp)
    lp.c = lp.c + 0.05 * np.random.default_rng(seed).standard_normal(lp.n)
    return lp


CASES = {
    "planted_25x40": lambda: _shifted(lpgen.planted_uniform(25, 40, 0.2, frac_boxed=0.7, seed_key=(60,)), 60),
    "mip_2000x5000": lambda: _shifted(lpgen.mip_like(2000, 5000, 30000, seed_key=(71,)), 71),
}


def _omega(lp, ruiz=10, pc=1):
    return oracle.unroll_schedule(lp, 1, ruiz_iters=ruiz, pock_chambolle=pc)[1]


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("persistent", [1, 0, 2])
@pytest.mark.parametrize("name", sorted(CASES))
def test_unrolled_map_matches_oracle(gpu_lib, oracle_lib, name, persistent):
    lp = CASES[name]()
    T = 120  # three checkpoint segments of 50, the last one ragged
    with P.Context.from_lp(lp, persistent=persistent) as ctx:
        x, y, eta = ctx.unroll(T, 50)
    assert eta.shape == (T,) and np.all(eta > 0)
    # the same map replayed by the oracle with the recorded step sizes
    x2, y2 = oracle.unroll_forward(lp, eta, _omega(lp))
    assert _rel(x, x2) <= 1e-10 and _rel(y, y2) <= 1e-10
    # the adaptive schedule itself: the oracle's, up to rounding, over the first steps
    eta_o = oracle.unroll_schedule(lp, 20)[0]
    assert np.allclose(eta[:20], eta_o, rtol=1e-9, atol=0)


@pytest.mark.parametrize("name", sorted(CASES))
def test_grad_matches_oracle_reverse_mode(gpu_lib, oracle_lib, name):
    lp = CASES[name]()
    T = 120
    rng = np.random.default_rng(5)
    gx, gy = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
    with P.Context.from_lp(lp) as ctx:
        _, _, eta = ctx.unroll(T, 50)
        dc, dq, dK = ctx.grad(gx, gy)
        dc1, dq1, dK1 = ctx.grad(gx, None)  # dL/dy_T absent
    rc, rq, rk = oracle.unroll_vjp(lp, eta, _omega(lp), gx, gy)
    assert _rel(dc, rc) <= 1e-9 and _rel(dq, rq) <= 1e-9 and _rel(dK, rk) <= 1e-9
    rc1, rq1, rk1 = oracle.unroll_vjp(lp, eta, _omega(lp), gx, None)
    assert _rel(dc1, rc1) <= 1e-9 and _rel(dq1, rq1) <= 1e-9 and _rel(dK1, rk1) <= 1e-9


@pytest.mark.parametrize("ruiz,pc,dirs", [(0, 0, "cqK"), (10, 1, "cq")])
def test_grad_matches_central_differences(gpu_lib, oracle_lib, ruiz, pc, dirs):
    # FD of the float64 oracle forward at the recorded schedule, h = 1e-6; the
    # preconditioner is frozen, so K directions are taken without it
    # (T = 40: no coordinate of this trajectory passes within h of a kink,
    # which the oracle's own FD check confirms; at T = 60 one does)
    lp = CASES["planted_25x40"]()
    T = 40
    rng = np.random.default_rng(11)
    gx, gy = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
    with P.Context.from_lp(lp, ruiz_iters=ruiz, pock_chambolle=pc) as ctx:
        _, _, eta = ctx.unroll(T, 15)
        dc, dq, dK = ctx.grad(gx, gy)
    omega = _omega(lp, ruiz, pc)

    def loss(c, q, val):
        lp2 = copy.copy(lp)
        lp2.c, lp2.q, lp2.val = c, q, val
        x, y = oracle.unroll_forward(lp2, eta, omega, ruiz_iters=ruiz, pock_chambolle=pc)
        return gx @ x + gy @ y

    h = 1e-6
    for _ in range(4):
        vc, vq = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
        vk = rng.standard_normal(lp.nnz) if "K" in dirs else np.zeros(lp.nnz)
        fd = (loss(lp.c + h * vc, lp.q + h * vq, lp.val + h * vk) -
              loss(lp.c - h * vc, lp.q - h * vq, lp.val - h * vk)) / (2 * h)
        an = dc @ vc + dq @ vq + dK @ vk
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_envelope_gradients_after_convergence(gpu_lib):
    # unique vertex optimum; started at it, the unrolled map stays there and
    # L = c^T x_T has dL/dq = y*, dL/dc = x*, dL/dK_ij = -y*_i x*_j
    rng = np.random.default_rng(12)
    m, n = 6, 10
    A = rng.standard_normal((m, n))
    ineq = np.array([1, 1, 1, 0, 0, 0], np.uint8)
    l, u = np.zeros(n), np.full(n, 4.0)
    x = np.zeros(n)
    x[:6] = rng.uniform(1, 3, 6)
    x[8:] = 4.0
    lam = np.zeros(n)
    lam[6:8] = rng.uniform(0.5, 1, 2)
    lam[8:] = -rng.uniform(0.5, 1, 2)
    y = np.concatenate([rng.uniform(0.5, 1, 3), rng.standard_normal(3)])
    q, c = A @ x, A.T @ y + lam
    Asp = sp.csr_matrix(A)
    lp = lpgen.LP(m=m, n=n, row_ptr=Asp.indptr.astype(np.int32), col_idx=Asp.indices.astype(np.int32),
                  val=Asp.data, c=c, q=q, l=l, u=u, ineq=ineq)
    with P.Context.from_lp(lp, ruiz_iters=0, pock_chambolle=0) as ctx:
        xT, yT, _ = ctx.unroll(30000, 200, x0=x, y0=y)
        dc, dq, dK = ctx.grad(c, None)
    assert np.allclose(xT, x, atol=1e-10)
    assert np.allclose(dq, y, atol=1e-6)
    assert np.allclose(dc + xT, x, atol=1e-6)
    rows = np.repeat(np.arange(m), np.diff(lp.row_ptr))
    assert np.allclose(dK, -y[rows] * x[lp.col_idx], atol=1e-6)


def test_grad_at_20k_x_50k_matches_oracle(gpu_lib, oracle_lib):
    # 20k x 50k, about 300k nonzeros, loss 1/2 ||x_T - x_target||^2
    lp = _shifted(lpgen.unroll_20k(), 4)
    T = 200
    with P.Context.from_lp(lp) as ctx:
        x, y, eta = ctx.unroll(T, 50)
        target = np.random.default_rng(4).standard_normal(lp.n)
        dc, dq, dK = ctx.grad(x - target, None)
    omega = _omega(lp)
    x2, _ = oracle.unroll_forward(lp, eta, omega)
    assert _rel(x, x2) <= 1e-9
    rc, rq, rk = oracle.unroll_vjp(lp, eta, omega, x - target, None)
    assert _rel(dc, rc) <= 1e-8 and _rel(dq, rq) <= 1e-8 and _rel(dK, rk) <= 1e-8


def test_autograd_function_backward_is_pdlp_grad(gpu_lib):
    import torch
    from paper_2106_04756_gb300.autograd import unrolled_pdhg
    lp = CASES["mip_2000x5000"]()
    dev = "cuda"
    t = lambda a, dt=torch.float64: torch.as_tensor(np.asarray(a)).to(dev, dt)
    c = t(lp.c).requires_grad_()
    q = t(lp.q).requires_grad_()
    kv = t(lp.val).requires_grad_()
    target = t(np.random.default_rng(3).standard_normal(lp.n))
    x, y = unrolled_pdhg(c, q, kv, t(lp.row_ptr, torch.int32), t(lp.col_idx, torch.int32), t(lp.l), t(lp.u),
                         t(lp.ineq, torch.uint8), 80, 40)
    loss = 0.5 * ((x - target) ** 2).sum()
    loss.backward()
    with P.Context.from_lp(lp) as ctx:
        x2, _, _ = ctx.unroll(80, 40)
        dc, dq, dK = ctx.grad(x2 - target.cpu().numpy(), None)
    assert np.array_equal(x.detach().cpu().numpy(), x2)
    assert np.array_equal(c.grad.cpu().numpy(), dc)
    assert np.array_equal(q.grad.cpu().numpy(), dq)
    assert np.array_equal(kv.grad.cpu().numpy(), dK)


def test_autograd_backward_twice_and_shared_context(gpu_lib):
    """The autograd node keeps its library context: backward runs twice with
    retain_graph (the same gradient both times), and with a caller's shared
    context, a second forward on that context before the first node's
    backward does not change the first node's gradient (the backward repeats
    its unroll)."""
    import torch
    from paper_2106_04756_gb300.autograd import unrolled_pdhg
    lp = CASES["mip_2000x5000"]()
    dev = "cuda"
    t = lambda a, dt=torch.float64: torch.as_tensor(np.asarray(a)).to(dev, dt)
    args = lambda c, q, kv: (c, q, kv, t(lp.row_ptr, torch.int32), t(lp.col_idx, torch.int32), t(lp.l), t(lp.u),
                             t(lp.ineq, torch.uint8))
    target = t(np.random.default_rng(5).standard_normal(lp.n))
    c = t(lp.c).requires_grad_()
    q = t(lp.q).requires_grad_()
    kv = t(lp.val).requires_grad_()
    x, _ = unrolled_pdhg(*args(c, q, kv), 60, 20)
    loss = 0.5 * ((x - target) ** 2).sum()
    loss.backward(retain_graph=True)
    g1 = [a.grad.clone() for a in (c, q, kv)]
    for a in (c, q, kv):
        a.grad = None
    loss.backward()
    for a, b in zip(g1, (c.grad, q.grad, kv.grad)):
        assert torch.equal(a, b)
    with P.Context.from_lp(lp) as shared:
        c2, q2, k2 = [t(a).requires_grad_() for a in (lp.c, lp.q, lp.val)]
        xa, _ = unrolled_pdhg(*args(c2, q2, k2), 60, 20, context=shared)
        xb, _ = unrolled_pdhg(*args(t(lp.c), t(lp.q), t(lp.val)), 30, 10, context=shared)  # another unroll
        (0.5 * ((xa - target) ** 2).sum()).backward()
        assert torch.equal(xa, x)
        for a, b in zip(g1, (c2.grad, q2.grad, k2.grad)):
            assert torch.equal(a, b)


def test_float32_forward_float64_adjoint(gpu_lib, oracle_lib):
    # the float32 map is the float64 map up to float32 rounding: x_T, y_T
    # agree to 1e-4; the adjoints agree to 1e-2, the difference coming from
    # dual-projection masks of rows that sit at their bound (y_i = 0), which
    # float32 rounding puts on the other side of the kink for a few steps
    lp = CASES["mip_2000x5000"]()
    T = 120
    rng = np.random.default_rng(21)
    gx = rng.standard_normal(lp.n)
    with P.Context.from_lp(lp, precision=P.PDLP_FP32) as ctx:
        x, y, eta = ctx.unroll(T, 50)
        dc, dq, dK = ctx.grad(gx, None)
    omega = _omega(lp)
    x2, y2 = oracle.unroll_forward(lp, eta, omega)
    assert _rel(x, x2) <= 1e-4 and _rel(y, y2) <= 1e-4
    rc, rq, rk = oracle.unroll_vjp(lp, eta, omega, gx, None)
    assert _rel(dc, rc) <= 1e-2 and _rel(dq, rq) <= 1e-2 and _rel(dK, rk) <= 1e-2


def test_grad_without_unroll_and_bad_checkpoints_are_rejected(gpu_lib):
    lp = CASES["planted_25x40"]()
    with P.Context.from_lp(lp) as ctx:
        with pytest.raises(P.PdlpError) as ei:
            ctx.grad(np.ones(lp.n))
        assert ei.value.code == P.PDLP_ERR_STATE
        for bad in (0, 257):
            with pytest.raises(P.PdlpError) as ei:
                ctx.unroll(10, bad)
            assert ei.value.code == P.PDLP_ERR_INVALID_ARG
