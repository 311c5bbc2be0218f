"""GPU adjoint (jgs2_step_adjoint) against the oracle's dense adjoint, and through
torch.autograd against central differences of the GPU forward."""
import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes
from oracle import adjoint, fem, newton, precompute

pytestmark = pytest.mark.gpu


def t(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


@pytest.fixture(scope="module")
def beam():
    s = scenes.small_beam_scene(9, 3, 3, E=2e5, vel_sigma=0.05, seed=2)
    E = s.youngs * np.random.default_rng(1).uniform(0.5, 1.5, s.n_tets)
    m = fem.Mesh(s.X, s.tets, E, s.poisson, s.density, s.pinned)
    x_t = scenes.perturbed_state(s.X, s.pinned, 1e-4, seed=4)
    x1, _, hist = newton.newton_solve(m, x_t, s.v0, s.dt, s.gravity, rel_tol=1e-12)
    cub = precompute.train_cubature(m, s.dt)
    return s, E, m, x_t, x1, cub


@pytest.mark.parametrize("prec,corr", [(p.FP64, p.CORR_OFF), (p.FP32, p.CORR_OFF),
                                       (p.FP64, p.CORR_ASM), (p.FP32, p.CORR_ASM)])
def test_adjoint_matches_dense_oracle(cuda, beam, prec, corr):
    """The adjoint system solved with block-Jacobi preconditioning (CORR_OFF) and with the
    corrected sweep's local solves as the preconditioner (CORR_ASM: H_ii plus the rotated
    cubature element Hessians at x*)."""
    s, E, m, x_t, x1, cub = beam
    r = np.random.default_rng(9)
    cx, cv = r.normal(size=x1.shape), r.normal(size=x1.shape)
    gx_o, gv_o, gE_o = adjoint.step_adjoint(m, x_t, s.v0, x1, cx, cv, s.dt)
    g = p.Mesh.from_scene(s)
    g.set_youngs(E)
    g.precompute_import(cub.elem, cub.weight, cub.ubar)
    tol = 1e-12 if prec == p.FP64 else 1e-6
    opts = p.jgs2.adjoint_opts(precision=prec, correction=corr, rel_tol=tol, max_iters=20000)
    gx, gv, gE, rep = g.step_adjoint(t(x_t, cuda), t(s.v0, cuda), t(x1, cuda), t(cx, cuda), t(cv, cuda), opts=opts)
    assert rep.converged == 1, rep.rel_residual
    bound = 1e-8 if prec == p.FP64 else 2e-3
    for got, ref in [(gx, gx_o), (gv, gv_o), (gE, gE_o)]:
        got = got.cpu().numpy()
        assert np.linalg.norm(got - ref) <= bound * np.linalg.norm(ref)


def _newton_tight(m, x_t, v_t, h, gravity):
    z = fem.inertia_target(x_t, v_t, h, gravity)
    x, best = x_t.copy(), np.inf
    for _ in range(40):
        xn = newton.newton_step_dense(m, x, z, h)
        r = np.linalg.norm(fem.vertex_gradient(m, xn, z, h)[m.free])
        if r >= best:
            break
        x, best = xn, r
    return x


def _newton_tight_sparse(m, x_t, v_t, h, gravity):
    """Projected Newton with backtracking from x_t, then full Newton steps with a sparse
    direct solve until the residual stops decreasing."""
    import scipy.sparse.linalg as spla
    z = fem.inertia_target(x_t, v_t, h, gravity)
    x, _, _ = newton.newton_solve(m, x_t, v_t, h, gravity, rel_tol=1e-6)
    g = fem.vertex_gradient(m, x, z, h)
    best = np.linalg.norm(g[m.free])
    for _ in range(30):
        dx = spla.spsolve(fem.global_hessian(m, x, h, dense=False), -fem.free_vector(m, g))
        xn = x.copy()
        xn[m.free] += dx.reshape(-1, 3)
        gn = fem.vertex_gradient(m, xn, z, h)
        r = np.linalg.norm(gn[m.free])
        if r >= best:
            break
        x, g, best = xn, gn, r
    return x


def test_autograd_step_against_central_differences(cuda, beam):
    """dL/dE through JGS2Step (GPU forward, GPU adjoint) against central differences (h = 1e-4
    relative) of the exact step map, on 20 seeded elements. The difference quotients use the
    oracle's Newton solve to machine precision: the JGS2 forward's own stopping tolerance is
    far above the tiny loss changes a 1e-4 modulus change makes."""
    import torch
    from paper_2506_06494_b300.autograd import JGS2Step
    s, E, m, x_t, x1, cub = beam
    g = p.Mesh.from_scene(s)
    g.precompute_import(cub.elem, cub.weight, cub.ubar)
    fopts = p.step_opts(precision=p.FP64, rel_tol=1e-9, max_sweeps=50000)
    aopts = p.jgs2.adjoint_opts(precision=p.FP64, rel_tol=1e-12, max_iters=20000, correction=p.CORR_OFF)
    xt, vt = t(x_t, cuda), t(s.v0, cuda)
    wn = np.random.default_rng(3).normal(size=x1.shape)
    w = t(wn, cuda)
    Et = t(E, cuda).requires_grad_(True)
    x_out, v_out = JGS2Step.apply(g, xt, vt, Et, fopts, aopts)
    loss = (w * x_out).sum() + (w * v_out).sum() * 0.01
    loss.backward()
    rel = 1e-4

    def L(Ep):
        mm = fem.Mesh(s.X, s.tets, Ep, s.poisson, s.density, s.pinned)
        xo = _newton_tight(mm, x_t, s.v0, s.dt, s.gravity)
        return float(np.sum(wn * xo) + np.sum(wn * (xo - x_t) / s.dt) * 0.01)

    scale = float(Et.grad.abs().max())
    for e in np.random.default_rng(5).choice(s.n_tets, size=20, replace=False):
        Ep, Em = E.copy(), E.copy()
        Ep[e] *= 1 + rel
        Em[e] *= 1 - rel
        fd = (L(Ep) - L(Em)) / (2 * rel * E[e])
        ad = float(Et.grad[e])
        assert abs(fd - ad) <= 1e-3 * abs(fd) + 1e-4 * scale, (e, fd, ad)


def test_checkpointed_rollout_equals_unrolled(cuda, beam):
    import torch
    from paper_2506_06494_b300.autograd import JGS2Step, rollout
    s, E, m, x_t, x1, cub = beam
    g = p.Mesh.from_scene(s)
    g.precompute_import(cub.elem, cub.weight, cub.ubar)
    fopts = p.step_opts(precision=p.FP64, correction=p.CORR_OFF, rel_tol=1e-8, max_sweeps=200000)
    aopts = p.jgs2.adjoint_opts(precision=p.FP64, rel_tol=1e-10, max_iters=20000, correction=p.CORR_OFF)
    xt, vt = t(x_t, cuda), t(s.v0, cuda)
    Ea = t(E, cuda).requires_grad_(True)
    x, v = xt, vt
    for _ in range(4):
        x, v = JGS2Step.apply(g, x, v, Ea, fopts, aopts)
    (x.sum() + v.sum()).backward()
    Eb = t(E, cuda).requires_grad_(True)
    xb, vb = rollout(g, xt, vt, Eb, 4, checkpoint_every=2, opts=fopts, adj_opts=aopts)
    (xb.sum() + vb.sum()).backward()
    assert torch.allclose(xb, x, rtol=0, atol=1e-12)
    assert torch.allclose(Eb.grad, Ea.grad, rtol=1e-6, atol=1e-9 * float(Ea.grad.abs().max()))


def test_rollout_gradient_against_central_differences(cuda):
    """The differentiation workload's recipe on a beam the JGS2 forward converges on (the
    9x3x3-vertex beam at E = 2e5; the full stiff beam's forward does not reach its
    tolerance): per-element E_e = 2e5 U(0.5, 1.5) (seed 0), a 30-step rollout with state
    checkpoints every 5 steps, loss = sum |x_30 - xbar_30|^2 against the rollout with
    uniform E = 2e5; dL/dE through autograd.rollout (GPU forward converged to 1e-9, GPU
    adjoint) against central differences (h = 1e-4 relative) of the oracle's tightly
    converged rollout on 20 elements drawn with seed 1."""
    import torch
    from paper_2506_06494_b300.autograd import rollout
    s = scenes.small_beam_scene(9, 3, 3, E=2e5, vel_sigma=0.05, seed=2)
    E0 = s.youngs.copy()
    E = E0 * np.random.default_rng(0).uniform(0.5, 1.5, s.n_tets)
    n, every = 30, 5
    g = p.Mesh.from_scene(s)
    fopts = p.step_opts(precision=p.FP64, correction=p.CORR_OFF, rel_tol=1e-9, max_sweeps=200000)
    aopts = p.jgs2.adjoint_opts(precision=p.FP64, rel_tol=1e-12, max_iters=20000, correction=p.CORR_OFF)
    xt, vt = t(s.X, cuda), t(s.v0, cuda)
    with torch.no_grad():
        xbar, _ = rollout(g, xt, vt, t(E0, cuda), n, every, fopts, aopts)
    Et = t(E, cuda).requires_grad_(True)
    xn, _ = rollout(g, xt, vt, Et, n, every, fopts, aopts)
    loss = ((xn - xbar) ** 2).sum()
    loss.backward()

    def oracle_rollout(Ep):
        mm = fem.Mesh(s.X, s.tets, Ep, s.poisson, s.density, s.pinned)
        x, v = s.X.copy(), s.v0.copy()
        for _ in range(n):
            x1 = _newton_tight_sparse(mm, x, v, s.dt, s.gravity)
            x, v = x1, (x1 - x) / s.dt
        return x

    xbar_o = oracle_rollout(E0)
    assert np.abs(xbar.cpu().numpy() - xbar_o).max() <= 1e-7 * np.abs(xbar_o - s.X).max()
    L = lambda Ep: float(np.sum((oracle_rollout(Ep) - xbar_o) ** 2))  # noqa: E731
    scale = float(Et.grad.abs().max())
    rel = 1e-4
    for e in np.random.default_rng(1).choice(s.n_tets, size=20, replace=False):
        Ep, Em = E.copy(), E.copy()
        Ep[e] *= 1 + rel
        Em[e] *= 1 - rel
        fd = (L(Ep) - L(Em)) / (2 * rel * E[e])
        ad = float(Et.grad[e])
        assert abs(fd - ad) <= 1e-3 * abs(fd) + 1e-4 * scale, (e, fd, ad)


def test_unconverged_forward_is_refused(cuda, beam):
    """The implicit-function adjoint needs grad E(x_{t+1}) = 0: a forward step that stops on
    its sweep cap raises instead of returning a meaningless gradient."""
    import torch
    from paper_2506_06494_b300.autograd import JGS2Step, NotConvergedError
    s, E, m, x_t, x1, cub = beam
    g = p.Mesh.from_scene(s)
    fopts = p.step_opts(precision=p.FP64, correction=p.CORR_OFF, rel_tol=1e-12, max_sweeps=3)
    Et = t(E, cuda).requires_grad_(True)
    with pytest.raises(NotConvergedError):
        JGS2Step.apply(g, t(x_t, cuda), t(s.v0, cuda), Et, fopts, None)
    x_out, _ = JGS2Step.apply(g, t(x_t, cuda), t(s.v0, cuda), Et, fopts, None, True)
    assert torch.isfinite(x_out).all()
