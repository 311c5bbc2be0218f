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


@pytest.mark.parametrize("prec,corr", [(p.FP64, p.CORR_OFF), (p.FP32, p.CORR_OFF)])
def test_adjoint_matches_dense_oracle(cuda, beam, prec, corr):
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
    fopts = p.step_opts(precision=p.FP64, rel_tol=1e-8, max_sweeps=20000)
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
