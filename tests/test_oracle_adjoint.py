"""Pins of the oracle's reverse-mode gradient (form 3) against central finite
differences of the oracle's own forward loss, which the closed-form pins of
test_oracle_pins.py fix.  A dropped stage term, a transposed G, a wrong RK
weight or a missing chain-rule factor J^-1 each moves the gradient far beyond
the finite-difference error."""
import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W


@pytest.mark.parametrize("dim,integrator", [(3, 4), (3, 2), (2, 4), (2, 1)])
def test_adjoint_matches_central_differences(oracle_mod, dim, integrator):
    O = oracle_mod
    if dim == 3:
        wl = W.curl_cube(4, 3, 3, 4)
    else:
        wl = W.c5_member(5, 3)
        wl.per_cell[:] = 3
    m = O.Mesh(wl.n, wl.X, wl.U)
    p = O.seed_particles(m, per_cell=wl.per_cell, uniform_count=wl.ppc or 0, seed=wl.pseed)
    g = np.random.default_rng(0)
    steps, dt = 3, 2 * wl.dt
    tg = p.x + 0.02 * g.standard_normal(p.x.shape)
    L, grad = O.advect_adjoint(m, p, dt, integrator, steps, tg)
    assert L == pytest.approx(O.advect_loss(m, p, dt, integrator, steps, tg), rel=1e-15)
    scale = np.abs(grad).max()
    assert scale > 0
    # the DOFs with the largest gradients plus random ones
    flat = np.argsort(-np.abs(grad).ravel())[:6].tolist() + g.choice(grad.size, 10, replace=False).tolist()
    h = 1e-6
    for q in flat:
        c, node = divmod(int(q), grad.shape[1])
        Up = wl.U.copy()
        Up[c, node] += h
        m.set_velocity(Up)
        Lp = O.advect_loss(m, p, dt, integrator, steps, tg)
        Up[c, node] -= 2 * h
        m.set_velocity(Up)
        Lm = O.advect_loss(m, p, dt, integrator, steps, tg)
        m.set_velocity(wl.U)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - grad[c, node]) <= 1e-6 * scale, (q, fd, grad[c, node])


def test_adjoint_lost_particles_contribute_nothing(oracle_mod):
    O = oracle_mod
    wl = W.c1(n=8, ppc=4)
    m = O.Mesh(wl.n, wl.X, wl.U)
    p = O.seed_particles(m, uniform_count=wl.ppc, seed=wl.pseed)
    steps, dt = 4, 40 * wl.dt  # corners leave the square
    tg = np.zeros_like(p.x)
    L, grad = O.advect_adjoint(m, p, dt, 2, steps, tg)
    alive = O.advect(m, p, dt, 2, steps)
    assert alive.n < p.n
    survivors = set(int(i) for i in alive.id)
    keep = np.array([int(i) in survivors for i in p.id])
    L2, grad2 = O.advect_adjoint(m, p.subset(keep), dt, 2, steps, tg[keep])
    assert L == pytest.approx(L2, rel=1e-14)
    np.testing.assert_allclose(grad, grad2, rtol=0, atol=1e-14 * np.abs(grad).max())


@pytest.mark.parametrize("dim,integrator,losses", [(3, 4, False), (3, 2, False), (2, 4, False), (2, 1, False),
                                                   (3, 4, True)])
def test_dot_product_reverse_against_tangent(oracle_mod, dim, integrator, losses):
    """<J V, W> = <V, J^T W> for the map U -> final positions: the tangent-
    linear sweep (forward mode, written apart) against the reverse sweep, with
    lambda_final = W through targets x_final - W/2.  Both are exact
    derivatives of the same discrete map, so they agree to rounding."""
    O = oracle_mod
    if dim == 3:
        wl = W.curl_cube(4, 3, 3, 4) if not losses else W.curl_cube(5, 4, 2, 9)
    else:
        wl = W.c5_member(5, 3)
        wl.per_cell[:] = 3
    m = O.Mesh(wl.n, wl.X, wl.U)
    p = O.seed_particles(m, per_cell=wl.per_cell, uniform_count=wl.ppc or 0, seed=wl.pseed)
    g = np.random.default_rng(5)
    steps, dt = 3, (12 if losses else 2) * wl.dt
    V = g.standard_normal(wl.U.shape)
    Wt = g.standard_normal(p.x.shape)
    dx, alive = O.advect_tangent(m, p, dt, integrator, steps, V)
    assert alive.any()
    if losses:
        assert not alive.all()
    fin = O.advect(m, p, dt, integrator, steps)
    x_final = dict(zip((int(i) for i in fin.id), fin.x))
    assert set(x_final) == set(int(i) for i in p.id[alive])
    tg = np.zeros_like(p.x)
    for q in np.nonzero(alive)[0]:
        tg[q] = x_final[int(p.id[q])] - 0.5 * Wt[q]
    _, grad = O.advect_adjoint(m, p, dt, integrator, steps, tg)
    lhs = float(np.sum(Wt[alive] * dx[alive]))
    rhs = float(np.sum(V * grad))
    mag = float(np.sum(np.abs(Wt[alive] * dx[alive])) + np.sum(np.abs(V * grad)))
    assert abs(lhs - rhs) <= 1e-12 * mag, (lhs, rhs, mag)
