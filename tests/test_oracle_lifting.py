"""Pins of the boundary lifting and of the lifted run of the paper's experiment
(Sec. 4, Eq. (13): A = e^{-t} (sin x cos y cos z, -2 cos x sin y cos z, cos x cos y sin z))."""
import numpy as np
import pytest

from workloads import small_problem
from oracle.lifting import A13, curl_A13, LiftedRun, boundary_projection
from oracle.manufactured import FieldEval
from oracle.stepping import OracleProblem


def two_subdomains(n, p, n_t):
    return small_problem(P=(2, 1, 1), n_el=((n, n), (n,), (n,)), degree=((p, p), (p,), (p,)),
                         conductor=((0.0, 0.5), (0.0, 1.0), (0.0, 1.0)), sigma=1.0, nu=1.0,
                         dt=1.0 / n_t, n_steps=n_t, perturb=0.0, J0=0.0, name="paper_two_subdomains")


def node_xyz(prob, lat):
    """Physical position of every lattice node (the control points of the identity map)."""
    X = np.zeros((lat.n_nodes, 3))
    for s in range(prob.n_patches):
        a = prob.patch_index(s)
        net = prob.patch_ctrl(s)                    # (n2, n1, n0, 3)
        n2, n1, n0 = net.shape[:3]
        K, J, I = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
        ids = lat.node_id(I + lat.off[0][a[0]], J + lat.off[1][a[1]],
                          K + lat.off[2][a[2]])
        X[ids.ravel()] = net.reshape(-1, 3)
    return X


@pytest.mark.parametrize("P,n,p", [((2, 1, 1), (2, 2), 2), ((2, 2, 1), (2, 3), 3), ((1, 1, 1), (3, 3), 1)])
def test_boundary_projection_reproduces_gradients(P, n, p):
    """A constant field c = grad(c . x) lies in the edge space: its coefficients are the
    differences of c . x between the end nodes of every edge.  The boundary
    projection must return them on every Dirichlet DOF."""
    prob = small_problem(P=P, n_el=(tuple([n[0]] * P[0]), tuple([n[1]] * P[1]), tuple([n[0]] * P[2])),
                         degree=(tuple([p] * P[0]), tuple([p] * P[1]), tuple([p] * P[2])), perturb=0.0)
    op = OracleProblem(prob, with_load=False)
    lat = op.asm.lat
    c = np.array([0.3, -1.1, 0.7])
    X = node_xyz(prob, lat)
    exact = (X[lat.node1] - X[lat.node0]) @ c
    aD, bnd = boundary_projection(prob, op.asm, lambda x: np.broadcast_to(c, x.shape))
    assert set(bnd.tolist()) == set(np.nonzero(lat.dirichlet)[0].tolist())
    assert np.max(np.abs(aD[bnd] - exact[bnd])) <= 1e-12 * np.max(np.abs(exact))


def test_curl_of_A13_and_source_identity():
    """curl A13 by central differences, and curl curl A13 = 3 A13 (div A13 = 0)."""
    rng = np.random.default_rng(1)
    x = rng.uniform(0.1, 0.9, size=(20, 3))
    h = 1e-5
    def curl(F, x):
        J = np.zeros((len(x), 3, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = h
            J[:, :, k] = (F(x + e) - F(x - e)) / (2 * h)
        return np.stack([J[:, 2, 1] - J[:, 1, 2], J[:, 0, 2] - J[:, 2, 0], J[:, 1, 0] - J[:, 0, 1]], axis=-1)
    assert np.allclose(curl(A13, x), curl_A13(x), atol=1e-8)
    assert np.allclose(curl(curl_A13, x), 3.0 * A13(x), atol=1e-6)


def _lifted_errors(n, p, n_t):
    prob = two_subdomains(n, p, n_t)
    op = OracleProblem(prob, with_load=False)
    sig = lambda x: (x[..., 0] < 0.5).astype(float)
    run = LiftedRun(op, A13, lambda x: (3.0 - sig(x))[..., None] * A13(x), sig)
    a0 = run.run_monolithic(n_t)
    fe = FieldEval(prob, op.asm)
    t1, t0 = 1.0, 1.0 - 1.0 / n_t
    A1, A0 = run.total(a0[-1], t1), run.total(a0[-2], t0)
    _, eB = fe.errors(A1, lambda x: np.exp(-t1) * A13(x), lambda x: np.exp(-t1) * curl_A13(x))
    eE, _ = fe.errors(-(A1 - A0) * n_t, lambda x: np.exp(-t1) * A13(x), lambda x: 0 * x)
    return eB, eE


def test_lifted_run_rates():
    """Sec. 4 bounds eps = O(h^p + 1/n_t): B converges at order ~p in h (p = 2, n_t
    large), E at first order in n_t."""
    eB2, _ = _lifted_errors(2, 2, 256)
    eB4, _ = _lifted_errors(4, 2, 256)
    assert eB2 / eB4 > 3.0, (eB2, eB4)                       # better than h^{1.6}
    _, eE16 = _lifted_errors(4, 2, 16)
    _, eE64 = _lifted_errors(4, 2, 64)
    assert 3.0 < eE16 / eE64 < 5.5, (eE16, eE64)             # first order in time


def test_lifted_run_dual_primal_equals_monolithic():
    """The lifting enters only through the initial state and the load vectors, so the
    oracle's IETI-DP solve of the lifted run (what the library is given) equals the
    monolithic solve step by step."""
    from oracle.ietidp import PRECOND_DIRICHLET
    n, p, n_t = 2, 2, 4
    prob = two_subdomains(n, p, n_t)
    op = OracleProblem(prob, with_load=False)
    sig = lambda x: (x[..., 0] < 0.5).astype(float)
    run = LiftedRun(op, A13, lambda x: (3.0 - sig(x))[..., None] * A13(x), sig)
    ref = run.run_monolithic(n_t)
    got, _ = op.run_ietidp(n_t, 1e-12, PRECOND_DIRICHLET, j_of_step=run.j_step, a0=run.a0)
    for a, b in zip(ref, got):
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)
    assert np.linalg.norm(run.a0) > 0 and np.linalg.norm(run.aD_star) > 0
