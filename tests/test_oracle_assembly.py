"""Pins of the oracle's discrete spaces and patch matrices (Sec. 2.2)."""
import json
import os

import numpy as np
import pytest

from workloads import make_problem, small_problem
from workloads.configs import build_problem, default_coil
from oracle.assembly import Assembled, PatchEval, coil_potential
from oracle.gauge import Gauge
from oracle.lattice import Lattice
from oracle.monolithic import Monolithic
from oracle.manufactured import A_star, curl_A_star, FieldEval, PI

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")))


def test_paper_dof_count_7260():
    """Sec. 4: two subdomains, p = 3, h = 2^-3 -> 7260 DOFs in a^(l+1)."""
    # h = 2^-3 is the parametric element size of each subdomain: 8 elements per
    # direction on each patch (each patch is a unit parameter cube)
    prob = build_problem("paper", (2, 1, 1), [[8, 8], [8], [8]], [[3, 3], [3], [3]],
                         sigma_fn=lambda s, C: 1.0 if s == 0 else 0.0, nu_fn=lambda s, C: 1.0,
                         dt=1 / 32, n_steps=32)
    lat = Lattice(prob)
    total = sum(len(lat.patch_local_to_global(s)) for s in range(prob.n_patches))
    assert total == GOLD["dofs_two_subdomains"]["value"]


def _gradient_coeffs(pe, net, a):
    """Edge coefficients of grad(a . x) on a patch: differences of the nodal values
    phi_ijk = a . c_ijk along each control-mesh edge (x = F(xi) lies in the H^1 space)."""
    phi = net @ a                                    # (n2, n1, n0)
    return np.concatenate([(phi[:, :, 1:] - phi[:, :, :-1]).ravel(),
                           (phi[:, 1:, :] - phi[:, :-1, :]).ravel(),
                           (phi[1:, :, :] - phi[:-1, :, :]).ravel()])


@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_gradients_exact_curl_free_and_mass(cfg):
    prob = make_problem(cfg)
    s = 0 if cfg == "c1" else 21                     # c2 patch 21 conducts and is curved
    pe = PatchEval(prob, s)
    net = prob.patch_ctrl(s)
    a = np.array([0.3, -1.1, 0.7])
    g = _gradient_coeffs(pe, net, a)
    K = pe.stiffness(prob.patch_nu(s).reshape(-1))
    sig = np.ones(pe.E)
    M = pe.mass(sig)
    vol = np.sum(pe.w * pe.det)
    assert np.abs(K @ g).max() < 1e-12 * np.abs(K).max() * np.abs(g).max()
    assert abs(g @ (M @ g) - (a @ a) * vol) < 1e-12 * (a @ a) * vol
    # volume of the (interior-perturbed) patch is the box volume
    box = 1.0 / np.prod(prob.P)
    assert abs(vol - box) < 1e-12
    # j = <T, curl w> annihilates gradients; <e, w> gives a . e * vol
    jT = pe.load_from_potential(coil_potential(prob.coil))
    assert abs(jT @ g) < 1e-12 * np.abs(jT).sum() * np.abs(g).max() + 1e-300
    e = np.array([0.2, 0.5, -0.9])
    jf = pe.load_from_field(lambda x: np.broadcast_to(e, x.shape))
    assert abs(jf @ g - (a @ e) * vol) < 1e-12


@pytest.mark.parametrize("p", [1, 2])
def test_linear_field_curl_energy(p):
    """A = (0, 0, x) on an identity-mapped patch: curl A = (0, -1, 0), so
    a^T K a = nu * vol and the L2 projection reproduces A."""
    prob = build_problem("lin", (1, 1, 1), [[3], [2], [2]], [[p], [p], [p]],
                         sigma_fn=lambda s, C: 1.0, nu_fn=lambda s, C: 2.5, dt=1.0, n_steps=1)
    pe = PatchEval(prob, 0)
    M = pe.mass(np.ones(pe.E))
    K = pe.stiffness(np.full(pe.E, 2.5))
    rhs = pe.load_from_field(lambda x: np.stack([0 * x[..., 0], 0 * x[..., 0], x[..., 0]], -1))
    c = np.linalg.solve(M.toarray(), rhs)
    assert abs(c @ (K @ c) - 2.5 * 1.0) < 1e-10
    V = pe.phys_values()
    Ah = np.einsum("ea,eqai->eqi", c[pe.loc], V)
    assert np.abs(Ah[..., 2] - pe.F[..., 0]).max() < 1e-10
    assert np.abs(Ah[..., :2]).max() < 1e-10


def test_matrices_symmetric_semidefinite():
    prob = small_problem()
    A = Assembled(prob)
    for s in range(prob.n_patches):
        for X in (A.K[s], A.M[s]):
            Xd = X.toarray()
            assert np.abs(Xd - Xd.T).max() <= 1e-14 * np.abs(Xd).max()
            assert np.linalg.eigvalsh(Xd).min() >= -1e-10 * np.abs(Xd).max()


def _mms_errors(p, ne):
    prob = small_problem(P=(2, 1, 1), n_el=((ne, ne), (2 * ne,), (2 * ne,)),
                         degree=((p, p), (p,), (p,)), conductor=((0, 0.5), (0, 1), (0, 1)),
                         sigma=1.0, dt=1.0, perturb=0.0)
    A = Assembled(prob, with_load=False)
    G = Gauge(prob, A.lat)
    Mo = Monolithic(prob, A, G)
    fe = FieldEval(prob, A)
    sig = lambda x: np.where(x[..., 0] < 0.5, 1.0, 0.0)[..., None]
    j = fe.load(lambda x: (2 * PI ** 2 + sig(x)) * A_star(x))
    a = Mo.step(np.zeros(A.lat.n_edges), j)
    return fe.errors(a, A_star, curl_A_star)


@pytest.mark.parametrize("p,sizes", [(1, (2, 4, 8)), (2, (2, 4))])
def test_manufactured_h_rates(p, sizes):
    """sigma A + curl curl A = J on a conductor/insulator split at x = 0.5 (the
    steady analogue of Sec. 4's test): the curl error decays like h^p."""
    errs = [_mms_errors(p, n) for n in sizes]
    rates_B = [np.log2(errs[k][1] / errs[k + 1][1]) for k in range(len(errs) - 1)]
    assert all(abs(r - p) < 0.25 for r in rates_B), rates_B
    rates_A = [np.log2(errs[k][0] / errs[k + 1][0]) for k in range(len(errs) - 1)]
    assert all(r > p + 0.7 for r in rates_A), rates_A
