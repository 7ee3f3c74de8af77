"""The seeded synthetic inputs: deterministic, and with the structure each workload
states (patch grid, element counts and degrees, material layout, curved patches that
keep planar matching faces).  No arithmetic of the method is involved."""
import numpy as np
import pytest

from workloads import make_problem


def _same(a, b):
    return (a.P == b.P and all(np.array_equal(x, y) for x, y in zip(a.n_el, b.n_el))
            and all(np.array_equal(x, y) for x, y in zip(a.degree, b.degree))
            and np.array_equal(a.ctrl, b.ctrl) and np.array_equal(a.sigma_el, b.sigma_el)
            and np.array_equal(a.nu_el, b.nu_el))


@pytest.mark.parametrize("name,kw", [("c1", {}), ("c2", {}), ("c3", dict(patches_per_dir=3, n_el=2)),
                                     ("c4", dict(patches_per_dir=3, el_range=(2, 3))), ("c5", {})])
def test_seeded_and_deterministic(name, kw):
    assert _same(make_problem(name, **kw), make_problem(name, **kw))


def test_c2_layout():
    prob = make_problem("c2")
    assert prob.P == (4, 4, 4) and prob.dt == 1e-3 and prob.coil["J0"] == 1e2
    assert all(np.all(prob.n_el[d] == 8) and np.all(prob.degree[d] == 2) for d in range(3))
    cond = [s for s in range(prob.n_patches) if np.all(prob.patch_sigma(s) == 1e2)]
    assert len(cond) == 8                                          # the inner 2^3 patches
    for s in range(prob.n_patches):
        sig = prob.patch_sigma(s)
        assert np.all(sig == sig.flat[0]) and sig.flat[0] in (0.0, 1e2)
    # curved: interior control points moved by at most 5% of an element, faces planar
    s = 21
    net = prob.patch_ctrl(s)
    a = prob.patch_index(s)
    h = 1.0 / (4 * 8)
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        face_lo = np.take(net[..., d], 0, axis=ax)
        assert np.allclose(face_lo, face_lo.flat[0])              # planar patch face
    inner = net[1:-1, 1:-1, 1:-1]
    assert np.abs(inner - np.round(inner / h * 2) * h / 2).max() > 0   # actually perturbed
    assert a == (1, 1, 1)


def test_c3_and_c4_families():
    c3 = make_problem("c3")
    assert c3.P == (8, 8, 8)
    sig = np.array([c3.patch_sigma(s).flat[0] for s in range(c3.n_patches)])
    nu = np.array([c3.patch_nu(s).flat[0] for s in range(c3.n_patches)])
    on = sig > 0
    assert 1.0 <= sig[on].min() and sig[on].max() <= 1e4 and 50 < on.sum() < 200
    assert 0.5 <= nu.min() and nu.max() <= 2.0
    for s in np.nonzero(on)[0]:
        a = np.array(c3.patch_index(s))
        assert np.linalg.norm((a + 0.5) / 8 - 0.5) < 0.35              # inside the ball
    c4 = make_problem("c4")
    assert c4.P == (7, 7, 7)
    for d in range(3):
        assert set(np.unique(c4.degree[d])) <= {2, 3}
        assert c4.n_el[d].min() >= 4 and c4.n_el[d].max() <= 12
    sig4 = np.array([c4.patch_sigma(s).flat[0] for s in range(c4.n_patches)])
    assert set(np.unique(sig4)) <= {0.0, 1e3} and 0.3 < np.mean(sig4 > 0) < 0.7
