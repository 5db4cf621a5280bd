"""Pins of oracle.adjoint: central finite differences of the float64 forward map, and
transpose identities <A x, y> = <x, A^T y> of its pieces against finite differences."""
import numpy as np
import pytest

from oracle import adjoint as oa
from oracle import lpt, mesh
from oracle.cola import ColaConfig
from oracle.cosmology import Cosmology


@pytest.fixture(scope="module")
def small():
    cfg = ColaConfig(n_p=12, n_g=24, box=100.0, nsteps=3)
    rng = np.random.default_rng(0)
    w = rng.standard_normal((12, 12, 12))
    target = oa.final_density(oa.forward_with_checkpoints(rng.standard_normal((12, 12, 12)), cfg)["s"], cfg)
    loss, grad, fw = oa.loss_and_gradient(w, target, cfg)
    return cfg, w, target, loss, grad


def test_loss_gradient_matches_central_differences(small):
    cfg, w, target, loss, grad = small
    rng = np.random.default_rng(1)
    rel = []
    for _ in range(6):
        e = rng.standard_normal(w.shape)
        eps = 1e-5
        fd = (oa.loss_only(w + eps * e, target, cfg) - oa.loss_only(w - eps * e, target, cfg)) / (2 * eps)
        rel.append(abs(fd / float(np.sum(grad * e)) - 1.0))
    # a direction may move a particle across a CIC kink inside +-eps; most must agree tightly
    assert np.median(rel) < 1e-6
    assert np.sum(np.array(rel) < 1e-4) >= 5


def test_gradient_checkpoints_follow_the_forward_run(small):
    cfg, w, target, loss, _ = small
    fw = oa.forward_with_checkpoints(w, cfg)
    assert len(fw["ckpt"]) == cfg.nsteps + 1
    assert loss == pytest.approx(float(np.sum((oa.final_density(fw["s"], cfg) - target) ** 2)), rel=1e-14)


def test_force_vjp_is_the_transpose_of_the_force_jacobian():
    rng = np.random.default_rng(3)
    box, ng, npart = 50.0, 16, 60
    pos = rng.uniform(0, box, size=(3, npart))
    lam = rng.standard_normal((3, npart))
    e = rng.standard_normal((3, npart))
    mu = oa.force_vjp(pos, lam, npart, ng, box, deconv=1)
    eps = 1e-6
    gp = mesh.unit_force_particles(pos + eps * e, npart, ng, box, 1)
    gm = mesh.unit_force_particles(pos - eps * e, npart, ng, box, 1)
    fd = float(np.sum(lam * (gp - gm))) / (2 * eps)
    assert float(np.sum(mu * e)) == pytest.approx(fd, rel=1e-6)


def test_density_vjp_is_the_transpose_of_the_density_jacobian():
    rng = np.random.default_rng(4)
    box, ng, npart = 30.0, 12, 40
    pos = rng.uniform(0, box, size=(3, npart))
    dbar = rng.standard_normal((ng, ng, ng))
    e = rng.standard_normal((3, npart))
    mu = oa.density_vjp(pos, dbar, npart, box)
    eps = 1e-6

    def dens(p):
        return mesh.overdensity(mesh.cic_deposit(p, ng, box), npart)

    fd = float(np.sum(dbar * (dens(pos + eps * e) - dens(pos - eps * e)))) / (2 * eps)
    assert float(np.sum(mu * e)) == pytest.approx(fd, rel=1e-6)


def test_ic_vjp_is_the_transpose_of_the_2lpt_map():
    cosmo = Cosmology()
    rng = np.random.default_rng(5)
    n, box = 10, 80.0
    w = rng.standard_normal((n, n, n))
    l1, l2 = rng.standard_normal((3, n**3)), rng.standard_normal((3, n**3))
    e = rng.standard_normal((n, n, n))
    g = oa.ic_vjp(w, l1, l2, box, cosmo)
    eps = 1e-4  # s1 is linear and s2 quadratic in the noise: central differences are exact
    p1, p2 = lpt.ic_2lpt(w + eps * e, box, cosmo)
    m1, m2 = lpt.ic_2lpt(w - eps * e, box, cosmo)
    fd = (float(np.sum(l1 * (p1 - m1))) + float(np.sum(l2 * (p2 - m2)))) / (2 * eps)
    assert float(np.sum(g * e)) == pytest.approx(fd, rel=1e-9)
