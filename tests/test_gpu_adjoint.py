"""GPU parity of the adjoint calls against the float64 oracle adjoint (oracle/adjoint.py), and
of the gradient with respect to the white noise against central finite differences.

Tolerances: the GPU differentiates the CIC weights at positions quantised to 2^-16 cell and
runs float32 FFTs; each adjoint piece agrees with the oracle's to <= 3e-4 of its largest
entry (as the forward force does).  The whole gradient is held to the 1e-3 target in two ways:
  * against the float64 oracle adjoint run along the GPU's own trajectory (its checkpoints and
    fixed-point positions), so that both sides differentiate the same piecewise-smooth map;
  * against float64 central differences of the oracle forward in the smooth regime (a_final =
    0.3, 3 steps), where central differences resolve 1e-3 (3e-5 for the oracle's own adjoint).
The loss of a full run to a = 1 is only piecewise smooth: every CIC cell face a particle crosses
is a kink.  Two runs whose particles differ by ~1e-5 cell (the GPU's quantisation and float32
rounding, amplified by the dynamics) differentiate on different sides of a few kinks: measured
on 32^3/64^3, the GPU gradient is within 3.9e-3 (L2) of the float64 oracle gradient of the
unquantised trajectory at a = 0.5 and within 1.8e-2 at a = 1, where even float64 central
differences of the oracle scatter by 0.3-5% around its exact adjoint.  Central differences of
the GPU forward also carry its 2^-16-cell quantisation steps; the 128^3/256^3 check against them
is held to that measured floor.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as oa
from oracle import mesh as omesh
from oracle.cola import ColaConfig
from oracle.cosmology import Cosmology
from paper_1301_0322_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cola():
    from paper_1301_0322_gb300 import build
    build.build(verbose=False)
    import paper_1301_0322_gb300 as c
    c.load_library()
    return c


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def test_density_adjoint_matches_oracle(cola):
    n_p, ng, box = 32, 64, 100.0
    plan = cola.Plan(np_side=n_p, ng=ng, box=box)
    s = inputs.gaussian_displacements(n_p, 1.0, 1)
    dbar = inputs.gaussian_noise(ng, 2)
    lam = host(plan.density_adjoint(dev(s), dev(dbar)))
    pos = np.mod(omesh.lattice_q(n_p, box) + s.astype(np.float64), box)
    ref = oa.density_vjp(pos, dbar.reshape(ng, ng, ng).astype(np.float64), n_p**3, box)
    assert np.abs(lam - ref).max() <= 3e-4 * np.abs(ref).max()


@pytest.mark.parametrize("step", [3, 10])
def test_step_adjoint_matches_oracle(cola, step):
    n_p, ng, box = 32, 64, 100.0
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, adjoint=True)
    row = plan.coeffs()[step]
    c, amp, t2d1, t2d2, cd, dd1, dd2, td1, td2 = (row[j] for j in (2, 1, 3, 4, 5, 6, 7, 8, 9))
    s = inputs.gaussian_displacements(n_p, 1.0, 3)
    rng = np.random.default_rng(4)
    ls, lv = (rng.standard_normal((3, n_p**3)).astype(np.float32) for _ in range(2))
    g_ls, g_lv = dev(ls), dev(lv)
    g_l1, g_l2 = torch.zeros_like(g_ls), torch.zeros_like(g_ls)
    plan.step_adjoint(step, dev(s), g_ls, g_lv, g_l1, g_l2)
    ls64, lv64 = ls.astype(np.float64), lv.astype(np.float64)
    if step < plan.nsteps:
        lv1 = lv64 + cd * ls64
        l1 = dd1 * ls64 - c * t2d1 * lv1
        l2 = dd2 * ls64 - c * t2d2 * lv1
    else:
        lv1 = lv64
        l1 = (td1 - c * t2d1) * lv64
        l2 = (td2 - c * t2d2) * lv64
    pos = np.mod(omesh.lattice_q(n_p, box) + s.astype(np.float64), box)
    vjp = c * amp * oa.force_vjp(pos, lv1, n_p**3, ng, box, deconv=1)
    assert np.allclose(host(g_lv), lv1, rtol=1e-5, atol=1e-6)
    assert np.allclose(host(g_l1), l1, rtol=1e-5, atol=1e-6 * np.abs(l1).max())
    assert np.allclose(host(g_l2), l2, rtol=1e-5, atol=1e-6 * np.abs(l2).max())
    assert np.abs(host(g_ls) - (ls64 + vjp)).max() <= 3e-4 * np.abs(vjp).max()


def test_ic_adjoint_matches_oracle(cola):
    n_p, box = 32, 100.0
    plan = cola.Plan(np_side=n_p, ng=64, box=box, adjoint=True)
    w = inputs.gaussian_noise(n_p, 5)
    rng = np.random.default_rng(6)
    ls, l1, l2 = (rng.standard_normal((3, n_p**3)).astype(np.float32) for _ in range(3))
    grad = host(plan.ic_adjoint(dev(w), dev(ls), dev(l1), dev(l2)))
    cosmo = Cosmology(**inputs.COSMOLOGY)
    g0 = cosmo.growth([0.1])
    l1r = l1.astype(np.float64) + g0["D1"][0] * ls
    l2r = l2.astype(np.float64) + g0["D2"][0] * ls
    ref = oa.ic_vjp(w.reshape(n_p, n_p, n_p).astype(np.float64), l1r, l2r, box, cosmo).reshape(-1)
    assert np.abs(grad - ref).max() <= 3e-4 * np.abs(ref).max()


@pytest.mark.parametrize("a_final,min_cos,max_rel", [(0.5, 0.99999, 1e-2), (1.0, 0.9995, 5e-2)])
def test_full_gradient_matches_oracle(cola, a_final, min_cos, max_rel):
    n_p, ng, box = 32, 64, 100.0
    cfg = ColaConfig(n_p=n_p, n_g=ng, box=box, cosmo=Cosmology(**inputs.COSMOLOGY), a_final=a_final)
    w = inputs.gaussian_noise(n_p, 1)
    target = oa.final_density(oa.forward_with_checkpoints(
        inputs.gaussian_noise(n_p, 7).reshape(n_p, n_p, n_p).astype(np.float64), cfg)["s"], cfg)
    _, gref, _ = oa.loss_and_gradient(w.reshape(n_p, n_p, n_p).astype(np.float64), target, cfg)
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, adjoint=True, a_final=a_final)
    x = dev(w).requires_grad_(True)
    delta = cola.cola_density_from_noise(x, plan)
    loss = ((delta.double() - dev(target.reshape(-1))) ** 2).sum()
    loss.backward()
    g = host(x.grad)
    gr = gref.reshape(-1)
    cos = float(g @ gr / np.linalg.norm(g) / np.linalg.norm(gr))
    rel = float(np.linalg.norm(g - gr) / np.linalg.norm(gr))
    print(f"a = {a_final}: gradient vs oracle cosine {cos:.8f}, relative L2 {rel:.2e}")
    assert cos > min_cos and rel < max_rel


def gpu_trajectory(plan, noise):
    """The GPU forward run of ColaDensity, keeping the displacement of every force evaluation
    (the same launches, hence bit for bit the trajectory the backward pass differentiates)."""
    s, v, s1, s2 = plan.ic_2lpt(noise)
    ckpt = []
    for i in range(plan.nsteps + 1):
        ckpt.append(host(s))
        plan.step(i, s, v, s1, s2)
    plan.status()
    return ckpt, host(s)


@pytest.mark.parametrize("n_p,ng,box,a_final,nsteps", [(32, 64, 100.0, 1.0, 10), (32, 64, 100.0, 0.5, 10),
                                                        (64, 128, 200.0, 1.0, 10)])
def test_gradient_matches_oracle_along_the_gpu_trajectory(cola, n_p, ng, box, a_final, nsteps):
    # Both sides differentiate the same trajectory: the float64 oracle adjoint sweep runs along
    # the GPU's own checkpoints at the GPU's fixed-point positions (2^-16 cell), so every CIC
    # kink is taken on the same side and what is left is the float32 rounding of the GPU
    # adjoint.  Target: relative L2 error <= 1e-3 of the gradient with respect to the noise.
    cosmo = Cosmology(**inputs.COSMOLOGY)
    cfg = ColaConfig(n_p=n_p, n_g=ng, box=box, cosmo=cosmo, a_final=a_final, nsteps=nsteps, fixed_bits=16)
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, adjoint=True, a_final=a_final, nsteps=nsteps)
    with torch.no_grad():
        target = cola.cola_density_from_noise(dev(inputs.gaussian_noise(n_p, 7)), plan).double()
    w = inputs.gaussian_noise(n_p, 1)
    x = dev(w).requires_grad_(True)
    loss = ((cola.cola_density_from_noise(x, plan).double() - target) ** 2).sum()
    loss.backward()
    g = host(x.grad).reshape(-1)
    ckpt, s_final = gpu_trajectory(plan, dev(w))
    unit = box / ng / 2.0**16

    def positions(s):
        return omesh.fixed_point_coords(s.astype(np.float32), n_p, ng, box, 16) * unit

    lref, gref = oa.loss_and_gradient_along(w.reshape(n_p, n_p, n_p).astype(np.float64),
                                            host(target).reshape(ng, ng, ng), cfg, ckpt, s_final, positions)
    gref = gref.reshape(-1)
    rel = float(np.linalg.norm(g - gref) / np.linalg.norm(gref))
    cos = float(g @ gref / np.linalg.norm(g) / np.linalg.norm(gref))
    print(f"{n_p}^3/{ng}^3, a = {a_final}: gradient vs oracle along the GPU trajectory: relative L2 {rel:.2e}, "
          f"cosine {cos:.9f}, loss {float(loss):.6e} vs {lref:.6e}")
    assert abs(float(loss) / lref - 1.0) <= 1e-5
    assert rel <= 1e-3


def test_gradient_matches_float64_central_differences_smooth_regime(cola):
    # Where the map is smooth enough for central differences to resolve 1e-3 -- early times
    # and few steps (a_final = 0.3, 3 steps; the float64 oracle's own central differences with
    # eps = 1e-6 agree with its exact adjoint to 3e-5 of the rms projection there) -- the GPU
    # gradient projected on 16 random low-k Fourier modes of the noise agrees with float64
    # central differences of the oracle forward map to 1e-3 of the rms projection.  (Central
    # differences of the GPU forward itself cannot resolve 1e-3: its positions move in 2^-16
    # cell steps, and any eps large enough to span many steps lets a fraction of the particles
    # cross CIC cell faces, whose kinks bias the difference quotient.)
    n_p, ng, box, a_final, nsteps = 32, 64, 100.0, 0.3, 3
    cosmo = Cosmology(**inputs.COSMOLOGY)
    cfg = ColaConfig(n_p=n_p, n_g=ng, box=box, cosmo=cosmo, a_final=a_final, nsteps=nsteps)
    w = inputs.gaussian_noise(n_p, 1)
    w64 = w.reshape(n_p, n_p, n_p).astype(np.float64)
    target = oa.final_density(oa.forward_with_checkpoints(
        inputs.gaussian_noise(n_p, 7).reshape(n_p, n_p, n_p).astype(np.float64), cfg)["s"], cfg)
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, adjoint=True, a_final=a_final, nsteps=nsteps)
    x = dev(w).requires_grad_(True)
    loss = ((cola.cola_density_from_noise(x, plan).double() - dev(target.reshape(-1))) ** 2).sum()
    loss.backward()
    g = host(x.grad)
    eps, fd, an = 1e-6, [], []
    for m in range(16):
        e = fourier_mode(n_p, 100 + m).astype(np.float64).reshape(n_p, n_p, n_p)
        fd.append((oa.loss_only(w64 + eps * e, target, cfg) - oa.loss_only(w64 - eps * e, target, cfg)) / (2 * eps))
        an.append(float(g @ e.reshape(-1)))
    fd, an = np.array(fd), np.array(an)
    err = np.abs(fd - an) / np.sqrt(np.mean(fd**2))
    print(f"a = {a_final}, {nsteps} steps: |fd - adj| / rms(fd) on 16 modes: max {err.max():.2e}, "
          f"median {np.median(err):.2e}")
    assert err.max() <= 1e-3


def fourier_mode(n, seed):
    rng = np.random.default_rng(seed)
    kvec = rng.integers(-n // 4, n // 4 + 1, size=3)
    if not kvec.any():
        kvec[0] = 1
    phase = rng.uniform(0, 2 * np.pi)
    i = np.arange(n)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    e = np.cos(2 * np.pi * (kvec[0] * x + kvec[1] * y + kvec[2] * z) / n + phase)
    return (e / np.sqrt(np.mean(e**2))).astype(np.float32).reshape(-1)


def test_gradient_matches_central_differences_128p_256g(cola):
    # the differentiable-COLA workload: 128^3 particles, 256^3 mesh, L = 200 Mpc/h, 10 steps to
    # z = 0, target density from the seed-7 run; 64 random low-k Fourier modes of the noise
    n_p, ng, box, seed = inputs.WORKLOADS["cola_128p_256g_L200"]
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, adjoint=True)
    with torch.no_grad():
        target = cola.cola_density_from_noise(plan.noise(seed), plan).double()
    w = plan.noise(seed + 1000)
    x = w.clone().requires_grad_(True)
    loss = ((cola.cola_density_from_noise(x, plan).double() - target) ** 2).sum()
    loss.backward()
    grad = x.grad.double()

    def loss_at(v):
        with torch.no_grad():
            return float(((cola.cola_density_from_noise(v, plan).double() - target) ** 2).sum())

    eps, fd, an = 3e-4, [], []
    for m in range(64):
        e = dev(fourier_mode(n_p, 100 + m))
        fd.append((loss_at(w + eps * e) - loss_at(w - eps * e)) / (2 * eps))
        an.append(float((grad * e.double()).sum()))
    fd, an = np.array(fd), np.array(an)
    scale = np.sqrt(np.mean(an**2))
    err = np.abs(fd - an) / scale
    corr = float(np.corrcoef(fd, an)[0, 1])
    print(f"central differences on 64 modes: correlation {corr:.5f}, median |fd - adj| / rms(adj) "
          f"{np.median(err):.2e}, max {err.max():.2e}")
    # the kink and quantisation floor of central differences at a = 1 (module docstring):
    # measured on GB300, correlation 0.986 and median 4e-2; the float64 oracle's own central
    # differences scatter by 0.3-5% around its exact adjoint in the same regime at 32^3/64^3
    assert corr > 0.97
    assert np.median(err) < 0.1
