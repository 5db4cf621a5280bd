"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances (float32 kernels against float64 references):
  * integer CIC deposit: bit-exact (same float32 positions on both sides);
  * FFT: rms error <= 4e-6 and max error <= 4e-5 of the rms amplitude (float32 Stockham
    with float64-derived twiddles: about eps * log2(N^3) ~ 1e-6 rms);
  * unit force at particles: max error <= 3e-4 of max |g| (positions quantised to 2^-16 cell
    on the GPU, float64 on the oracle side: |grad g| 2^-16 H ~ 2e-5 |g|, plus float32 FFTs);
  * after a full 10-step run: |ds| <= 1e-3 mesh cells and P(k) relative error <= 1e-4 for
    k < k_Nyquist / 2 (the stated targets).  The float64 oracle with its own positions
    quantised to 2^-F cell differs from itself unquantised by 1.0e-3 (F = 15) and 5.1e-4
    (F = 16) cells at 32^3/64^3: the 2^-F quantisation, amplified by the nonlinear dynamics,
    is the dominant difference, hence the default F = 16.
"""
import numpy as np
import pytest
import scipy.fft
import torch

from oracle import cola as ocola
from oracle import lpt as olpt
from oracle import mesh as omesh
from oracle import power as opower
from oracle.cosmology import Cosmology, time_grid
from oracle.philox import white_noise
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
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("n", [32, 48, 64, 96, 128, 192, 256])
def test_fft_r2c_matches_numpy(cola, n):
    plan = cola.Plan(np_side=32, ng=n, box=100.0)
    x = inputs.gaussian_noise(n, 100 + n)
    got = host(plan.fft_r2c(dev(x), which=0))
    ref = scipy.fft.rfftn(x.reshape(n, n, n).astype(np.float64))
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    err = np.abs(got - ref)
    assert np.sqrt(np.mean(err**2)) <= 4e-6 * rms
    assert err.max() <= 4e-5 * rms
    plan.status()


def test_fft_lattice_transform(cola):
    plan = cola.Plan(np_side=48, ng=96, box=150.0)
    x = inputs.gaussian_noise(48, 5)
    got = host(plan.fft_r2c(dev(x), which=1))
    ref = scipy.fft.rfftn(x.reshape(48, 48, 48).astype(np.float64))
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.abs(got - ref).max() <= 4e-5 * rms


@pytest.mark.parametrize("n", [32, 48])
def test_noise_matches_oracle_philox(cola, n):
    plan = cola.Plan(np_side=n, ng=2 * n)
    for seed in (1, 0x1234567890):
        got = host(plan.noise(seed))
        ref = white_noise(n, seed).reshape(-1)
        assert np.abs(got - ref).max() < 2e-5
        assert abs(got.mean()) < 0.05 and abs(got.std() - 1) < 0.05


def deposit_cases():
    return [
        (32, 64, 100.0, inputs.gaussian_displacements(32, 1.5, 1)),
        (32, 96, 100.0, inputs.gaussian_displacements(32, 0.7, 2)),
        (48, 96, 150.0, inputs.clustered_displacements(48, 150.0, 3)),
        (32, 64, 100.0, inputs.clustered_displacements(32, 100.0, 4, frac=0.9, radius=0.05)),
        (32, 64, 100.0, np.zeros((3, 32**3), np.float32)),  # every particle on a node
        (32, 64, 100.0, inputs.gaussian_displacements(32, 60.0, 5)),  # crosses the box
    ]


@pytest.mark.parametrize("case", range(6))
def test_deposit_bit_exact(cola, case):
    n_p, ng, box, s = deposit_cases()[case]
    plan = cola.Plan(np_side=n_p, ng=ng, box=box)
    rho, delta = plan.density(dev(s))
    rho = host(rho).reshape(ng, ng, ng)
    ref = omesh.cic_deposit_fixed(s, n_p, ng, box, 16)
    # exact total mass (the global sum can exceed int64, so add the high and low parts apart)
    total = int((rho >> 24).sum()) * 2**24 + int((rho & (2**24 - 1)).sum())
    assert total == n_p**3 * 2**48
    assert np.array_equal(rho, ref)
    d = host(delta).reshape(ng, ng, ng)
    dref = ref.astype(np.float64) * (ng**3 / (n_p**3 * 2.0**48)) - 1.0
    assert np.abs(d - dref).max() <= 1e-6 * (1.0 + np.abs(dref).max())
    # exactly fma(float32(rho), dscale, -1): the integer rounded to the nearest float32 (ties to
    # even), times dscale = (ng/np)^3 2^-48 (a float32 without rounding), minus 1 with one rounding
    # (the float64 product is exact; the float64 subtraction is exact unless rho is tiny)
    d32 = (ref.astype(np.float32).astype(np.float64) * (ng**3 / (n_p**3 * 2.0**48)) - 1.0).astype(np.float32)
    assert np.array_equal(d, d32)
    plan.status()


# the smallest meshes (32, 48: 8-thread deposit blocks), a lattice as fine as the mesh and one
# finer than it
@pytest.mark.parametrize("n_p,ng,deconv", [(32, 64, 1), (32, 64, 0), (32, 96, 2), (48, 96, 1), (32, 48, 1),
                                           (32, 32, 1), (48, 32, 1), (48, 48, 0)])
def test_unit_force_matches_oracle(cola, n_p, ng, deconv):
    box = 100.0
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, deconv=deconv)
    s = inputs.gaussian_displacements(n_p, 1.0, 11)
    g = host(plan.force(dev(s)))
    pos = omesh.lattice_q(n_p, box) + s.astype(np.float64)
    ref = omesh.unit_force_particles(np.mod(pos, box), n_p**3, ng, box, deconv)
    assert np.abs(g - ref).max() <= 3e-4 * np.abs(ref).max()
    # momentum conservation of the GPU force
    assert np.abs(g.astype(np.float64).sum(axis=1)).max() <= 1e-5 * np.abs(g).sum()


@pytest.mark.parametrize("n_p,box", [(32, 100.0), (48, 150.0)])
def test_ic_2lpt_matches_oracle(cola, n_p, box):
    plan = cola.Plan(np_side=n_p, ng=2 * n_p, box=box)
    w = inputs.gaussian_noise(n_p, 21)
    s, v, s1, s2 = (host(t) for t in plan.ic_2lpt(dev(w)))
    cosmo = Cosmology(**inputs.COSMOLOGY)
    r1, r2 = olpt.ic_2lpt(w.reshape(n_p, n_p, n_p).astype(np.float64), box, cosmo)
    assert np.abs(s1 - r1).max() <= 2e-5 * np.abs(r1).max()
    assert np.abs(s2 - r2).max() <= 2e-4 * np.abs(r2).max()
    g = cosmo.growth([0.1])
    sref = g["D1"][0] * r1 + g["D2"][0] * r2
    assert np.abs(s - sref).max() <= 2e-5 * np.abs(sref).max()
    assert np.all(v == 0.0)


@pytest.mark.parametrize("ng,nbins", [(64, 32), (96, 48), (384, 384)])
def test_power_matches_oracle(cola, ng, nbins):
    box = 100.0
    plan = cola.Plan(np_side=32, ng=ng, box=box)
    d = inputs.gaussian_noise(ng, 31) * 0.3
    k, p, nm = (host(t) for t in plan.power(dev(d), nbins))
    kr, pr, nr = opower.power_spectrum(d.reshape(ng, ng, ng).astype(np.float64), box, nbins)
    assert np.array_equal(nm, nr)
    assert np.allclose(k, kr, rtol=1e-6)
    assert np.allclose(p, pr, rtol=1e-5)


def gpu_run(cola, plan, w):
    s, v, s1, s2 = plan.ic_2lpt(dev(w))
    for i in range(plan.nsteps + 1):
        plan.step(i, s, v, s1, s2)
    plan.status()
    return s, v


# the paper's optimal variant (eq. KDKALC, steps uniform in a), the other discretisations of
# App. A (eq. KDKALCstd; the standard PM leapfrog eq. KDKStd; u = 1 in the Drift) and steps
# uniform in ln a (App. A.2)
@pytest.mark.parametrize("scheme,log_a", [("cola", False), ("cola_std", False), ("pm_std", False),
                                          ("cola_u1", False), ("cola", True), ("pm_std", True)])
def test_full_run_parity_32p_64g(cola, scheme, log_a):
    n_p, ng, box = 32, 64, 100.0
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, scheme=scheme, log_a=log_a)
    w = inputs.gaussian_noise(n_p, 1)
    s, v = gpu_run(cola, plan, w)
    sg, vg = host(s), host(v)
    cfg = ocola.ColaConfig(n_p=n_p, n_g=ng, box=box, spacing="loga" if log_a else "a")
    ref = ocola.run(w.reshape(n_p, n_p, n_p).astype(np.float64), cfg, scheme=scheme)
    cell = box / ng
    ds = np.abs(sg - ref["s"]).max() / cell
    print("max |ds| in cells:", ds, " max |dv|/rms v:", np.abs(vg - ref["v"]).max() / np.sqrt(np.mean(ref["v"] ** 2)))
    assert ds <= 1e-3
    assert np.abs(vg - ref["v"]).max() <= 1e-3 * np.sqrt(np.mean(ref["v"] ** 2))
    # P(k) of the final density, k < k_Nyquist / 2
    _, d = plan.density(s, rho=False)
    nb = ng // 4
    k, p, nm = (host(t) for t in plan.power(d, nb))
    # the same spectrum with no density mesh of the caller's: the same kernels, bit for bit
    k2, p2, nm2 = (host(t) for t in plan.density_power(s, nb))
    assert np.array_equal(k2, k) and np.array_equal(p2, p) and np.array_equal(nm2, nm)
    pos = np.mod(omesh.lattice_q(n_p, box) + ref["s"], box)
    dref = omesh.overdensity(omesh.cic_deposit(pos, ng, box), n_p**3)
    _, pr, nr = opower.power_spectrum(dref, box, nb)
    assert np.array_equal(nm, nr)
    rel = np.abs(p / pr - 1.0)
    print("max P(k) relative error:", rel.max())
    assert rel.max() <= 1e-4


def test_runs_are_deterministic(cola):
    plan = cola.Plan(np_side=32, ng=64, box=100.0)
    w = inputs.gaussian_noise(32, 3)
    s1_, v1_ = (host(t) for t in gpu_run(cola, plan, w))
    s2_, v2_ = (host(t) for t in gpu_run(cola, plan, w))
    assert np.array_equal(s1_, s2_) and np.array_equal(v1_, v2_)


def test_nonfinite_positions_are_reported(cola):
    plan = cola.Plan(np_side=32, ng=64)
    s = np.zeros((3, 32**3), np.float32)
    s[1, 77] = np.nan
    plan.density(dev(s), rho=True, delta=False)
    with pytest.raises(cola.ColaError) as e:
        plan.status()
    assert e.value.code == 3
    plan.status()  # the error was cleared


def test_cross_power_in_shell_ranges_matches_oracle(cola):
    # 384 shells of five sums each are more than one binning launch takes (352): binned in two
    # ranges of 192; two correlated fields, so that P_ab stays away from zero
    ng, box, nb = 384, 100.0, 384
    plan = cola.Plan(np_side=32, ng=ng, box=box)
    da = inputs.gaussian_noise(ng, 41) * 0.3
    db = da + 0.5 * inputs.gaussian_noise(ng, 42) * 0.3
    got = [host(t) for t in plan.cross_power(dev(da), dev(db), nb)]
    plan.status()
    ref = opower.cross_correlation(da.reshape(ng, ng, ng).astype(np.float64),
                                   db.reshape(ng, ng, ng).astype(np.float64), box, nb)
    k, pa, pb, pab, rho, nmax, nm = got
    assert np.array_equal(nm, ref[6])
    full = ref[6] > 0  # shells beyond |n| = sqrt(3) ng/2 hold no mode
    assert full.sum() > 300 and np.all(pa[~full] == 0.0)
    assert np.allclose(k, ref[0], rtol=1e-6)
    for g_, r_ in ((pa, ref[1]), (pb, ref[2]), (pab, ref[3])):
        assert np.abs(g_[full] / r_[full] - 1.0).max() <= 1e-4
    assert np.abs(rho[full] - ref[4][full]).max() <= 1e-5


def test_cross_power_matches_oracle(cola):
    # rho(k) and n_max(k) (Sec. 3.1, eq. nmax) between the 10-step COLA run and the 10-step
    # standard PM run of the same initial conditions, the paper's comparison; the oracle
    # evaluates the estimator in float64 on the same float32 density meshes
    n_p, ng, box = 32, 64, 100.0
    w = inputs.gaussian_noise(n_p, 1)
    deltas = []
    for scheme in ("cola", "pm_std"):
        plan = cola.Plan(np_side=n_p, ng=ng, box=box, scheme=scheme)
        s, _ = gpu_run(cola, plan, w)
        deltas.append(plan.density(s, rho=False)[1])
    nb = ng // 2
    got = [host(t) for t in plan.cross_power(deltas[0], deltas[1], nb)]
    plan.status()
    da, db = (host(d).reshape(ng, ng, ng).astype(np.float64) for d in deltas)
    ref = opower.cross_correlation(da, db, box, nb)
    k, pa, pb, pab, rho, nmax, nm = got
    assert np.array_equal(nm, ref[6])
    assert np.allclose(k, ref[0], rtol=1e-6)
    for g_, r_ in ((pa, ref[1]), (pb, ref[2]), (pab, ref[3])):
        assert np.abs(g_ / r_ - 1.0).max() <= 1e-4
    assert np.abs(rho - ref[4]).max() <= 1e-5
    slope = (2.0 / 3.0) / (1.0 - ref[4] ** 2) ** 1.5  # d n_max / d rho
    assert np.all(np.abs(nmax - ref[5]) <= 1e-5 * slope + 1e-9)
    print("rho(k) COLA vs PM, first bins:", np.round(rho[:8], 5))
    # a field with itself
    _, _, _, _, rho_self, _, _ = (host(t) for t in plan.cross_power(deltas[0], deltas[0], nb))
    assert np.abs(rho_self - 1.0).max() <= 1e-12



@pytest.mark.parametrize("fbits", [8, 12, 18])
def test_deposit_bit_exact_other_fixed_point_widths(cola, fbits):
    # at F = 18 one cell holds at most 2^8 particles below the 2^62 guard: smooth displacements
    n_p, ng, box = 32, 64, 100.0
    s = inputs.gaussian_displacements(n_p, 1.5, 6)
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, fixed_bits=fbits)
    rho, _ = plan.density(dev(s), delta=False)
    assert np.array_equal(host(rho).reshape(ng, ng, ng), omesh.cic_deposit_fixed(s, n_p, ng, box, fbits))
    plan.status()


def test_fixed_point_overflow_is_reported_by_both_deposits(cola):
    # every particle on one node: 32^3 x 2^48 = 2^63 of integer weight, above the 2^62 guard
    n_p, ng, box = 32, 64, 100.0
    q = omesh.lattice_q(n_p, box)
    s = (box / ng * 10.0 - q).astype(np.float32)  # every particle on node (10, 10, 10)
    plan = cola.Plan(np_side=n_p, ng=ng, box=box)
    plan.density(dev(s), rho=True, delta=False)
    with pytest.raises(cola.ColaError) as e:
        plan.status()
    assert e.value.code == 3
    plan.force(dev(s))  # the fused deposit of the force path
    with pytest.raises(cola.ColaError) as e:
        plan.status()
    assert e.value.code == 3
    plan.status()


@pytest.mark.parametrize("nsteps", [1, 3, 10])
def test_runs_match_the_quantised_oracle(cola, nsteps):
    # the oracle with the force's positions rounded to 2^-16 cell as the library's fixed-point
    # CIC rounds them: what is left is float32 rounding.  One step is a single K-D-K plus the
    # final kick and L+ (eq. ALCtimestep with n = 0).  Against the unquantised oracle the same
    # runs differ by the quantisation itself (1.7e-3 cell after one step from seed 2, the
    # largest step), which the oracle reproduces on its own.
    n_p, ng, box = 32, 64, 100.0
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, nsteps=nsteps)
    w = inputs.gaussian_noise(n_p, 2)
    s, v = gpu_run(cola, plan, w)
    w64 = w.reshape(n_p, n_p, n_p).astype(np.float64)
    ref_q = ocola.run(w64, ocola.ColaConfig(n_p=n_p, n_g=ng, box=box, nsteps=nsteps, fixed_bits=16))
    ref = ocola.run(w64, ocola.ColaConfig(n_p=n_p, n_g=ng, box=box, nsteps=nsteps))
    cell = box / ng
    sg, vg = host(s), host(v)
    ds_q = np.abs(sg - ref_q["s"]).max() / cell
    dv_q = np.abs(vg - ref_q["v"]).max() / np.sqrt(np.mean(ref_q["v"] ** 2))
    print(f"{nsteps} steps: |ds| vs quantised oracle {ds_q:.2e} cell, |dv|/rms {dv_q:.2e}; vs exact oracle "
          f"{np.abs(sg - ref['s']).max() / cell:.2e} cell; quantised vs exact oracle "
          f"{np.abs(ref_q['s'] - ref['s']).max() / cell:.2e} cell")
    assert ds_q <= 1e-3
    assert dv_q <= 1e-3


def test_mesh_coarser_than_the_lattice_gathers_in_lattice_order(cola):
    # 48^3 particles on a 32^3 mesh: a half spectrum (32^2 x 20 complex) cannot hold one force
    # component per particle, so the step gathers in lattice order (k_gather_kick_drift)
    # instead of in bin order; the run must still follow the quantised oracle (also a
    # lattice that is not an integer multiple of the mesh: fixed-point origin by division)
    import ctypes
    n_p, ng, box, nsteps = 48, 32, 100.0, 3
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, nsteps=nsteps)
    lib = cola.load_library()
    lib.cola_profile(plan.handle, 1)
    w = inputs.gaussian_noise(n_p, 2)
    s, v = gpu_run(cola, plan, w)
    lib.cola_profile(plan.handle, 0)
    names = ctypes.create_string_buffer(64 * 64)
    launches, ms, count = (ctypes.c_int64 * 64)(), (ctypes.c_double * 64)(), ctypes.c_int32()
    lib.cola_profile_read(plan.handle, 64, names, launches, ms, ctypes.byref(count))
    kernels = {names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode() for i in range(count.value)}
    assert "gather_kick_drift" in kernels and "gather_binned" not in kernels
    w64 = w.reshape(n_p, n_p, n_p).astype(np.float64)
    ref_q = ocola.run(w64, ocola.ColaConfig(n_p=n_p, n_g=ng, box=box, nsteps=nsteps, fixed_bits=16))
    cell = box / ng
    sg, vg = host(s), host(v)
    assert np.abs(sg - ref_q["s"]).max() / cell <= 1e-3
    assert np.abs(vg - ref_q["v"]).max() / np.sqrt(np.mean(ref_q["v"] ** 2)) <= 1e-3


# larger boxes against the quantised oracle over all 10 steps: an ensemble-sized box (64^3 /
# 128^3, L = 200 Mpc/h), every particle within 1e-3 cell
def test_larger_run_matches_the_quantised_oracle(cola):
    n_p, ng, box, seed, nsteps = 64, 128, 200.0, 5, 10
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, nsteps=nsteps)
    w = inputs.gaussian_noise(n_p, seed)
    s, v = gpu_run(cola, plan, w)
    ref_q = ocola.run(w.reshape(n_p, n_p, n_p).astype(np.float64),
                      ocola.ColaConfig(n_p=n_p, n_g=ng, box=box, nsteps=nsteps, fixed_bits=16))
    cell = box / ng
    ds = np.abs(host(s) - ref_q["s"]).max() / cell
    dv = np.abs(host(v) - ref_q["v"]).max() / np.sqrt(np.mean(ref_q["v"] ** 2))
    print(f"{n_p}^3 / {ng}^3, L = {box}: |ds| {ds:.2e} cell, |dv|/rms {dv:.2e}")
    assert ds <= 1e-3
    assert dv <= 1e-3


def test_run_at_the_benchmark_resolution_tracks_the_oracle(cola):
    # a sub-volume at the 256^3 / 768^3 benchmark's resolution (64^3 / 192^3, L = 25 Mpc/h: the
    # same 0.13 Mpc/h cells and 3 cells per particle spacing), strongly nonlinear after 10 steps.
    # There the dynamics amplify rounding: the float64 oracle itself moves by up to 7e-3 cell
    # when its noise is perturbed by one float32 rounding (2^-24 relative).  The bulk of the
    # particles must agree to 1e-3 cell, and the largest deviations may not exceed 3x the
    # oracle's own response to that perturbation.
    n_p, ng, box, seed, nsteps = 64, 192, 25.0, 6, 10
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, nsteps=nsteps)
    w = inputs.gaussian_noise(n_p, seed)
    s, v = gpu_run(cola, plan, w)
    cfg = ocola.ColaConfig(n_p=n_p, n_g=ng, box=box, nsteps=nsteps, fixed_bits=16)
    w64 = w.reshape(n_p, n_p, n_p).astype(np.float64)
    ref = ocola.run(w64, cfg)
    flip = np.random.default_rng(1).choice([-1.0, 1.0], size=w64.shape)
    ref_p = ocola.run(w64 * (1.0 + 2.0**-24 * flip), cfg)
    cell = box / ng
    vrms = np.sqrt(np.mean(ref["v"] ** 2))
    d_gpu = np.abs(host(s) - ref["s"]).max(axis=0) / cell
    d_own = np.abs(ref_p["s"] - ref["s"]).max(axis=0) / cell
    dv_gpu = np.abs(host(v) - ref["v"]).max() / vrms
    dv_own = np.abs(ref_p["v"] - ref["v"]).max() / vrms
    print(f"GPU vs oracle: |ds| max {d_gpu.max():.2e}, p99 {np.quantile(d_gpu, 0.99):.2e}, median "
          f"{np.median(d_gpu):.2e} cell, |dv|/rms {dv_gpu:.2e}; oracle vs perturbed oracle: |ds| max "
          f"{d_own.max():.2e}, p99 {np.quantile(d_own, 0.99):.2e} cell, |dv|/rms {dv_own:.2e}")
    assert np.quantile(d_gpu, 0.99) <= 1e-3
    assert np.median(d_gpu) <= 1e-4
    assert d_gpu.max() <= 3.0 * d_own.max()
    assert dv_gpu <= 3.0 * dv_own
    # P(k) of the final density for k < k_Nyquist / 2 (the stated 1e-4 target; the oracle's own
    # response to the one-rounding perturbation is 2.4e-6 here)
    _, d = plan.density(s, rho=False)
    nb = ng // 4
    k, p, nm = (host(t) for t in plan.power(d, nb))
    # the same spectrum with no density mesh of the caller's: the same kernels, bit for bit
    k2, p2, nm2 = (host(t) for t in plan.density_power(s, nb))
    assert np.array_equal(k2, k) and np.array_equal(p2, p) and np.array_equal(nm2, nm)
    pos = np.mod(omesh.lattice_q(n_p, box) + ref["s"], box)
    dref = omesh.overdensity(omesh.cic_deposit(pos, ng, box), n_p**3)
    _, pr, nr = opower.power_spectrum(dref, box, nb)
    assert np.array_equal(nm, nr)
    rel = np.abs(p / pr - 1.0)
    print(f"P(k) relative error, k < k_Ny/2: max {rel.max():.2e}")
    assert rel.max() <= 1e-4


def test_one_step_at_the_benchmark_sub_volume_matches_the_oracle(cola):
    # the 1/8 sub-volume of the 256^3 / 768^3 benchmark (128^3 particles, 384^3 mesh, L = 50
    # Mpc/h, seed 2) in the benchmark's launch configuration: 2LPT initial conditions, then the
    # first step of eq. ALCtimestep (force at a_0, Kick to a_1/2, Drift to a_1), every particle
    # against the float64 oracle (positions quantised to 2^-16 cell as the fixed-point CIC does)
    n_p, ng, box, seed = inputs.WORKLOADS["cola_128p_384g_L50"]
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, nsteps=10)
    w = inputs.gaussian_noise(n_p, seed)
    s, v, s1, s2 = plan.ic_2lpt(dev(w))
    plan.step(0, s, v, s1, s2)
    plan.status()
    cosmo = Cosmology(**inputs.COSMOLOGY)
    cfg = ocola.ColaConfig(n_p=n_p, n_g=ng, box=box, cosmo=cosmo, nsteps=10, fixed_bits=16)
    r1, r2 = olpt.ic_2lpt(w.reshape(n_p, n_p, n_p).astype(np.float64), box, cosmo)
    a, mid = time_grid(cfg.a_init, cfg.a_final, cfg.nsteps)
    g = cosmo.growth(a)
    rs = g["D1"][0] * r1 + g["D2"][0] * r2
    acc = ocola.acceleration(rs, cfg, a[0])
    rv = cosmo.kick_cola(a[0], mid[0], a[0], cfg.n_lpt) * (acc - g["T2D1"][0] * r1 - g["T2D2"][0] * r2)
    rs = rs + cosmo.drift_cola(a[0], a[1], mid[0], cfg.n_lpt) * rv + (g["D1"][1] - g["D1"][0]) * r1 \
        + (g["D2"][1] - g["D2"][0]) * r2
    cell = box / ng
    ds = np.abs(host(s) - rs).max() / cell
    dv = np.abs(host(v) - rv).max() / np.sqrt(np.mean(rv**2))
    print(f"one step at 128^3 / 384^3: |ds| {ds:.2e} cell, |dv| / rms {dv:.2e}")
    assert ds <= 1e-3
    assert dv <= 1e-3


@pytest.mark.parametrize("n_lpt", [-2.0, -3.0])
def test_other_nlpt_runs_match_the_oracle(cola, n_lpt):
    # the modified Kick/Drift of eq. KDKALC with u = a^nLPT at the other ends of the paper's
    # +-0.5 range around nLPT = -2.5 (App. A.3.2): full 10-step runs against the quantised
    # oracle, positions, velocities and P(k)
    n_p, ng, box = 32, 64, 100.0
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, n_lpt=n_lpt)
    w = inputs.gaussian_noise(n_p, 2)
    s, v = gpu_run(cola, plan, w)
    ref = ocola.run(w.reshape(n_p, n_p, n_p).astype(np.float64),
                    ocola.ColaConfig(n_p=n_p, n_g=ng, box=box, n_lpt=n_lpt, fixed_bits=16))
    cell = box / ng
    ds = np.abs(host(s) - ref["s"]).max() / cell
    dv = np.abs(host(v) - ref["v"]).max() / np.sqrt(np.mean(ref["v"] ** 2))
    _, d = plan.density(s, rho=False)
    nb = ng // 4
    _, p, _ = (host(t) for t in plan.power(d, nb))
    pos = np.mod(omesh.lattice_q(n_p, box) + ref["s"], box)
    _, pr, _ = opower.power_spectrum(omesh.overdensity(omesh.cic_deposit(pos, ng, box), n_p**3), box, nb)
    rel = np.abs(p / pr - 1.0).max()
    print(f"nLPT = {n_lpt}: |ds| {ds:.2e} cell, |dv|/rms {dv:.2e}, P(k) {rel:.2e}")
    assert ds <= 1e-3 and dv <= 1e-3 and rel <= 1e-4
