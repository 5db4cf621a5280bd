"""Pins of oracle.mesh: Fourier convention, CIC deposit/gather, PM force on single modes,
momentum conservation (Sec. 2 PM code; App. A.1 eq. eom)."""
import itertools

import numpy as np
import pytest
import scipy.fft

from oracle import mesh


def naive_dft3(f):
    """Brute-force f_k = sum_x f(x) exp(-2 pi i n.x / N) over the full spectrum."""
    n = f.shape[0]
    idx = np.arange(n)
    e = np.exp(-2j * np.pi * np.outer(idx, idx) / n)
    out = np.zeros(f.shape, dtype=np.complex128)
    for kz, ky, kx in itertools.product(range(n), repeat=3):
        out[kz, ky, kx] = np.sum(f * e[kz][:, None, None] * e[ky][None, :, None] * e[kx][None, None, :])
    return out


def test_fft_convention_matches_naive_dft():
    rng = np.random.default_rng(3)
    f = rng.standard_normal((6, 6, 6))
    ref = naive_dft3(f)
    got = scipy.fft.rfftn(f)
    assert np.allclose(got, ref[:, :, :4], atol=1e-10)
    assert np.allclose(scipy.fft.irfftn(got, s=f.shape), f, atol=1e-12)


def brute_cic(pos, ng, box):
    rho = np.zeros((ng, ng, ng))
    h = box / ng
    for p in range(pos.shape[1]):
        for c in itertools.product(range(ng), repeat=3):  # c = (cz, cy, cx)
            w = 1.0
            for d, cd in zip((2, 1, 0), c):
                dx = pos[d, p] / h - cd
                dx -= ng * np.round(dx / ng)  # periodic image
                w *= max(0.0, 1.0 - abs(dx))
            rho[c] += w
    return rho


def test_cic_deposit_brute_force_and_mass():
    rng = np.random.default_rng(0)
    box, ng = 10.0, 6
    pos = rng.uniform(-3.0, 13.0, size=(3, 9))
    rho = mesh.cic_deposit(pos, ng, box)
    assert np.allclose(rho, brute_cic(pos, ng, box), atol=1e-12)
    assert rho.sum() == pytest.approx(9.0, abs=1e-12)
    on_node = np.array([[0.0, 5.0], [10.0 / 6 * 2, 0.0], [0.0, 10.0 / 6 * 5]])
    r2 = mesh.cic_deposit(on_node, ng, box)
    assert r2[0, 2, 0] == pytest.approx(1.0) and r2[5, 0, 3] == pytest.approx(1.0)
    assert r2.sum() == pytest.approx(2.0)


def brute_fixed(s32, n_p, ng, box, fbits):
    one = 1 << fbits
    scale32 = np.float32(ng / box)
    rho = {}
    for p in range(n_p**3):
        lat = (p % n_p, (p // n_p) % n_p, p // (n_p * n_p))
        cells, ts = [], []
        for d in range(3):
            q = (lat[d] * ng * one) // n_p
            w = np.float32(s32[d, p]) * scale32
            f = (q + int(np.floor(np.float64(w) * one))) % (ng * one)
            cells.append(f // one)
            ts.append(f % one)
        for dz, dy, dx in itertools.product((0, 1), repeat=3):
            wz = ts[2] if dz else one - ts[2]
            wy = ts[1] if dy else one - ts[1]
            wx = ts[0] if dx else one - ts[0]
            key = ((cells[2] + dz) % ng, (cells[1] + dy) % ng, (cells[0] + dx) % ng)
            rho[key] = rho.get(key, 0) + wz * wy * wx
    out = np.zeros((ng, ng, ng), dtype=np.int64)
    for k, v in rho.items():
        out[k] = v
    return out


@pytest.mark.parametrize("n_p,ng", [(4, 8), (3, 9), (4, 6)])
def test_fixed_point_deposit_brute_force(n_p, ng):
    rng = np.random.default_rng(n_p * 100 + ng)
    box, fbits = 50.0, 15
    s32 = rng.normal(0, 9.0, size=(3, n_p**3)).astype(np.float32)
    rho = mesh.cic_deposit_fixed(s32, n_p, ng, box, fbits)
    assert np.array_equal(rho, brute_fixed(s32, n_p, ng, box, fbits))
    assert int(rho.sum()) == n_p**3 * (1 << (3 * fbits))
    # agrees with the float64 CIC of the same positions to the fixed-point resolution
    q = mesh.lattice_q(n_p, box)
    ref = mesh.cic_deposit(q + s32.astype(np.float64), ng, box)
    assert np.abs(rho * 2.0 ** (-3 * fbits) - ref).max() < 8 * n_p**3 * 2.0**-fbits


def test_fixed_point_lattice_on_nodes():
    # zero displacement, integer mesh/particle ratio: each particle sits on a node
    n_p, ng, fbits = 4, 12, 15
    rho = mesh.cic_deposit_fixed(np.zeros((3, n_p**3), np.float32), n_p, ng, 100.0, fbits)
    expect = np.zeros((ng, ng, ng), dtype=np.int64)
    expect[::3, ::3, ::3] = 1 << (3 * fbits)
    assert np.array_equal(rho, expect)


def test_cic_gather_linear_and_constant():
    box, ng = 8.0, 8
    h = box / ng
    z, y, x = np.meshgrid(np.arange(ng), np.arange(ng), np.arange(ng), indexing="ij")
    lin = 2.0 * x * h - 0.5 * y * h + 0.25 * z * h + 1.0
    rng = np.random.default_rng(1)
    pos = rng.uniform(0.2, box - h - 0.2, size=(3, 50))  # no wrap across the box edge
    got = mesh.cic_gather(lin, pos, box)
    assert np.allclose(got, 2.0 * pos[0] - 0.5 * pos[1] + 0.25 * pos[2] + 1.0, atol=1e-12)
    assert np.allclose(mesh.cic_gather(np.full((ng,) * 3, 3.5), pos, box), 3.5)


@pytest.mark.parametrize("modes,deconv", [((3, 0, 0), 0), ((1, 2, 3), 0), ((2, -1, 4), 1), ((0, 5, 1), 2)])
def test_unit_force_single_mode(modes, deconv):
    # delta = A cos(k.x)  =>  g = -grad d^-2 delta = -A k sin(k.x) / k^2, times 1/W^p
    ng, box, amp = 16, 40.0, 0.3
    h = box / ng
    z, y, x = np.meshgrid(np.arange(ng) * h, np.arange(ng) * h, np.arange(ng) * h, indexing="ij")
    kf = 2 * np.pi / box
    kvec = kf * np.array(modes, dtype=float)
    phase = kvec[0] * x + kvec[1] * y + kvec[2] * z
    delta = amp * np.cos(phase)
    g = mesh.unit_force_mesh(delta, box, deconv)
    w = np.prod([np.sinc(m / ng) ** 2 for m in modes])
    k2 = kvec @ kvec
    for j in range(3):
        expect = -amp * kvec[j] * np.sin(phase) / k2 / w**deconv
        assert np.allclose(g[j], expect, atol=1e-12)


def test_force_zero_on_nyquist_plane():
    ng, box = 8, 8.0
    x = np.arange(ng)
    delta = np.cos(np.pi * x)[None, None, :] * np.cos(2 * np.pi * x / ng)[None, :, None] * np.ones((ng, 1, 1))
    gx, gy, gz = mesh.unit_force_mesh(delta, box, 0)
    assert np.abs(gx).max() < 1e-14  # x-gradient of the n_x = N/2 mode is zeroed
    assert np.abs(gy).max() > 1e-3 and np.abs(gz).max() < 1e-14


@pytest.mark.parametrize("deconv", [0, 1, 2])
def test_momentum_conservation_and_no_self_force(deconv):
    rng = np.random.default_rng(7)
    box, ng = 20.0, 12
    pos = rng.uniform(0, box, size=(3, 40))
    g = mesh.unit_force_particles(pos, 40, ng, box, deconv)
    assert np.abs(g.sum(axis=1)).max() < 1e-12 * np.abs(g).sum()
    single = rng.uniform(0, box, size=(3, 1))
    g1 = mesh.unit_force_particles(single, 1, ng, box, deconv)
    assert np.abs(g1).max() < 1e-13
    # pair forces are equal and opposite (Newton's third law on the mesh)
    pair = rng.uniform(0, box, size=(3, 2))
    g2 = mesh.unit_force_particles(pair, 2, ng, box, deconv)
    assert np.allclose(g2[:, 0], -g2[:, 1], atol=1e-13)


@pytest.mark.parametrize("n_p,ng,box,axis,m", [(16, 32, 50.0, 0, 1), (16, 32, 50.0, 1, 2), (12, 36, 40.0, 2, 1),
                                               (8, 32, 30.0, 0, 3)])
@pytest.mark.parametrize("deconv", [0, 1, 2])
def test_axis_wave_reduction_equals_the_3d_force(n_p, ng, box, axis, m, deconv):
    # the one-dimensional reduction of the PM force for a lattice displaced along one axis
    # (mesh side r * lattice side) against the brute three-dimensional deposit/FFT/gather
    k = 2 * np.pi * m / box
    line = (0.4 / k * np.sin(k * np.arange(n_p) * box / n_p)).astype(np.float32).astype(np.float64)
    q = mesh.lattice_q(n_p, box)
    idx = mesh.lattice_index(n_p)[axis]
    s = np.zeros_like(q)
    s[axis] = line[idx]
    g = mesh.unit_force_particles(np.mod(q + s, box), n_p**3, ng, box, deconv)
    ref = mesh.unit_force_axis_wave(line, axis, n_p, ng, box, deconv)
    scale = np.abs(ref).max()
    assert np.abs(g[axis] - ref[idx]).max() <= 1e-12 * scale
    assert np.abs(np.delete(g, axis, 0)).max() <= 1e-12 * scale



def test_quantised_positions_deposit_the_fixed_point_density():
    # displacements a fraction (0.1-0.9) of a quantum above a multiple of 2^-F cell: the float64
    # rounding-down of oracle.cola.quantise_positions and the library's fixed-point coordinates
    # agree, and the float64 CIC density of the quantised positions equals rho_fix / 2^3F
    from oracle.cola import quantise_positions
    n_p, ng, box, F = 8, 16, 16.0, 12  # H = 1 Mpc/h: cell units = Mpc/h
    rng = np.random.default_rng(11)
    k = rng.integers(-3000, 3000, size=(3, n_p**3))
    s = ((k + rng.uniform(0.1, 0.9, size=k.shape)) / 2.0**F).astype(np.float32)
    pos = np.mod(mesh.lattice_q(n_p, box) + s.astype(np.float64), box)
    rho = mesh.cic_deposit(quantise_positions(pos, ng, box, F), ng, box)
    fixed = mesh.cic_deposit_fixed(s, n_p, ng, box, F).astype(np.float64) / 2.0 ** (3 * F)
    assert np.abs(rho - fixed).max() <= 1e-12 * fixed.max()
