"""Parity at the full single-box sizes: 256^3 particles on a 768^3 mesh (L = 100 Mpc/h, the
benchmark workload, in the launch configuration the benchmark times) and 1024^3 particles on a
2048^3 mesh (L = 1000 Mpc/h).

The three-dimensional oracle cannot run at these sizes (one float64 mesh is 3.6 GB at 768^3 and
69 GB at 2048^3, and its transforms take minutes), so the force is checked on inputs whose PM
force the oracle computes exactly in one dimension: a lattice displaced by a plane wave along
one axis (oracle.mesh.unit_force_axis_wave, pinned against the brute 3-D force in
test_oracle_mesh.py).  One force evaluation per axis runs every fused pass (deposit + x r2c,
forward y, z with the Green's function, the inverse y and x passes) and the gather, with the
transform axis of the wave different each time.  Tolerance as the small-size force parity:
3e-4 of max |g| (positions quantised to 2^-16 cell, float32 transforms); the transverse
components vanish up to float32 rounding.

A full COLA step at each size (2LPT from Philox seed 3, first kick + drift) then checks the
error flags, finiteness and momentum conservation.
"""
import numpy as np
import pytest
import torch

from oracle import mesh as omesh

pytestmark = pytest.mark.gpu

# (particles per side, mesh, box in Mpc/h, device bytes needed: workspace + particle arrays)
SIZES = {768: (256, 768, 100.0, 16 * 10**9), 2048: (1024, 2048, 1000.0, 250 * 10**9)}


@pytest.fixture(scope="module")
def cola():
    from paper_1301_0322_gb300 import build
    build.build(verbose=False)
    import paper_1301_0322_gb300 as c
    c.load_library()
    return c


@pytest.fixture(scope="module", params=sorted(SIZES))
def big_plan(cola, request):
    n_p, ng, box, needed = SIZES[request.param]
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < needed:
        pytest.skip(f"needs {needed / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")
    plan = cola.Plan(np_side=n_p, ng=ng, box=box)
    yield plan, n_p, ng, box
    del plan
    torch.cuda.empty_cache()


@pytest.mark.parametrize("axis,m", [(0, 1), (1, 2), (2, 5)])
def test_plane_wave_force_at_full_size(big_plan, axis, m):
    big_plan, N_P, NG, BOX = big_plan
    k = 2 * np.pi * m / BOX
    line = (0.4 / k * np.sin(k * np.arange(N_P) * BOX / N_P)).astype(np.float32)
    shape = [1, 1, 1]
    shape[2 - axis] = N_P  # [iz][iy][ix]
    line_d = torch.from_numpy(line).cuda().view(shape)
    s = torch.zeros((3, N_P, N_P, N_P), dtype=torch.float32, device="cuda")
    s[axis].copy_(line_d.expand(N_P, N_P, N_P))
    g = big_plan.force(s.view(3, -1)).view(3, N_P, N_P, N_P)
    del s
    big_plan.status()
    ref = omesh.unit_force_axis_wave(line.astype(np.float64), axis, N_P, NG, BOX, deconv=1)
    scale = np.abs(ref).max()
    ref_d = torch.from_numpy(ref).cuda().view(shape)
    err, trans = 0.0, 0.0
    for z in range(0, N_P, 64):
        chunk = g[:, z:z + 64].double()
        refc = ref_d if axis != 2 else ref_d[z:z + 64]
        err = max(err, float((chunk[axis] - refc).abs().max()))
        others = [c for c in range(3) if c != axis]
        trans = max(trans, float(chunk[others].abs().max()))
    print(f"N = {NG}, axis {axis}, mode {m}: max |g - g_oracle| / max |g| = {err / scale:.2e}, "
          f"transverse {trans / scale:.2e}")
    assert err <= 3e-4 * scale
    assert trans <= 1e-4 * scale


def test_full_step_at_full_size_conserves_momentum(cola, big_plan):
    # 2LPT initial conditions from Philox seed 3, then the first kick + drift: the PM force
    # sums to zero over the particles (antisymmetric operator, same deposit and gather
    # weights) and s1, s2 have zero mean, so the kicked velocities sum to ~0
    big_plan = big_plan[0]
    noise = big_plan.noise(3)
    s, v, s1, s2 = big_plan.ic_2lpt(noise)
    del noise
    big_plan.step(0, s, v, s1, s2)
    big_plan.status()
    del s1, s2
    tot, mag, finite = torch.zeros(3, dtype=torch.float64, device="cuda"), 0.0, True
    for c in range(0, v.shape[1], 1 << 24):
        chunk = v[:, c:c + (1 << 24)].double()
        tot += chunk.sum(dim=1)
        mag += float(chunk.abs().sum())
        finite = finite and bool(torch.isfinite(chunk).all()) and bool(torch.isfinite(s[:, c:c + (1 << 24)]).all())
    assert finite
    print(f"|sum v| / sum |v| = {float(tot.abs().max()) / mag:.2e}")
    assert float(tot.abs().max()) <= 1e-5 * mag
