"""GPU friends-of-friends (Sec. 3.2) against the oracle's brute-force groups.

Both sides use the same fixed-point positions and the exact integer linking rule, so the
groups, their labels (smallest member index), sizes and the mass function must agree exactly.
"""
import numpy as np
import pytest
import torch

from oracle import fof as ofof
from oracle import mesh as omesh
from paper_1301_0322_gb300 import inputs

pytestmark = pytest.mark.gpu

THRESHOLDS = [25, 50, 100, 200, 400, 800, 1600]


@pytest.fixture(scope="module")
def cola():
    from paper_1301_0322_gb300 import build
    build.build(verbose=False)
    import paper_1301_0322_gb300 as c
    c.load_library()
    return c


def check(cola, plan, s32, n_p, ng, box, b=(1, 5), nmin=25):
    group, size, n_ge = plan.fof(torch.from_numpy(s32).cuda(), nmin=nmin, b=b, thresholds=THRESHOLDS)
    plan.status()
    g, sz, ng_ = (t.cpu().numpy() for t in (group, size, n_ge))
    f = omesh.fixed_point_coords(s32, n_p, ng, box, 16)
    rg, rs = ofof.fof_groups(f, ng << 16, (ng // n_p) << 16, nmin, *b)
    assert np.array_equal(g, rg)
    assert np.array_equal(sz, rs)
    assert np.array_equal(ng_, ofof.mass_function(rg, rs, THRESHOLDS))
    return int(np.unique(rg[rg >= 0]).size)


@pytest.mark.parametrize("n_p,ng,box,seed", [(32, 64, 50.0, 3), (32, 96, 40.0, 4)])
def test_fof_of_clustered_particles(cola, n_p, ng, box, seed):
    plan = cola.Plan(np_side=n_p, ng=ng, box=box)
    s32 = inputs.clustered_displacements(n_p, box, seed)
    nhalo = check(cola, plan, s32, n_p, ng, box)
    assert nhalo >= 4


def test_fof_of_an_evolved_cola_box_and_other_linking_length(cola):
    n_p, ng, box = 32, 64, 25.0
    plan = cola.Plan(np_side=n_p, ng=ng, box=box)
    s, v, s1, s2 = plan.run(plan.noise(5))
    s32 = s.cpu().numpy()
    nhalo = check(cola, plan, s32, n_p, ng, box)
    print("halos at z = 0 (32^3 particles, L = 25 Mpc/h):", nhalo)
    check(cola, plan, s32, n_p, ng, box, b=(1, 4), nmin=10)
