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


def test_union_retry_limit_reports_timeout_and_recovers(cola):
    # The union-find is a bounded loop: when its retries run out, cola_fof latches COLA_ETIMEOUT
    # (read by cola_status) instead of spinning.  With 0 tries every union gives up at once; with
    # 1 try on a dense clump the run either reports the timeout or has exact groups; afterwards
    # the default limit gives exact groups on the same plan (the context stays usable).
    n_p, ng, box = 32, 64, 50.0
    plan = cola.Plan(np_side=n_p, ng=ng, box=box)
    s32 = inputs.clustered_displacements(n_p, box, 3, nclump=2, frac=0.8, radius=0.3)
    s_dev = torch.from_numpy(s32).cuda()
    cola.cola_set_fof_union_tries(plan.handle, 0)
    plan.fof(s_dev, nmin=25, b=(1, 5), thresholds=THRESHOLDS)
    with pytest.raises(cola.ColaError) as e:
        plan.status()
    assert e.value.code == 6 and "union-find" in str(e.value)
    cola.cola_set_fof_union_tries(plan.handle, 1)
    group, size, n_ge = plan.fof(s_dev, nmin=25, b=(1, 5), thresholds=THRESHOLDS)
    try:
        plan.status()
        exact = True
    except cola.ColaError as err:
        assert err.code == 6
        exact = False
    if exact:
        f = omesh.fixed_point_coords(s32, n_p, ng, box, 16)
        rg, _ = ofof.fof_groups(f, ng << 16, (ng // n_p) << 16, 25, 1, 5)
        assert np.array_equal(group.cpu().numpy(), rg)
    with pytest.raises(cola.ColaError):
        cola.cola_set_fof_union_tries(plan.handle, -1)
    cola.cola_set_fof_union_tries(plan.handle, 1 << 20)
    assert check(cola, plan, s32, n_p, ng, box) >= 1
