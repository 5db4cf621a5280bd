"""The allocation-free power-spectrum entry point against the plan-based one.

cola_power_noalloc is for callers that may not allocate device memory themselves: code
hosted in an application whose own pool allocator owns every device buffer, or a monitor
attached to a running simulation that must not change its memory footprint.  It keeps its
scratch in one static device array, so it must give the same answer as cola_power (a plan
with a caller-allocated workspace) on every call, including a second call in a row that finds
the first call's leftovers in that array.  Tolerances are those of the P(k) parity test:
mode counts exact, k within 1e-6 and P within 1e-5 relative.
"""
import numpy as np
import pytest
import torch

from paper_1301_0322_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cola():
    from paper_1301_0322_gb300 import build
    build.build(verbose=False)
    import paper_1301_0322_gb300 as c
    c.load_library()
    return c


@pytest.mark.parametrize("ng,box,nbins", [(32, 50.0, 16), (64, 100.0, 32), (96, 150.0, 48), (128, 250.0, 64),
                                         (128, 250.0, 128)])
def test_noalloc_power_matches_plan_power_on_consecutive_calls(cola, ng, box, nbins):
    # nbins = ng fills the shell-sum region up to its bound
    from paper_1301_0322_gb300.cola import cola_power_noalloc
    plan = cola.Plan(np_side=32, ng=ng, box=box)
    for call in range(2):
        d = torch.from_numpy(inputs.gaussian_noise(ng, 40 + call) * (0.3 + call)).cuda()
        k_ref, p_ref, n_ref = (t.cpu().numpy() for t in plan.power(d, nbins))
        k = torch.empty(nbins, dtype=torch.float64, device="cuda")
        p = torch.empty(nbins, dtype=torch.float64, device="cuda")
        n = torch.empty(nbins, dtype=torch.int64, device="cuda")
        cola_power_noalloc(d, ng, box, nbins, k, p, n)
        torch.cuda.synchronize()
        assert np.array_equal(n.cpu().numpy(), n_ref)
        assert np.allclose(k.cpu().numpy(), k_ref, rtol=1e-6)
        assert np.allclose(p.cpu().numpy(), p_ref, rtol=1e-5)


def test_noalloc_rejects_meshes_beyond_its_static_scratch(cola):
    from paper_1301_0322_gb300.cola import cola_power_noalloc
    d = torch.zeros(192**3, dtype=torch.float32, device="cuda")
    out = torch.empty(96, dtype=torch.float64, device="cuda")
    cnt = torch.empty(96, dtype=torch.int64, device="cuda")
    with pytest.raises(cola.ColaError) as e:
        cola_power_noalloc(d, 192, 100.0, 96, out, out, cnt)
    assert e.value.code == 1 and "static scratch" in str(e.value)
