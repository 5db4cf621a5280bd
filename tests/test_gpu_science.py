"""The paper's COLA-versus-PM comparison (Sec. 3.1, Fig. "cc"), reproduced with the GPU path.

Same initial conditions (64^3 particles on a 192^3 mesh, L = 100 Mpc/h: the paper's
mesh/particle ratio and box, 1/64 of its particles; Philox seed 2), evolved from z = 9 to 0:
  * reference: the standard PM leapfrog (eq. KDKStd) with 100 steps uniform in ln a (the grid
    App. A.2 prefers for it) -- a stand-in for the paper's many-step GADGET-2 truth;
  * COLA: eq. KDKALC, 10 steps uniform in a (the paper's optimal variant);
  * PM: eq. KDKStd, 10 steps uniform in ln a.
The paper finds that (i) 10-step PM underestimates P(k) by several percent even on the
largest scales while COLA does not, and (ii) COLA keeps the cross-correlation with the truth
above 95% out to a scale about 80% smaller than PM does.  Both are checked on rho(k) and P(k)
from cola_cross_power.  The float64 oracle run of the same set-up gives k(rho = 0.95) = 2.1
(COLA) and 1.1 h/Mpc (PM), P/P_ref = 0.99 (COLA) and 0.93 (PM) at k = 0.32 h/Mpc.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

N_P, NG, BOX, SEED = 64, 192, 100.0, 2


@pytest.fixture(scope="module")
def cola():
    from paper_1301_0322_gb300 import build
    build.build(verbose=False)
    import paper_1301_0322_gb300 as c
    c.load_library()
    return c


def final_density(cola, scheme, nsteps, log_a):
    plan = cola.Plan(np_side=N_P, ng=NG, box=BOX, scheme=scheme, nsteps=nsteps, log_a=log_a)
    s, v, s1, s2 = plan.run(plan.noise(SEED))
    _, delta = plan.density(s, rho=False)
    plan.status()
    return plan, delta


def k_at(k, rho, level):
    below = np.nonzero(rho < level)[0]
    return k[below[0]] if below.size else k[-1]


def test_cola_beats_pm_with_ten_steps(cola):
    plan, ref = final_density(cola, "pm_std", 100, True)
    _, d_cola = final_density(cola, "cola", 10, False)
    _, d_pm = final_density(cola, "pm_std", 10, True)
    nb = NG // 4
    out = {}
    for name, d in (("cola", d_cola), ("pm", d_pm)):
        k, pa, pb, pab, rho, nmax, nm = (t.cpu().numpy() for t in plan.cross_power(d, ref, nb))
        out[name] = (k, pa / pb, rho, nmax)
    torch.cuda.synchronize()
    k = out["cola"][0]
    k95 = {n: k_at(k, out[n][2], 0.95) for n in out}
    large = (k > 0.2) & (k < 0.4)
    ratio = {n: float(np.mean(out[n][1][large])) for n in out}
    print(f"k(rho=0.95): COLA {k95['cola']:.2f}, PM {k95['pm']:.2f} h/Mpc; "
          f"P/P_ref at 0.2-0.4 h/Mpc: COLA {ratio['cola']:.3f}, PM {ratio['pm']:.3f}")
    assert k95["cola"] >= 1.5 * k95["pm"]
    assert abs(ratio["cola"] - 1.0) <= 0.02
    assert ratio["pm"] <= 0.97
    # n_max of eq. nmax where rho < 1
    r, nmax = out["cola"][2], out["cola"][3]
    sel = np.abs(r) < 0.999999
    assert np.allclose(nmax[sel], 2.0 / 3.0 * r[sel] / np.sqrt(1.0 - r[sel] ** 2), rtol=1e-9)
