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


@pytest.fixture(scope="module")
def reference(cola):
    return final_density(cola, "pm_std", 100, True)


def test_cola_beats_pm_with_ten_steps(cola, reference):
    plan, ref = reference
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


def test_nlpt_half_unit_changes_have_no_noticeable_effect(cola, reference):
    # App. A.3.2: nLPT = -2.5 was chosen by a global fit, and moving it by +-0.5 has no
    # noticeable effect.  Against the same 100-step reference, the 10-step COLA runs with
    # nLPT = -2, -2.5 and -3 keep rho > 0.95 to within 10% of the same scale, agree on rho(k)
    # at k = 1 and 2 h/Mpc to 0.005 and 0.01, and reproduce the large-scale power to 2% (the
    # float64 oracle of this set-up: k(rho = 0.95) = 2.33, 2.26, 2.20 h/Mpc; P/P_ref on
    # 0.2-0.4 h/Mpc = 0.983, 0.987, 0.991), while 10-step PM stays far behind all three.
    plan, ref = reference
    nb = NG // 4
    out = {}
    for n_lpt in (-2.0, -2.5, -3.0):
        p = cola.Plan(np_side=N_P, ng=NG, box=BOX, scheme="cola", nsteps=10, n_lpt=n_lpt)
        s, v, s1, s2 = p.run(p.noise(SEED))
        _, d = p.density(s, rho=False)
        p.status()
        k, pa, pb, pab, rho, nmax, nm = (t.cpu().numpy() for t in plan.cross_power(d, ref, nb))
        large = (k > 0.2) & (k < 0.4)
        out[n_lpt] = (k_at(k, rho, 0.95), float(np.mean((pa / pb)[large])), np.interp(1.0, k, rho),
                      np.interp(2.0, k, rho))
    _, d_pm = final_density(cola, "pm_std", 10, True)
    k, _, _, _, rho_pm, _, _ = (t.cpu().numpy() for t in plan.cross_power(d_pm, ref, nb))
    k95_pm = k_at(k, rho_pm, 0.95)
    for n_lpt, (k95, ratio, r1, r2) in out.items():
        print(f"nLPT = {n_lpt}: k(rho=0.95) {k95:.3f} h/Mpc, P/P_ref {ratio:.4f}, rho(1) {r1:.4f}, rho(2) {r2:.4f}")
    print(f"10-step PM: k(rho=0.95) {k95_pm:.3f} h/Mpc")
    k95s = [o[0] for o in out.values()]
    assert max(k95s) <= 1.1 * min(k95s)
    assert min(k95s) >= 1.5 * k95_pm
    base = out[-2.5]
    for k95, ratio, r1, r2 in out.values():
        assert abs(ratio - 1.0) <= 0.02
        assert abs(r1 - base[2]) <= 0.005 and abs(r2 - base[3]) <= 0.01
