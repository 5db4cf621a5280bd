"""The oracle against the few values the paper prints (tests/golden/paper_values.json)."""
import json
import math
import os

import numpy as np
import pytest

from oracle.cola import ColaConfig
from oracle.cosmology import Cosmology

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_oracle_defaults_are_the_papers_setup():
    cfg = ColaConfig()
    assert cfg.n_lpt == GOLD["n_lpt"]["value"]
    assert cfg.a_init == pytest.approx(1.0 / (1.0 + GOLD["z_initial"]["value"]))
    assert cfg.nsteps == GOLD["timesteps"]["value"]


def test_mode_powers_map_to_the_nlpt_range():
    # s_res ~ a^p has v_res = T[s_res] ~ a^(p + 1/2) in matter domination, i.e. nLPT = p + 1/2;
    # the printed mode powers must span the printed nLPT interval.
    eds = Cosmology(omega_m=1.0, omega_l=0.0)
    a = np.array([0.2, 0.4])
    n_lpt = []
    for p in GOLD["third_order_mode_powers"]["value"]:
        t = eds.Q(a) * p * a ** (p - 1.0)  # T[a^p]
        slope = math.log(t[1] / t[0]) / math.log(a[1] / a[0])
        n_lpt.append(slope)
    assert min(n_lpt) == pytest.approx(GOLD["n_lpt_range"]["value"][0])
    assert max(n_lpt) == pytest.approx(GOLD["n_lpt_range"]["value"][1])
    lo, hi = GOLD["n_lpt_range"]["value"]
    assert lo < GOLD["n_lpt"]["value"] < hi


def test_halo_radius_ratio_and_nmax_coefficient():
    g = GOLD["halo_radius_ratio"]
    ratio = (4 * math.pi * g["delta"] / (3 * g["N"])) ** (-1.0 / 3.0)
    assert ratio == pytest.approx(g["value"], abs=0.01)
    c = GOLD["n_max_coefficient"]
    rho2 = 1.0 - c["P_eps_over_P_NL"]  # rho^2 = R^2 P_M / P_NL = 1 - P_eps / P_NL
    assert c["value"] * math.sqrt(rho2 / (1.0 - rho2)) == pytest.approx(c["n_max"])
