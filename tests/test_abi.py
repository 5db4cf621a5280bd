"""CPU-side checks of the C ABI: the library builds and loads, exports every symbol that
include/cola.h declares, validates its arguments, and its host float64 coefficient module
matches the oracle (App. A.3, eq. KDKALC, eq. ALCtimestep).  No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.cosmology import Cosmology, time_grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1301_0322_gb300 import build
    build.build(verbose=False)
    from paper_1301_0322_gb300 import cola
    return cola


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "cola.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(cola_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(lib):
    cdll = lib.load_library()
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(cdll, n), n


def test_binding_names_every_error_code(lib):
    text = open(os.path.join(ROOT, "include", "cola.h")).read()
    codes = {int(v): k for k, v in re.findall(r"#define\s+(COLA_E[A-Z]+)\s+(\d+)\s", text)}
    assert codes and codes == lib.ERRORS
    assert "COLA_ETIMEOUT" in str(lib.ColaError(6, "x"))


def test_header_has_no_torch_types():
    text = open(os.path.join(ROOT, "include", "cola.h")).read()
    assert "torch" not in text.lower().replace("torch-", "")
    assert 'extern "C"' in text


def test_config_validation(lib):
    cfg = lib.cola_config_default()
    assert (cfg.np, cfg.ng, cfg.nsteps, cfg.deconv, cfg.fixed_bits) == (32, 64, 10, 1, 16)
    assert cfg.n_lpt == -2.5 and cfg.a_init == 0.1
    assert (cfg.scheme, cfg.log_a) == (0, 0)
    for field, bad, code in (("ng", 100, 4), ("np", 7, 4), ("nsteps", 0, 1), ("deconv", 3, 1),
                             ("fixed_bits", 30, 1), ("a_init", 2.0, 1), ("box", -1.0, 1), ("scheme", 4, 1),
                             ("log_a", 2, 1)):
        c = lib.cola_config_default()
        setattr(c, field, bad)
        with pytest.raises(lib.ColaError) as e:
            lib.cola_plan_create(c)
        assert e.value.code == code, field


def test_adjoint_needs_the_lpt_frame(lib):
    c = lib.cola_config_default()
    c.scheme, c.adjoint = lib.SCHEMES["pm_std"], 1
    with pytest.raises(lib.ColaError) as e:
        lib.cola_plan_create(c)
    assert e.value.code == 1


def test_calls_without_workspace_are_rejected(lib):
    h = lib.cola_plan_create(lib.cola_config_default())
    try:
        assert lib.cola_workspace_bytes(h) > 0
        cdll = lib.load_library()
        rc = cdll.cola_step(h, 0, None, None, None, None, None)
        assert rc == 5  # COLA_ENOWORKSPACE
        assert b"workspace" in cdll.cola_last_error()
        # every compute call checks for the workspace before it looks at its arguments
        for call, args in (("cola_density_power", (h, None, 8, None, None, None, None)),
                           ("cola_power", (h, None, 8, None, None, None, None)),
                           ("cola_density", (h, None, None, None, None)),
                           ("cola_force", (h, None, None, None))):
            assert getattr(cdll, call)(*args) == 5, call
    finally:
        lib.cola_plan_destroy(h)


@pytest.mark.parametrize("om,ol,n_lpt,nsteps,scheme,log_a", [(0.27, 0.73, -2.5, 10, "cola", 0),
                                                            (1.0, 0.0, -2.5, 3, "cola", 0),
                                                            (0.3, 0.6, 1.5, 5, "cola", 0),
                                                            (0.27, 0.73, -2.5, 10, "cola_std", 0),
                                                            (0.27, 0.73, -2.5, 10, "pm_std", 1),
                                                            (0.27, 0.73, -2.0, 6, "cola_u1", 1),
                                                            (0.27, 0.73, -2.5, 7, "cola", 1)])
def test_host_coefficients_match_oracle(lib, om, ol, n_lpt, nsteps, scheme, log_a):
    cfg = lib.cola_config_default()
    cfg.cosmo.omega_m, cfg.cosmo.omega_l, cfg.n_lpt, cfg.nsteps = om, ol, n_lpt, nsteps
    cfg.scheme, cfg.log_a = lib.SCHEMES[scheme], log_a
    h = lib.cola_plan_create(cfg)
    try:
        tab = lib.cola_coeffs(h, nsteps)
    finally:
        lib.cola_plan_destroy(h)
    cosmo = Cosmology(omega_m=om, omega_l=ol)
    a, mid = time_grid(0.1, 1.0, nsteps, "loga" if log_a else "a")
    modified_kick = scheme in ("cola", "cola_u1")

    def kick(ai, af, ac):
        return cosmo.kick_cola(ai, af, ac, n_lpt) if modified_kick else cosmo.kick_std(ai, af, ac)

    def drift(ai, af, ac):
        return cosmo.drift_cola(ai, af, ac, n_lpt) if scheme == "cola" else cosmo.drift_std(ai, af)
    g = cosmo.growth(a)
    for i in range(nsteps + 1):
        ka = a[0] if i == 0 else mid[i - 1]
        kb = a[-1] if i == nsteps else mid[i]
        row = tab[i]
        assert row[0] == pytest.approx(a[i], rel=1e-15)
        assert row[1] == pytest.approx(1.5 * om * a[i], rel=1e-14)
        # the merged kick K(a_i-1/2, a_i; a_i) K(a_i, a_i+1/2; a_i) of eq. ALCtimestep
        merged = kick(ka, a[i], a[i]) + kick(a[i], kb, a[i])
        assert row[2] == pytest.approx(merged, rel=1e-10)
        assert row[3] == pytest.approx(g["T2D1"][i], rel=1e-9)
        assert row[4] == pytest.approx(g["T2D2"][i], rel=1e-8)
        assert row[8] == pytest.approx(g["TD1"][i], rel=1e-9)
        assert row[9] == pytest.approx(g["TD2"][i], rel=1e-8)
        assert row[10] == pytest.approx(g["D1"][i], rel=1e-9)
        assert row[11] == pytest.approx(g["D2"][i], rel=1e-8)
        if i < nsteps:
            assert row[5] == pytest.approx(drift(a[i], a[i + 1], mid[i]), rel=1e-10)
            assert row[6] == pytest.approx(g["D1"][i + 1] - g["D1"][i], rel=1e-8)
            assert row[7] == pytest.approx(g["D2"][i + 1] - g["D2"][i], rel=1e-7)
        assert row[15] == pytest.approx(g["d2u1"], rel=1e-9)


def test_ensemble_create_validates_and_lays_out_the_boxes(lib):
    def cfg(n_p, ng, nsteps=10):
        c = lib.cola_config_default()
        c.np, c.ng, c.nsteps = n_p, ng, nsteps
        return c

    h = lib.cola_ensemble_create([cfg(32, 64), cfg(48, 96), cfg(64, 256)])
    try:
        assert lib.cola_ensemble_workspace_bytes(h) > 0
        poff, moff = lib.cola_ensemble_offsets(h, 3)
        assert list(poff) == [0, 32**3, 32**3 + 48**3, 32**3 + 48**3 + 64**3]
        assert list(moff) == [0, 64**3, 64**3 + 96**3, 64**3 + 96**3 + 256**3]
        cdll = lib.load_library()
        assert cdll.cola_ensemble_step(h, 0, None, None, None, None, None) == 5  # COLA_ENOWORKSPACE
        t = lib.cola_ensemble_get_tuning(h)
        assert (t.threads, t.tile_shape, t.blocks_per_sm, t.radix, t.launch, t.mesh_streams) == (256, 0, 0, 0, 0, 0)
        assert lib.COLA_ENSEMBLE_TUNE_CANDIDATES == 25
    finally:
        lib.cola_ensemble_destroy(h)
    with pytest.raises(lib.ColaError) as e:
        lib.cola_ensemble_create([cfg(32, 64), cfg(32, 64, nsteps=5)])
    assert e.value.code == 1
    for bad_ng in (48, 384):
        with pytest.raises(lib.ColaError) as e:
            lib.cola_ensemble_create([cfg(32, 64), cfg(32, bad_ng)])
        assert e.value.code == 4 and b"box 1" in lib.load_library().cola_last_error()
    with pytest.raises(lib.ColaError) as e:
        lib.cola_ensemble_create([])
    assert e.value.code == 1


def test_fof_needs_a_workspace(lib):
    h = lib.cola_plan_create(lib.cola_config_default())
    try:
        cdll = lib.load_library()
        assert cdll.cola_fof(h, None, 1, 5, 25, None, None, 0, None, None, None) == 5  # COLA_ENOWORKSPACE
    finally:
        lib.cola_plan_destroy(h)
