"""Time evolution of the COLA method, applied literally one operator at a time.

Oracle (test infrastructure only).  Float64.

Paper passages (arXiv:1301.0322, App. A):
  * eq. ALCtimestep: L+(a_{n+1}) prod_i K(a_{i+1/2}, a_{i+1}; a_{i+1}) D(a_i, a_{i+1}; a_{i+1/2})
    K(a_i, a_{i+1/2}; a_i) L-(a_0), applied right to left to (x(a_0), v(a_0) = T[s](a_0));
  * eq. Lops: L+-: v -> v +- (T[D1] s1 + T[D2] s2);
  * eq. KDKALC (the "optimal COLA variant", Sec. 3):
        D: x += v(a_c)/u(a_c) int_{ai}^{af} u/Q da + (D1(af)-D1(ai)) s1 + (D2(af)-D2(ai)) s2
        K: v += (u(af)-u(ai))/T[u](a_c) * (-(3/2) Om a_c d d^-2 delta - T^2[D1] s1 - T^2[D2] s2)
    with u = a^nLPT, nLPT = -2.5 (App. A.3.2) and steps uniform in a;
  * eq. KDKALCstd (scheme "cola_std"): the standard coefficients int da/Q and
    int (a/a_c)/Q da; the leading minus sign printed in its Kick is read as a plus (with it,
    setting s1 = s2 = 0 would not give back eq. KDKStd, as the paper says it does);
  * eq. KDKStd (scheme "pm_std"): the standard leapfrog, no LPT frame, no L+-.
  * scheme "cola_u1": eq. KDKALC with u = 1 in the Drift and u = a^nLPT in the Kick (the
    variant of the footnote on the ansatz u = A + B a^nLPT, App. A.3.2).
  * time grid (cfg.spacing): uniform in a ("a", App. A.3.2) or in ln a ("loga", App. A.2).
  * 2LPT initial conditions: x = q + D1(a0) s1 + D2(a0) s2, v = T[D1](a0) s1 + T[D2](a0) s2.

State: the displacement s with x = q + s (eq. eom), positions taken modulo L for the mesh.
"""
from dataclasses import dataclass, field

import numpy as np

from .cosmology import Cosmology, time_grid
from .lpt import ic_2lpt
from .mesh import lattice_q, unit_force_particles


@dataclass
class ColaConfig:
    n_p: int = 32
    n_g: int = 64
    box: float = 100.0
    cosmo: Cosmology = field(default_factory=Cosmology)
    n_lpt: float = -2.5
    nsteps: int = 10
    a_init: float = 0.1
    a_final: float = 1.0
    deconv: int = 1
    spacing: str = "a"
    fixed_bits: int = 0  # > 0: the force sees positions quantised to 2^-fixed_bits mesh cell


def quantise_positions(pos, n_g, box, fbits):
    """Positions rounded down to a multiple of 2^-fbits mesh cell (float64), periodic."""
    scale = 2.0**fbits
    u = np.floor(pos * (n_g / box) * scale) / scale
    return np.mod(u, n_g) * (box / n_g)


def acceleration(s, cfg, a):
    """-(3/2) Om a d d^-2 delta at the particles (eq. eom), from the PM mesh of the config.

    With cfg.fixed_bits = F > 0 the deposit and the gather see every position rounded down to a
    multiple of 2^-F mesh cell (in float64), the quantisation the library's fixed-point CIC
    applies; comparing against that run isolates the float32 rounding of the GPU path."""
    pos = np.mod(lattice_q(cfg.n_p, cfg.box) + s, cfg.box)
    if cfg.fixed_bits > 0:
        pos = quantise_positions(pos, cfg.n_g, cfg.box, cfg.fixed_bits)
    g = unit_force_particles(pos, cfg.n_p**3, cfg.n_g, cfg.box, cfg.deconv)
    return 1.5 * cfg.cosmo.omega_m * a * g


def evolve(s1, s2, cfg, scheme="cola", stop_after=None, offset=0.0, accel_fn=None, record=None):
    """Evolve from the 2LPT initial conditions at a_init to a_final.

    Returns dict with s (displacement), v (velocity T[s] in the lab frame after L+ for the COLA
    schemes), and the time grid.  ``stop_after`` = number of full K-D-K steps to apply (for
    partial-run parity checks); the final L+ is applied either way for the COLA schemes.
    ``offset`` translates every initial position by the same vector (a symmetry of the
    periodic problem; the tests use it to move lattice particles off the mesh nodes).
    ``accel_fn(s, a)`` replaces the PM acceleration (the tests use the exact 2LPT force to
    check the Kick/Drift/L+- operators on their own).  If ``record`` is a list, the
    displacement of every force evaluation is appended to it (checkpoints for the adjoint)."""
    if accel_fn is None:
        accel_fn = lambda s_, a_: acceleration(s_, cfg, a_)
    cosmo = cfg.cosmo
    a, mid = time_grid(cfg.a_init, cfg.a_final, cfg.nsteps, cfg.spacing)
    g = cosmo.growth(a)
    D1, D2, TD1, TD2, T2D1, T2D2 = (g[k] for k in ("D1", "D2", "TD1", "TD2", "T2D1", "T2D2"))
    if scheme not in ("cola", "cola_std", "pm_std", "cola_u1"):
        raise ValueError(f"unknown scheme {scheme!r}")
    lpt = scheme in ("cola", "cola_std", "cola_u1")
    if not lpt:
        zero = np.zeros_like(s1)
        s1_frame, s2_frame = zero, zero
    else:
        s1_frame, s2_frame = s1, s2

    # 2LPT initial conditions at a_0 (position and velocity T[s] of the 2LPT trajectory)
    s = D1[0] * s1 + D2[0] * s2 + offset
    v = TD1[0] * s1 + TD2[0] * s2
    if lpt:
        v = v - (TD1[0] * s1_frame + TD2[0] * s2_frame)  # L-(a_0), eq. Lops

    def kick(v, ai, af, ic, accel):
        ac = a[ic]
        if scheme in ("cola", "cola_u1"):
            coef = cosmo.kick_cola(ai, af, ac, cfg.n_lpt)
        elif scheme == "cola_std":
            coef = cosmo.kick_std(ai, af, ac)
        else:  # eq. KDKStd: v += (3/2) Om g int a/Q da  ==  int (a/ac)/Q da * (3/2) Om ac g
            coef = cosmo.kick_std(ai, af, ac)
        return v + coef * (accel - T2D1[ic] * s1_frame - T2D2[ic] * s2_frame)

    def drift(s, v, i):
        ai, af, ac = a[i], a[i + 1], mid[i]
        if scheme == "cola":
            coef = cosmo.drift_cola(ai, af, ac, cfg.n_lpt)
        else:
            coef = cosmo.drift_std(ai, af)
        return s + coef * v + (D1[i + 1] - D1[i]) * s1_frame + (D2[i + 1] - D2[i]) * s2_frame

    nrun = cfg.nsteps if stop_after is None else stop_after
    if record is not None:
        record.append(s.copy())
    accel = accel_fn(s, a[0])
    for i in range(nrun):
        v = kick(v, a[i], mid[i], i, accel)              # K(a_i, a_{i+1/2}; a_i)
        s = drift(s, v, i)                                # D(a_i, a_{i+1}; a_{i+1/2})
        if record is not None:
            record.append(s.copy())
        accel = accel_fn(s, a[i + 1])                     # force at the new positions
        v = kick(v, mid[i], a[i + 1], i + 1, accel)       # K(a_{i+1/2}, a_{i+1}; a_{i+1})
    if lpt:
        v = v + TD1[nrun] * s1_frame + TD2[nrun] * s2_frame  # L+(a_{n+1}), eq. Lops
    return {"s": s, "v": v, "a": a, "mid": mid}


def run(noise, cfg, scheme="cola"):
    """Full run from white noise (n_p^3 lattice): 2LPT ICs, then ``evolve``."""
    s1, s2 = ic_2lpt(np.asarray(noise, dtype=np.float64), cfg.box, cfg.cosmo)
    out = evolve(s1, s2, cfg, scheme)
    out["s1"], out["s2"] = s1, s2
    return out
