"""FP64 CPU oracle for the COLA hot path (Tassev, Zaldarriaga & Eisenstein 2013, arXiv:1301.0322).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its Python
binding) may import, call or link anything in this package; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of ``bench.py`` use it.

The oracle is a plain, slow, obviously correct restatement of the method in float64:

* ``cosmology`` -- background Q(a), growth factors D1/D2 and T[D], T^2[D] (App. A.1, eq. eom;
  App. A.3), the modified kick/drift coefficients (eq. KDKALC) and the standard ones
  (eq. KDKStd / KDKALCstd), the BBKS linear power spectrum normalised to sigma8.
* ``philox`` -- Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the
  Box-Muller white noise built from it.
* ``mesh`` -- cloud-in-cell deposit (float64 and the fixed-point int64 variant), CIC gather,
  the PM force -(3/2) Om a d/dx d^-2 delta of eq. eom on a periodic mesh.
* ``lpt`` -- Zel'dovich and 2LPT displacement fields s1, s2 (App. A.3).
* ``cola`` -- the time evolution of eq. ALCtimestep with the L+- operators of eq. Lops and
  the Kick/Drift operators of eq. KDKALC, applied literally (one operator at a time).
* ``power`` -- shell-averaged power spectrum estimator (Sec. 3.1).

Every function in these modules names the passage it follows and is pinned by
``tests/test_oracle_*.py`` against closed forms, brute force and invariants.
"""
