"""Seeded synthetic inputs shared by the tests and the benchmark (no COLA arithmetic here).

The paper's workload is a periodic box of particles on a Lagrangian lattice evolved from
Gaussian initial conditions (Sec. 2); the benchmark configurations below follow the sizes of
that workload and of its batched / differentiable / large variants.  White noise here comes
from numpy's PCG64 so that tests can hand the same float32 array to the CUDA path and to the
oracle; the library's own Philox generator (cola_noise) is tested separately.
"""
import numpy as np

# name -> (np, ng, box [Mpc/h], Philox seed)
WORKLOADS = {
    "cola_32p_64g_L100": (32, 64, 100.0, 1),
    "cola_256p_768g_L100": (256, 768, 100.0, 2),
    "cola_128p_384g_L50": (128, 384, 50.0, 2),  # 1/8 sub-volume of the above (profiling captures)
    "cola_128p_256g_L200": (128, 256, 200.0, 7),
    "cola_1024p_2048g_L1000": (1024, 2048, 1000.0, 3),
}
COSMOLOGY = dict(omega_m=0.27, omega_l=0.73, h=0.7, sigma8=0.8, n_s=0.96)

# the mock ensemble: 48 independent boxes of three sizes, all with 0.78 Mpc/h mesh cells;
# (np, ng, box [Mpc/h]) per box in order, Philox seeds 100..147
ENSEMBLE_48 = [(64, 128, 100.0)] * 16 + [(96, 192, 150.0)] * 16 + [(128, 256, 200.0)] * 16
ENSEMBLE_48_SEEDS = list(range(100, 148))


def gaussian_noise(n, seed):
    """Unit-variance white noise on the n^3 lattice, float32, shape (n^3,) in [iz][iy][ix] order."""
    return np.random.default_rng(seed).standard_normal(n**3).astype(np.float32)


def gaussian_displacements(n, sigma, seed):
    """Independent Gaussian displacements (3, n^3) float32 with standard deviation sigma."""
    return (np.random.default_rng(seed).standard_normal((3, n**3)) * sigma).astype(np.float32)


def clustered_displacements(n, box, seed, nclump=8, frac=0.5, radius=0.5):
    """Displacements that pull a fraction of the lattice into a few tight clumps (dense cells),
    float32 (3, n^3); the rest get small random offsets."""
    rng = np.random.default_rng(seed)
    p = np.arange(n**3)
    q = np.stack([p % n, (p // n) % n, p // (n * n)]).astype(np.float64) * (box / n)
    centres = rng.uniform(0, box, size=(nclump, 3))
    target = centres[rng.integers(0, nclump, size=n**3)].T + rng.normal(0, radius, size=(3, n**3))
    pick = rng.uniform(size=n**3) < frac
    disp = np.where(pick, target - q, rng.normal(0, 0.3 * box / n, size=(3, n**3)))
    disp = (disp + 0.5 * box) % box - 0.5 * box  # shortest periodic displacement
    return disp.astype(np.float32)
