"""Friends-of-friends (FOF) halo groups and their mass function (Sec. 3.2).

Oracle (test infrastructure only).  Exact integer arithmetic.

Paper passage: Sec. 3.2 (halo statistics): FOF with a fixed linking length 0.2 (in units of
the mean interparticle separation), at least 25 particles per halo; the mass function n(>M).
Readings of this library (the paper runs an external FOF code and gives no more detail):
  * positions are the fixed-point CIC coordinates of the particles (mesh cells x 2^F, the
    same quantised positions the PM force uses; oracle.mesh.fixed_point_coords);
  * two particles are friends iff their periodic minimum-image distance d satisfies
    d < b s, s = (ng / np) 2^F the mean separation in those units; with b = num/den (1/5 in
    the paper) the test is the integer comparison den^2 d^2 < num^2 s^2 (exact, no rounding);
  * groups are the connected components of the friendship graph; a group is labelled by the
    smallest particle index it contains; halos are groups of at least nmin particles;
  * the mass function is reported as the number of halos with at least N_k particles for
    given thresholds N_k (mass = particles x particle mass).
"""
import numpy as np
import scipy.sparse
import scipy.sparse.csgraph


def exact_friends(f, i, j, period, s_fixed, b_num, b_den):
    """Keep the candidate pairs (i, j) that satisfy den^2 |d|^2 < num^2 s^2 (int64)."""
    d2 = np.zeros(i.size, dtype=np.int64)
    for ax in range(3):
        d = f[ax][i] - f[ax][j]
        d = np.mod(d + period // 2, period) - period // 2  # minimum image
        d2 += d * d
    keep = np.int64(b_den) ** 2 * d2 < np.int64(b_num) ** 2 * np.int64(s_fixed) * np.int64(s_fixed)
    return i[keep], j[keep]


def friend_pairs(f, period, s_fixed, b_num=1, b_den=5, chunk=2048, method="auto"):
    """All pairs (i < j) with den^2 |d|^2 < num^2 s^2, f: (3, n) int64.

    method "brute": every pair; "tree": candidates from a periodic k-d tree (scipy) within a
    slightly larger float64 radius (a superset), then the same exact integer test; "auto"
    uses the tree above 4096 particles."""
    f = np.asarray(f, dtype=np.int64)
    n = f.shape[1]
    if method == "tree" or (method == "auto" and n > 4096):
        import scipy.spatial
        tree = scipy.spatial.cKDTree(f.T.astype(np.float64), boxsize=float(period))
        r = float(s_fixed) * b_num / b_den * (1.0 + 1e-9) + 1.0
        cand = tree.query_pairs(r, output_type="ndarray")
        if cand.size == 0:
            return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64)
        i, j = np.minimum(cand[:, 0], cand[:, 1]), np.maximum(cand[:, 0], cand[:, 1])
        return exact_friends(f, i.astype(np.int64), j.astype(np.int64), period, s_fixed, b_num, b_den)
    lim = np.int64(b_num) ** 2 * np.int64(s_fixed) * np.int64(s_fixed)
    den2 = np.int64(b_den) ** 2
    out_i, out_j = [], []
    for a in range(0, n, chunk):
        fa = f[:, a:a + chunk]
        d2 = np.zeros((fa.shape[1], n), dtype=np.int64)
        for ax in range(3):
            d = fa[ax][:, None] - f[ax][None, :]
            d = np.mod(d + period // 2, period) - period // 2  # minimum image
            d2 += d * d
        ii, jj = np.nonzero(den2 * d2 < lim)
        ii = ii + a
        keep = ii < jj
        out_i.append(ii[keep])
        out_j.append(jj[keep])
    return np.concatenate(out_i), np.concatenate(out_j)


def fof_groups(f, period, s_fixed, nmin, b_num=1, b_den=5):
    """Returns (group, size): per particle, the smallest particle index of its FOF group if the
    group has at least nmin particles (else -1), and the size of its group."""
    n = f.shape[1]
    i, j = friend_pairs(f, period, s_fixed, b_num, b_den)
    adj = scipy.sparse.coo_matrix((np.ones(i.size, dtype=np.int8), (i, j)), shape=(n, n))
    _, comp = scipy.sparse.csgraph.connected_components(adj, directed=False)
    first = np.full(comp.max() + 1, n, dtype=np.int64)
    np.minimum.at(first, comp, np.arange(n))
    sizes = np.bincount(comp)
    size = sizes[comp]
    group = np.where(size >= nmin, first[comp], -1)
    return group.astype(np.int64), size.astype(np.int64)


def mass_function(group, size, thresholds):
    """Number of halos with at least N_k particles, for each threshold N_k."""
    roots = np.unique(group[group >= 0])
    hs = size[roots]  # a halo's label is one of its members, so size[label] is its size
    return np.array([int(np.sum(hs >= t)) for t in thresholds], dtype=np.int64)
