"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the method: it only builds charge sets
(positions, the two charge forms qA/qB of each titratable site, the site map
and the lambda vector).  The shapes follow the workloads of arXiv 2410.01626:
water-like solvent with TIP3P-like charges (O -0.834 e, H +0.417 e; the
charge-buffer passage of Sec. 2.5 quotes the -0.834 e oxygen), protein-like
clusters of charged atoms, and titratable sites whose two forms differ only
in their charges (Sec. 2.1) and change the site's net charge by -1
(a titratable site's net charge changes by one unit, Sec. 2.1).

Readings where the workload descriptions are silent:
water H-O-H angle 104.52 deg; water oxygens on a jittered FCC lattice (a
literal random sequential placement at O-O >= 0.28 nm jams at this density);
cluster radius = half the quoted sphere size; sites are compact groups of
nearby cluster atoms; qB = qA + delta with delta ~ U(-0.5, 0.5) shifted so
that every site's net change is exactly -1.

Every system is a dict with keys
  name, x (float32 [N,3], nm), qA, qB (float32 [N], e), site (int32 [N], -1 =
  no site), lam (float32 [K]), L (box edge, nm), origin (3 floats), periodic,
  p, depth (the FMM order and tree depth the workload is run with).
"""
from __future__ import annotations

import math

import numpy as np

O_CHARGE = -0.834
H_CHARGE = 0.417
OH_BOND = 0.09572
HOH_ANGLE_DEG = 104.52
OO_MIN = 0.28


def _site_deltas(rng, n):
    d = rng.uniform(-0.5, 0.5, n)
    return d - d.mean() - 1.0 / n


def _finish(name, x, qA, site_groups, rng, L, periodic, p, depth, origin=(0.0, 0.0, 0.0)):
    n = len(qA)
    site = np.full(n, -1, np.int32)
    qB = qA.astype(np.float64).copy()
    for k, g in enumerate(site_groups):
        g = np.asarray(g)
        site[g] = k
        qB[g] = qA[g] + _site_deltas(rng, len(g))
    lam = rng.uniform(0.0, 1.0, len(site_groups))
    return {
        "name": name,
        "x": np.ascontiguousarray(x, np.float32),
        "qA": np.ascontiguousarray(qA, np.float32),
        "qB": np.ascontiguousarray(qB, np.float32),
        "site": site,
        "lam": np.ascontiguousarray(lam, np.float32),
        "L": float(L),
        "origin": tuple(float(o) for o in origin),
        "periodic": bool(periodic),
        "p": int(p),
        "depth": int(depth),
    }


def open_uniform(seed=0, n=1000, L=4.0, n_sites=10, site_size=4, p=8, depth=2):
    """Point charges +-1 uniform in an open cube; random distinct site atoms."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, L, (n, 3)).astype(np.float32)
    qA = np.concatenate([np.ones(n // 2), -np.ones(n - n // 2)])
    qA = rng.permutation(qA)
    chosen = rng.choice(n, n_sites * site_size, replace=False)
    groups = [chosen[site_size * k: site_size * (k + 1)] for k in range(n_sites)]
    return _finish(f"open_uniform_n{n}", x, qA, groups, rng, L, False, p, depth)


def periodic_uniform(seed=0, n=2000, L=3.0, n_sites=8, site_size=4, p=8, depth=3, neutral=True):
    """Random charges in a periodic cube (small parity cases)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, L, (n, 3)).astype(np.float32)
    qA = rng.normal(0.0, 0.5, n)
    if neutral:
        qA -= qA.mean()
    chosen = rng.choice(n, n_sites * site_size, replace=False)
    groups = [chosen[site_size * k: site_size * (k + 1)] for k in range(n_sites)]
    return _finish(f"periodic_uniform_n{n}", x, qA, groups, rng, L, True, p, depth)


def periodic_dense_cluster(seed=0, n_bg=6000, n_cluster=3000, radius=0.3, center=(1.1, 1.3, 2.2), L=4.0,
                           n_sites=8, site_size=4, p=10, depth=3):
    """A periodic cube of +-1 charges, uniform, plus a dense ball of +-1 charges (about 30 times
    the background density at the defaults): the leaves around the ball hold hundreds of atoms."""
    rng = np.random.default_rng(seed)
    xb = rng.uniform(0.0, L, (n_bg, 3))
    d = rng.normal(size=(n_cluster, 3))
    d *= (radius * rng.uniform(0.0, 1.0, (n_cluster, 1)) ** (1.0 / 3.0)) / np.linalg.norm(d, axis=1, keepdims=True)
    x = np.concatenate([xb, np.asarray(center) + d]).astype(np.float32)
    n = n_bg + n_cluster
    qA = rng.permutation(np.concatenate([np.ones(n // 2), -np.ones(n - n // 2)]))
    chosen = rng.choice(n, n_sites * site_size, replace=False)
    groups = [chosen[site_size * k: site_size * (k + 1)] for k in range(n_sites)]
    return _finish(f"periodic_dense_cluster_n{n}", x, qA, groups, rng, L, True, p, depth)


def _random_rotations(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, a, b, c = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (b * b + c * c)
    R[:, 0, 1] = 2 * (a * b - c * w)
    R[:, 0, 2] = 2 * (a * c + b * w)
    R[:, 1, 0] = 2 * (a * b + c * w)
    R[:, 1, 1] = 1 - 2 * (a * a + c * c)
    R[:, 1, 2] = 2 * (b * c - a * w)
    R[:, 2, 0] = 2 * (a * c - b * w)
    R[:, 2, 1] = 2 * (b * c + a * w)
    R[:, 2, 2] = 1 - 2 * (a * a + b * b)
    return R


def _cluster(rng, n, radius, center, min_dist=0.1):
    pts = np.empty((n, 3))
    k = 0
    while k < n:
        c = rng.uniform(-radius, radius, (4 * (n - k) + 16, 3))
        c = c[(c * c).sum(1) <= radius * radius]
        for v in c:
            if k == n:
                break
            if k and np.min(((pts[:k] - v) ** 2).sum(1)) < min_dist * min_dist:
                continue
            pts[k] = v
            k += 1
    return pts + np.asarray(center)


def _compact_sites(rng, pts, n_sites, site_size, seed_sep=0.5):
    """Seeds at least seed_sep apart (relaxed step by step when the cluster is too small to
    hold that many), each with its nearest unused cluster atoms."""
    order = rng.permutation(len(pts))
    for sep in (seed_sep, 0.35, 0.25, 0.0):
        seeds = []
        for i in order:
            if all(np.sum((pts[i] - pts[j]) ** 2) >= sep ** 2 for j in seeds):
                seeds.append(i)
                if len(seeds) == n_sites:
                    break
        if len(seeds) == n_sites:
            break
    if len(seeds) < n_sites or n_sites * site_size > len(pts):
        raise ValueError("cluster too small for the requested number of sites")
    used = np.zeros(len(pts), bool)
    used[seeds] = True
    groups = []
    for s in seeds:
        d = ((pts - pts[s]) ** 2).sum(1)
        d[used] = np.inf
        near = np.argsort(d, kind="stable")[: site_size - 1]
        used[near] = True
        groups.append(np.concatenate([[s], near]))
    return groups


def _water_oxygens(rng, L, n_w, n_cell, exclude):
    a = L / n_cell
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) + 0.25
    g = np.stack(np.meshgrid(*[np.arange(n_cell)] * 3, indexing="ij"), -1).reshape(-1, 1, 3)
    sites = ((g + base[None]) * a).reshape(-1, 3)
    keep = np.ones(len(sites), bool)
    for c, r in exclude:
        d = sites - np.asarray(c)
        d -= L * np.round(d / L)
        keep &= (d * d).sum(1) > r * r
    sites = sites[keep]
    if len(sites) < n_w:
        raise ValueError("not enough lattice sites for the requested waters")
    pick = np.sort(rng.choice(len(sites), n_w, replace=False))
    return sites[pick] + rng.uniform(-0.01, 0.01, (n_w, 3))


def water_cluster(seed, L, n_waters, clusters, sites_per_cluster, site_size=5, n_cell=None,
                  p=8, depth=4, name="water_cluster"):
    """Periodic box of rigid 3-site waters plus protein-like charged clusters.

    clusters: list of (center (3,), n_atoms, radius).  Returns a system dict.
    """
    rng = np.random.default_rng(seed)
    if n_cell is None:
        n_cell = int(math.ceil((1.25 * n_waters / 4.0) ** (1.0 / 3.0)))
    cl_pts, cl_q, groups, off = [], [], [], 0
    for (c, nat, rad), ns in zip(clusters, sites_per_cluster):
        pts = _cluster(rng, nat, rad, c)
        q = rng.normal(0.0, 0.3, nat)
        q -= q.mean()
        for g in _compact_sites(rng, pts, ns, site_size):
            groups.append(g + off)
        cl_pts.append(pts)
        cl_q.append(q)
        off += nat
    exclude = [(c, rad + OO_MIN) for (c, nat, rad) in clusters]
    O = _water_oxygens(rng, L, n_waters, n_cell, exclude)
    R = _random_rotations(rng, n_waters)
    half = math.radians(HOH_ANGLE_DEG) / 2.0
    h1 = OH_BOND * np.array([math.sin(half), 0.0, math.cos(half)])
    h2 = OH_BOND * np.array([-math.sin(half), 0.0, math.cos(half)])
    H1 = O + R @ h1
    H2 = O + R @ h2
    wat = np.stack([O, H1, H2], 1).reshape(-1, 3)
    wq = np.tile([O_CHARGE, H_CHARGE, H_CHARGE], n_waters)
    x = np.concatenate(cl_pts + [wat]) if cl_pts else wat
    qA = np.concatenate(cl_q + [wq]) if cl_q else wq
    x = np.mod(x, L)
    out = _finish(name, x, qA, groups, rng, L, True, p, depth)
    out["n_solute"] = off  # cluster atoms come first, then the waters as (O, H, H)
    return out


def oxygen_min_distance(sys_):
    """Smallest O-O distance (minimum image) of a water_cluster system."""
    from scipy.spatial import cKDTree
    q = sys_["qA"]
    O = sys_["x"][np.isclose(q, O_CHARGE) & (sys_["site"] < 0)].astype(np.float64)
    L = sys_["L"]
    t = cKDTree(np.mod(O, L), boxsize=L)
    d, _ = t.query(np.mod(O, L), k=2)
    return float(d[:, 1].min())


BUFFER_QA = -0.834  # a water oxygen ...
BUFFER_QB = 0.166   # ... whose charge changes by +1 (Sec. 2.5, charge buffers)


def charge_buffers(s, distance=3.0, exclusion=2.0):
    """The charge-buffer variant of a water_cluster system (Sec. 2.5): every site k is paired
    with one water oxygen that joins the site and changes from -0.834 e (qA) to +0.166 e (qB)
    with lambda_k, so that the pair's net charge, and the box's, does not depend on lambda.
    The buffer of site k is the not yet used oxygen whose distance from the site's centroid is
    nearest to `distance` (3 nm), among the oxygens at least `exclusion` (2 nm) from every
    cluster atom (minimum image).  Returns a new system dict (name + "_buf")."""
    from scipy.spatial import cKDTree
    L = s["L"]
    ns = s["n_solute"]
    x = s["x"].astype(np.float64)
    ox = np.arange(ns, len(x), 3)  # the water oxygens
    assert np.allclose(s["qA"][ox], O_CHARGE)
    tree = cKDTree(np.mod(x[:ns], L), boxsize=L)
    dmin, _ = tree.query(np.mod(x[ox], L), k=1)
    cand = ox[dmin >= exclusion]
    site = s["site"].copy()
    qB = s["qB"].copy()
    used = np.zeros(len(cand), bool)
    for k in range(len(s["lam"])):
        g = np.nonzero(site == k)[0]
        ref = x[g[0]]
        d = x[g] - ref
        d -= L * np.round(d / L)
        c = ref + d.mean(0)
        r = x[cand] - c
        r -= L * np.round(r / L)
        dist = np.sqrt((r * r).sum(1))
        score = np.abs(dist - distance)
        score[used] = np.inf
        j = int(np.argmin(score))
        used[j] = True
        site[cand[j]] = k
        qB[cand[j]] = BUFFER_QB
    t = dict(s)
    t["site"] = site
    t["qB"] = np.ascontiguousarray(qB, np.float32)
    t["name"] = s["name"] + "_buf"
    return t


# ---- the workloads ----

def small_open(seed=0):
    """1000 charges +-1 in an open 4 nm cube, 10 sites x 4 atoms, p=8, depth 2."""
    return open_uniform(seed=seed, n=1000, L=4.0, n_sites=10, site_size=4, p=8, depth=2)


def solvated_30k(seed=1, p=8):
    """6.5 nm periodic box: 9000 waters + 2000-atom cluster (20 sites x 5); p=8, depth 4."""
    L = 6.5
    return water_cluster(seed, L, 9000, [((L / 2,) * 3, 2000, 1.5)], [20], n_cell=14, p=p,
                         depth=4, name="solvated_30k")


def solvated_30k_buf(seed=1, p=8):
    """The 30k system with one charge buffer per site (Sec. 2.5): neutral at every lambda."""
    return charge_buffers(solvated_30k(seed, p))


def solvated_500k(seed=5, p=10):
    """17 nm periodic box: 160000 waters + 4 clusters x 5000 atoms (200 sites x 5); p=10, depth 5."""
    L = 17.0
    cs = [(0.25, 0.25, 0.25), (0.75, 0.75, 0.25), (0.75, 0.25, 0.75), (0.25, 0.75, 0.75)]
    clusters = [(tuple(L * np.asarray(c)), 5000, 2.04) for c in cs]
    return water_cluster(seed, L, 160000, clusters, [50] * 4, n_cell=36, p=p, depth=5,
                         name="solvated_500k")


def replica(seed, p=8):
    """One replica of the batched workload: N log-uniform in [5k, 50k] at 100 atoms/nm^3."""
    rng = np.random.default_rng(seed)
    N = int(round(math.exp(rng.uniform(math.log(5e3), math.log(5e4)))))
    L = (N / 100.0) ** (1.0 / 3.0)
    nc = int(round(N * 2000 / 29000))
    nw = (N - nc) // 3
    nc = N - 3 * nw
    rad = 1.5 * (nc / 2000.0) ** (1.0 / 3.0)
    K = int(rng.integers(5, 41))
    K = min(K, nc // 5)
    depth = int(min(5, max(2, round(math.log(N / 16.0, 8)))))
    s = water_cluster(seed + 100000, L, nw, [((L / 2,) * 3, nc, rad)], [K], p=p, depth=depth,
                      name=f"replica_{seed}")
    return s


def replicas(n=64, first_seed=100, p=8):
    return [replica(first_seed + i, p=p) for i in range(n)]


def tautomer_sites(s, seed=0, tautomer_fraction=0.5):
    """Four charge forms per site (Sec. 2.1, Eq. 2): A and B are the two protonated
    tautomers, C = D the deprotonated form.  B redistributes A's charges within the site
    (shift U(-0.3, 0.3), mean removed per site, so A and B carry the same net charge);
    sites without a tautomer have B = A.  lam becomes [2K] = (lambda_p, lambda_t) per site,
    both U(0, 1).  Returns a new system dict with keys qA, qB, qC, qD and forms = 4."""
    rng = np.random.default_rng(seed)
    t = dict(s)
    site = s["site"]
    K = len(s["lam"])
    qA = s["qA"].astype(np.float64)
    qB = qA.copy()
    has_t = rng.uniform(size=K) < tautomer_fraction
    for k in range(K):
        g = np.nonzero(site == k)[0]
        if has_t[k] and len(g):
            d = rng.uniform(-0.3, 0.3, len(g))
            qB[g] = qA[g] + d - d.mean()
    t["qA"] = s["qA"].copy()
    t["qB"] = np.ascontiguousarray(qB, np.float32)
    t["qC"] = s["qB"].copy()
    t["qD"] = s["qB"].copy()
    t["lam"] = np.ascontiguousarray(rng.uniform(0.0, 1.0, 2 * K), np.float32)
    t["forms"] = 4
    t["name"] = s["name"] + "_tautomers"
    return t
