"""Seeded synthetic inputs (geometry, materials, loads, unknown vectors).

This module holds none of the method's arithmetic: it only draws fracture
geometries and vectors from fixed seeds, with the shapes, sizes and
distributions of the workloads the paper studies (a single pressurised crack,
randomly distributed pressurised fractures, parallel hydraulic fractures from
a horizontal well, batches of uneven fracture sets).  The paper's own
geometries are not published, so these stand in for them.

Geometry arrays are (4, N) float64: rows x0, y0, x1, y1 (element end points);
elements of one fracture are consecutive and run from one tip to the other.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 1812

# Rock of the synthetic workloads: G = 6 GPa, nu = 0.2, nu_u = 0.33, B = 0.8,
# k = 1e-18 m^2, mu = 1e-3 Pa s.
MATERIAL = {"G": 6e9, "nu": 0.2, "nu_u": 0.33, "B": 0.8, "perm": 1e-18, "visc": 1e-3}
# Westerly granite as printed in the paper's Table 1 (c follows from k/mu).
WESTERLY = {"G": 15e9, "nu": 0.25, "nu_u": 0.331, "B": 0.81, "perm": 4e-19, "visc": 1e-3}


def material_tuple(m=MATERIAL):
    return tuple(float(m[k]) for k in ("G", "nu", "nu_u", "B", "perm", "visc"))


def discretise(p0, p1, n):
    """n equal constant elements from p0 to p1 -> (4, n)."""
    s = np.linspace(0.0, 1.0, n + 1)
    x = p0[0] + s * (p1[0] - p0[0])
    y = p0[1] + s * (p1[1] - p0[1])
    return np.stack([x[:-1], y[:-1], x[1:], y[1:]])


def single_crack(n=200, a=1.0, angle=0.0, center=(0.0, 0.0)):
    """Straight crack of half-length a, n uniform elements."""
    c, s = math.cos(angle), math.sin(angle)
    p0 = (center[0] - a * c, center[1] - a * s)
    p1 = (center[0] + a * c, center[1] + a * s)
    return discretise(p0, p1, n)


def _seg_dist(a0, a1, b0, b1):
    """Minimum distance between segments (0 if they intersect)."""
    def orient(p, q, r):
        return (q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0])

    o1, o2 = orient(a0, a1, b0), orient(a0, a1, b1)
    o3, o4 = orient(b0, b1, a0), orient(b0, b1, a1)
    if o1 * o2 < 0 and o3 * o4 < 0:
        return 0.0

    def pt_seg(p, s0, s1):
        d = (s1[0] - s0[0], s1[1] - s0[1])
        L2 = d[0] * d[0] + d[1] * d[1]
        t = 0.0 if L2 == 0 else max(0.0, min(1.0, ((p[0] - s0[0]) * d[0] + (p[1] - s0[1]) * d[1]) / L2))
        return math.hypot(p[0] - s0[0] - t * d[0], p[1] - s0[1] - t * d[1])

    return min(pt_seg(a0, b0, b1), pt_seg(a1, b0, b1), pt_seg(b0, a0, a1), pt_seg(b1, a0, a1))


def random_fracture_segments(n_frac=200, box=200.0, lmin=2.0, lmax=10.0, elems=100, seed=SEED,
                             max_tries=200000):
    """Rejection-sampled non-intersecting cracks in a box x box square:
    centre uniform (whole segment inside), length U[lmin, lmax], angle
    U[0, pi); a candidate is rejected if it intersects an accepted crack or
    lies closer to it than one element length of either.  Returns a list of
    (p0, p1, n_elems).  Accepted cracks are bucketed on a grid of cell side
    >= lmax so that a candidate is tested only against cracks near it (the
    same draws and the same accept/reject decisions as testing all)."""
    rng = np.random.default_rng(seed)
    segs = []
    cell = max(lmax, 1e-12)
    margin = lmax / elems                     # the largest separation a rejection can need
    grid = {}

    def cells(x0, y0, x1, y1):
        for i in range(int(math.floor(x0 / cell)), int(math.floor(x1 / cell)) + 1):
            for j in range(int(math.floor(y0 / cell)), int(math.floor(y1 / cell)) + 1):
                yield (i, j)

    tries = 0
    while len(segs) < n_frac:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_fracture_segments: could not place all fractures")
        L = rng.uniform(lmin, lmax)
        th = rng.uniform(0.0, math.pi)
        hx, hy = 0.5 * L * math.cos(th), 0.5 * L * math.sin(th)
        cx = rng.uniform(abs(hx), box - abs(hx))
        cy = rng.uniform(abs(hy), box - abs(hy))
        p0, p1 = (cx - hx, cy - hy), (cx + hx, cy + hy)
        ok = True
        seen = set()
        for c in cells(min(p0[0], p1[0]), min(p0[1], p1[1]), max(p0[0], p1[0]), max(p0[1], p1[1])):
            for k in grid.get(c, ()):
                if k in seen:
                    continue
                seen.add(k)
                q0, q1, _ = segs[k]
                sep = max(L, math.hypot(q1[0] - q0[0], q1[1] - q0[1])) / elems
                if _seg_dist(p0, p1, q0, q1) < sep:
                    ok = False
                    break
            if not ok:
                break
        if ok:
            k = len(segs)
            segs.append((p0, p1, elems))
            for c in cells(min(p0[0], p1[0]) - margin, min(p0[1], p1[1]) - margin,
                           max(p0[0], p1[0]) + margin, max(p0[1], p1[1]) + margin):
                grid.setdefault(c, []).append(k)
    return segs


def assemble(segs):
    return np.concatenate([discretise(p0, p1, n) for (p0, p1, n) in segs], axis=1)


def tips_of(segs):
    """Indices of the first and last element of every fracture."""
    out, k = [], 0
    for (_, _, n) in segs:
        out += [k, k + n - 1]
        k += n
    return np.array(out, dtype=np.int64)


def random_fractures(n_frac=200, box=200.0, elems=100, seed=SEED):
    segs = random_fracture_segments(n_frac, box, 2.0, 10.0, elems, seed)
    return assemble(segs), segs


def clustered_fracture_segments(n_clusters=4, per_cluster=100, cluster_box=12.0, elems_small=20,
                                n_sparse=20, box=400.0, elems_sparse=100, seed=SEED + 6):
    """Strongly clustered fracture set: n_clusters swarms of per_cluster
    small cracks (lengths U[0.4, 1.5] m, elems_small elements each) packed
    in cluster_box x cluster_box squares, plus n_sparse long cracks
    (U[10, 40] m, elems_sparse elements) spread over a box x box domain.
    The swarm centres are drawn uniformly and rejected within 1.5
    cluster_box of a long crack or of another swarm, so no crack crosses
    another.  Element sizes span 0.02 to 0.4 m and the densities differ by
    orders of magnitude across the domain.  Returns (p0, p1, n_elems)
    segments."""
    rng = np.random.default_rng(seed)
    segs = random_fracture_segments(n_sparse, box, 10.0, 40.0, elems_sparse, seed=seed + 1)

    def point_seg(px, py, a, b):
        ax, ay = a
        bx, by = b
        dx, dy = bx - ax, by - ay
        t = max(0.0, min(1.0, ((px - ax) * dx + (py - ay) * dy) / (dx * dx + dy * dy)))
        return math.hypot(px - ax - t * dx, py - ay - t * dy)

    centres = []
    tries = 0
    while len(centres) < n_clusters:
        tries += 1
        if tries > 100000:
            raise RuntimeError("clustered_fracture_segments: could not place the swarms")
        cx, cy = rng.uniform(cluster_box, box - cluster_box, size=2)
        if any(point_seg(cx, cy, p0, p1) < 1.5 * cluster_box for (p0, p1, _) in segs[:n_sparse]):
            continue
        if any(math.hypot(cx - qx, cy - qy) < 3.0 * cluster_box for (qx, qy) in centres):
            continue
        centres.append((cx, cy))
    for k, (cx, cy) in enumerate(centres):
        local = random_fracture_segments(per_cluster, cluster_box, 0.4, 1.5, elems_small, seed=seed + 2 + k)
        ox, oy = cx - 0.5 * cluster_box, cy - 0.5 * cluster_box
        segs += [((p0[0] + ox, p0[1] + oy), (p1[0] + ox, p1[1] + oy), n) for (p0, p1, n) in local]
    return segs


def clustered_fractures(**kw):
    segs = clustered_fracture_segments(**kw)
    return assemble(segs), segs


def parallel_fractures(n_frac=10, spacing=20.0, half_length=100.0, elems=2000):
    """Transverse fractures of a horizontal well along y: fracture k lies on
    y = k * spacing, x in [-half_length, half_length]."""
    segs = [((-half_length, k * spacing), (half_length, k * spacing), elems) for k in range(n_frac)]
    return assemble(segs), segs


# Horizontal-well example (paper Sec. 5, Table 2): in-situ stresses and
# initial pore pressure; a constant injection of 0.01 m^3/s per fracture,
# carried by the plane-strain model per unit thickness over a fracture
# height of 100 m and split uniformly along the fracture; time steps of 60 s.
WELL_LOADS = {"sigma_H": 58.60e6, "sigma_h": 55.15e6, "p0": 48.26e6}
WELL_INJECTION = 0.01     # m^3/s per fracture
WELL_HEIGHT = 100.0       # m
WELL_DT = 60.0


def well_source(half_length=100.0, injection=WELL_INJECTION, height=WELL_HEIGHT):
    """Fluid source per unit element length (m^2/s per m) of a fracture of
    the given half-length carrying `injection` over `height`, split
    uniformly."""
    return injection / (height * 2.0 * half_length)


def batch_problems(n_problems=512, nmin=100, nmax=20000, seed=SEED + 4):
    """Uneven fracture sets: N log-uniform in [nmin, nmax], fracture count
    U{1..100} capped at N/10, box side scaled with sqrt(N / 20000) * 200 m so
    the element density stays comparable; 1-10 time steps each."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_problems):
        N = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        nf = int(min(rng.integers(1, 101), max(1, N // 10)))
        per = max(10, N // nf)
        box = 200.0 * math.sqrt(N / 20000.0) + 12.0
        segs = random_fracture_segments(nf, box, 2.0, min(10.0, box / 2), per, seed=int(rng.integers(1 << 30)))
        out.append({"xy": assemble(segs), "segs": segs, "steps": int(rng.integers(1, 11))})
    return out


def serving_trace(duration=60.0, rate=50.0, nmin=1000, nmax=200000, seed=SEED + 5):
    """Poisson arrivals with N log-uniform in [nmin, nmax] and 1-100 steps."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        N = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        out.append({"t": t, "N": N, "steps": int(rng.integers(1, 101)), "seed": int(rng.integers(1 << 30))})
    return out


def serving_geometry(n_target, seed):
    """Fracture set of one serving request: about n_target elements as
    n_target / 100 random fractures of 100 elements (lengths U[2, 10] m, the
    element size of the 20,000-element set) in a box whose side grows with
    sqrt(n_target), so the fracture density stays that of the 20,000-element
    set at every size."""
    nf = max(1, n_target // 100)
    box = 200.0 * (n_target / 20000.0) ** 0.5 + 12.0
    return assemble(random_fracture_segments(nf, box, 2.0, min(10.0, box / 2), 100, seed=seed))


def unknowns(n, seed=SEED, dd_scale=1e-4, q_scale=1e-9):
    """Random unknown vector [Ds, Dn, Dq] with physical magnitudes."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(3 * n)
    x[:2 * n] *= dd_scale
    x[2 * n:] *= q_scale
    return x
