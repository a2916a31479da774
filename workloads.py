"""Seeded synthetic inputs shared by the tests, the oracle runs and bench.py.

This module holds only input generation (random coefficients, patch-centre
layouts, wire layouts, target points).  It contains none of the method's
arithmetic: no Green's functions, no walks, no quadrature, no solves.  Both the
CUDA path and the oracle consume what it returns.

All host-side randomness uses NumPy's PCG64 with an explicit seed.  The random
numbers of the walks themselves are not drawn here: both sides generate them
from the counter-based Philox4x32-10 definition (key = walk seed).

Workload shapes follow the five configurations of the method's GPU study
(unit-cube single patch, unit-ball full boundary, 200-wire box layout, scaled
unit ball, serving).  The paper itself uses a planar interface (Sec. 5.1) and a
sphere of radius 3 (Sec. 5.2); the shapes below keep its parameters where they
are given (hemisphere Gauss products, patch radius, epsilon-shell).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# geometry kinds (same numeric values as the C ABI enum)
GEOM_BALL_INTERIOR = 0
GEOM_BOX_INTERIOR = 1
GEOM_BOX_MINUS_BOXES = 2
GEOM_HALF_SPACE = 3
GEOM_DISK_EXTERIOR = 4
GEOM_BALL_EXTERIOR = 5

# Dirichlet data kinds
DATA_POINT_SOURCE = 0
DATA_HARMONIC_SH = 1
DATA_CONSTANT = 2


@dataclasses.dataclass
class Geometry:
    kind: int
    center: tuple = (0.0, 0.0, 0.0)
    radius: float = 1.0
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    boxes: np.ndarray | None = None  # (n, 6) float64: lo xyz, hi xyz
    truncation: float = 0.0          # unbounded regions: radius of the truncation sphere

    @property
    def n_boxes(self) -> int:
        return 0 if self.boxes is None else int(self.boxes.shape[0])


@dataclasses.dataclass
class Dirichlet:
    kind: int
    x0: tuple = (0.0, 0.0, 0.0)
    strength: float = 1.0            # g = strength / (4 pi |x - x0|)
    lmax: int = 0
    clm: np.ndarray | None = None    # (lmax+1)^2, index l*l + l + m
    center: tuple = (0.0, 0.0, 0.0)
    scale: float = 1.0
    constant: float = 0.0


@dataclasses.dataclass
class PatchBatch:
    centers: np.ndarray              # (n, 3) float64, points on the boundary
    radius: np.ndarray               # (n,) float64
    n_theta: np.ndarray              # (n,) int32, polar Gauss order on the hemisphere
    n_phi: np.ndarray                # (n,) int32, azimuthal Gauss order
    n_rings: np.ndarray              # (n,) int32, panel rings on the patch
    n_sectors: np.ndarray            # (n,) int32, panel sectors on the patch
    walks: np.ndarray                # (n,) int64, walks per hemisphere node
    patch_id_base: int = 0

    @property
    def n(self) -> int:
        return int(self.centers.shape[0])

    def subset(self, idx) -> "PatchBatch":
        idx = np.asarray(idx)
        return PatchBatch(self.centers[idx].copy(), self.radius[idx].copy(),
                          self.n_theta[idx].copy(), self.n_phi[idx].copy(),
                          self.n_rings[idx].copy(), self.n_sectors[idx].copy(),
                          self.walks[idx].copy(), self.patch_id_base)


@dataclasses.dataclass
class Workload:
    name: str
    geometry: Geometry
    data: Dirichlet
    batch: PatchBatch
    epsilon: float = 1e-4
    seed: int = 0
    patch_ids: np.ndarray | None = None  # explicit RNG patch ids (default: base + index)


def _uniform_batch(centers, a, nt, nph, nr, ns, walks, base=0) -> PatchBatch:
    n = centers.shape[0]
    return PatchBatch(
        centers=np.ascontiguousarray(centers, dtype=np.float64),
        radius=np.full(n, a, dtype=np.float64),
        n_theta=np.full(n, nt, dtype=np.int32),
        n_phi=np.full(n, nph, dtype=np.int32),
        n_rings=np.full(n, nr, dtype=np.int32),
        n_sectors=np.full(n, ns, dtype=np.int32),
        walks=np.full(n, walks, dtype=np.int64),
        patch_id_base=base,
    )


def fibonacci_sphere(n: int, radius: float = 1.0) -> np.ndarray:
    """n points on a sphere: z_i = 1 - (2i+1)/n, azimuth i * golden angle."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def random_clm(lmax: int, seed: int = 0) -> np.ndarray:
    """c_lm ~ N(0,1), (lmax+1)^2 of them, PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((lmax + 1) ** 2)


# ---------------------------------------------------------------- configurations

def cube_single_patch(walks: int = 10_000, n_theta: int = 16, n_phi: int = 16,
                      n_rings: int = 8, n_sectors: int = 8) -> Workload:
    """Unit cube interior, point-source data below face z=0, one flat patch.

    x0 = (0.5, 0.5, -0.3), patch centre (0.5, 0.5, 0), a = 0.1, 8x8 panels,
    16x16 hemisphere nodes, 1e4 walks per node, epsilon = 1e-4, seed 0.
    """
    geom = Geometry(GEOM_BOX_INTERIOR, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0))
    data = Dirichlet(DATA_POINT_SOURCE, x0=(0.5, 0.5, -0.3), strength=1.0)
    batch = _uniform_batch(np.array([[0.5, 0.5, 0.0]]), 0.1, n_theta, n_phi,
                           n_rings, n_sectors, walks)
    return Workload("cube_1patch_a0.1_np64_P256", geom, data, batch)


def unit_ball(n_patches: int = 2000, walks: int = 4096, n_theta: int = 16,
              n_phi: int = 32, n_rings: int = 8, n_sectors: int = 16,
              lmax: int = 8, a: float = 0.1, seed: int = 0) -> Workload:
    """Unit ball interior with a random harmonic polynomial as data.

    g = sum_{l<=8} c_lm r^l Y_lm, c_lm ~ N(0,1) (PCG64(seed)); patch centres on a
    Fibonacci sphere; a = 0.1; 128 panels (8 rings x 16 sectors); 512
    hemisphere nodes (16 polar x 32 azimuthal); 4096 walks per node.
    """
    geom = Geometry(GEOM_BALL_INTERIOR, center=(0.0, 0.0, 0.0), radius=1.0)
    data = Dirichlet(DATA_HARMONIC_SH, lmax=lmax, clm=random_clm(lmax, seed),
                     center=(0.0, 0.0, 0.0), scale=1.0)
    batch = _uniform_batch(fibonacci_sphere(n_patches), a, n_theta, n_phi,
                           n_rings, n_sectors, walks)
    name = f"unit_ball_{n_patches}p_np{n_rings * n_sectors}_P{n_theta * n_phi}_W{walks}"
    return Workload(name, geom, data, batch)


def unit_ball_scaled(n_patches: int = 20_000, walks: int = 8192) -> Workload:
    """Unit-ball study scaled up: 256 panels (16x16), 1024 nodes (32x32), 8192 walks."""
    return unit_ball(n_patches=n_patches, walks=walks, n_theta=32, n_phi=32,
                     n_rings=16, n_sectors=16)


def wire_layout(n_wires: int = 200, seed: int = 0, outer_lo=(0.0, 0.0, 0.0),
                outer_hi=(64.0, 64.0, 16.0), gap: float = 0.6,
                max_tries: int = 200_000) -> np.ndarray:
    """Axis-aligned wire boxes inside the outer box, by rejection sampling.

    Layer k in {0..3} at z-centre 2 + 4k; x-oriented for even k, y-oriented for
    odd k; length U[2,20], width and thickness U[0.2,1.0]; gap >= 0.6 to other
    wires and to the outer box.  Returns (n, 6) float64 rows (lo xyz, hi xyz).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    olo = np.asarray(outer_lo, dtype=np.float64)
    ohi = np.asarray(outer_hi, dtype=np.float64)
    boxes: list[np.ndarray] = []
    tries = 0
    while len(boxes) < n_wires:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("wire layout: too many rejections")
        k = len(boxes) % 4
        length = rng.uniform(2.0, 20.0)
        width = rng.uniform(0.2, 1.0)
        thick = rng.uniform(0.2, 1.0)
        ext = np.array([length, width, thick]) if k % 2 == 0 else np.array([width, length, thick])
        zc = 2.0 + 4.0 * k
        cx = rng.uniform(olo[0] + gap + ext[0] / 2, ohi[0] - gap - ext[0] / 2)
        cy = rng.uniform(olo[1] + gap + ext[1] / 2, ohi[1] - gap - ext[1] / 2)
        c = np.array([cx, cy, zc])
        lo, hi = c - ext / 2, c + ext / 2
        ok = True
        for b in boxes:
            sep = np.maximum(b[:3] - hi, lo - b[3:])
            if np.max(sep) < gap:
                ok = False
                break
        if ok:
            boxes.append(np.concatenate([lo, hi]))
    return np.array(boxes, dtype=np.float64)


def wire_patch_centers(boxes: np.ndarray, n: int, a: float, seed: int = 1,
                       margin: float = 1e-9, max_tries: int = 5_000_000,
                       outer_lo=(0.0, 0.0, 0.0), outer_hi=(64.0, 64.0, 16.0), allow_wrapped: bool = True):
    """Area-uniform patch centres on the wire faces (reading R15).

    A centre c on face f of wire w is kept when no other wire and no face of the
    outer box comes within a of c (the ball meets one conductor only) and the
    wire is at least a thick along the face normal (the hemisphere is then
    star-shaped about its pole).  The ball may meet further faces of wire w (a
    wrapped patch); with allow_wrapped=False such centres are rejected too.
    Returns (centres (n,3), wire index (n,), faces met (n,), rejected).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ext = boxes[:, 3:] - boxes[:, :3]
    # face areas: faces 2*axis+side, area = product of the two other extents
    areas = np.stack([ext[:, 1] * ext[:, 2], ext[:, 1] * ext[:, 2],
                      ext[:, 0] * ext[:, 2], ext[:, 0] * ext[:, 2],
                      ext[:, 0] * ext[:, 1], ext[:, 0] * ext[:, 1]], axis=1)
    flat = areas.reshape(-1)
    prob = flat / flat.sum()
    olo = np.asarray(outer_lo)
    ohi = np.asarray(outer_hi)
    out, owner, nfaces = [], [], []
    rejected = 0
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("wire patch centres: too many rejections")
        idx = rng.choice(flat.size, p=prob)
        w, f = divmod(int(idx), 6)
        axis, side = divmod(f, 2)
        lo, hi = boxes[w, :3], boxes[w, 3:]
        c = rng.uniform(lo, hi)
        c[axis] = lo[axis] if side == 0 else hi[axis]
        good = ext[w, axis] >= a + margin     # star-shaped hemisphere
        # faces of wire w the ball reaches besides f
        met = 1
        for ax in range(3):
            if ax == axis:
                continue
            met += int(c[ax] - lo[ax] < a) + int(hi[ax] - c[ax] < a)
        if met > 1 and not allow_wrapped:
            good = False
        # the outer box and the other wires must stay farther than a
        if good and np.min(np.minimum(c - olo, ohi - c)) <= a + margin:
            good = False
        if good:
            e = np.maximum(np.maximum(boxes[:, :3] - c, 0.0), c - boxes[:, 3:])
            d = np.sqrt((e * e).sum(axis=1))
            d[w] = np.inf
            if np.min(d) <= a + margin:
                good = False
        if not good:
            rejected += 1
            continue
        out.append(c)
        owner.append(w)
        nfaces.append(met)
    return np.array(out), np.array(owner, dtype=np.int64), np.array(nfaces, dtype=np.int64), rejected


def _rect_disk_area(lo_u, hi_u, lo_v, hi_v, cu, cv, r, m=256):
    """Area of the rectangle [lo_u, hi_u] x [lo_v, hi_v] inside the disk of radius
    r about (cu, cv) (midpoint rule over u of the clipped chord)."""
    u0, u1 = max(lo_u, cu - r), min(hi_u, cu + r)
    if u1 <= u0:
        return 0.0
    u = u0 + (np.arange(m) + 0.5) * (u1 - u0) / m
    h = np.sqrt(np.maximum(r * r - (u - cu) ** 2, 0.0))
    chord = np.clip(np.minimum(hi_v, cv + h) - np.maximum(lo_v, cv - h), 0.0, None)
    return float(chord.sum() * (u1 - u0) / m)


def patch_area_on_box(box: np.ndarray, c: np.ndarray, a: float) -> float:
    """Area of the box surface inside the ball B(c, a) (all six faces)."""
    lo, hi = box[:3], box[3:]
    tot = 0.0
    for ax in range(3):
        o = [i for i in range(3) if i != ax]
        for fv in (lo[ax], hi[ax]):
            d = c[ax] - fv
            if abs(d) >= a:
                continue
            r = np.sqrt(a * a - d * d)
            tot += _rect_disk_area(lo[o[0]], hi[o[0]], lo[o[1]], hi[o[1]], c[o[0]], c[o[1]], r)
    return tot


def wires(n_patches: int = 10_000, walks: int = 2048, a: float = 0.3,
          seed: int = 0, allow_wrapped: bool = True) -> Workload:
    """200-wire layout in the grounded box [0,64]^2 x [0,16].

    Data: point source at the centre of wire 0 (outside the region).  Centres
    area-uniform on the wire faces (R15); a ball that reaches further faces of
    its wire gives a wrapped patch.  Collocation points by the intersected area
    (R8): n_p = clamp(round(area(S) / h^2), 32, 512), h = a / 8, as rings x
    sectors with rings = round(sqrt(n_p / pi)); hemisphere nodes by area bucket
    (R19): 16^2 on a flat patch, 24^2 up to 1.4 times its area, 32^2 above.
    The generator's rejected-centre count is kept in `rejected`.
    """
    boxes = wire_layout(seed=seed)
    geom = Geometry(GEOM_BOX_MINUS_BOXES, lo=(0.0, 0.0, 0.0), hi=(64.0, 64.0, 16.0),
                    boxes=boxes)
    x0 = tuple(0.5 * (boxes[0, :3] + boxes[0, 3:]))
    data = Dirichlet(DATA_POINT_SOURCE, x0=x0, strength=1.0)
    centers, owner, nfaces, rejected = wire_patch_centers(boxes, n_patches, a, seed=seed + 1,
                                                          allow_wrapped=allow_wrapped)
    h = a / 8.0
    flat_area = np.pi * a * a
    rings = np.zeros(n_patches, np.int32)
    sectors = np.zeros(n_patches, np.int32)
    nodes = np.zeros(n_patches, np.int32)
    for p in range(n_patches):
        area = patch_area_on_box(boxes[owner[p]], centers[p], a) if nfaces[p] > 1 else flat_area
        n_p = int(min(max(round(area / (h * h)), 32), 512))
        nr = max(2, int(round(np.sqrt(n_p / np.pi))))
        ns = max(8, int(round(n_p / nr)))
        while nr * ns > 512:
            ns -= 1
        rings[p], sectors[p] = nr, ns
        nodes[p] = 16 if area <= 1.0001 * flat_area else (24 if area <= 1.4 * flat_area else 32)
    batch = PatchBatch(centers=centers.astype(np.float64),
                       radius=np.full(n_patches, a),
                       n_theta=nodes.copy(), n_phi=nodes.copy(),
                       n_rings=rings, n_sectors=sectors,
                       walks=np.full(n_patches, walks, dtype=np.int64))
    wl = Workload(f"wires200_{n_patches}p_by_area", geom, data, batch)
    wl.rejected = rejected
    wl.faces_met = nfaces
    return wl


def half_space_charge(depth: float = 1.0, truncation: float = 1e5) -> tuple:
    """The planar-interface problem of Sec. 4.1.3 (Test 1): the region z > 0
    above the plane z = 0, a unit point charge at (0, 0, -depth) below it, so
    u = 1 / |x - (0, 0, -depth)| (point-source data of strength 4 pi); walks
    that leave the sphere of radius `truncation` about the origin have gone
    to infinity.  Returns (Geometry, Dirichlet)."""
    geom = Geometry(GEOM_HALF_SPACE, center=(0.0, 0.0, 0.0), truncation=truncation)
    data = Dirichlet(DATA_POINT_SOURCE, x0=(0.0, 0.0, -depth), strength=4.0 * np.pi)
    return geom, data


def sphere_exterior(n_patches: int = 64, R: float = 3.0, a: float = 1.0, walks: int = 1000,
                    n_theta: int = 16, n_phi: int = 32, n_rings: int = 8, n_sectors: int = 16,
                    truncation: float = 1e5) -> Workload:
    """Sec. 5.2: the DtN map on the sphere of radius R = 3 seen from outside,
    with unit potential on the sphere and u = 0 at infinity (u = R/|x|, exact
    Neumann data along the outward normal of the region, which points into the
    sphere: q = 1/R); patch centres on a Fibonacci sphere, a = 1, cap patches."""
    geom = Geometry(GEOM_BALL_EXTERIOR, center=(0.0, 0.0, 0.0), radius=R, truncation=truncation)
    data = Dirichlet(DATA_CONSTANT, constant=1.0)
    batch = _uniform_batch(fibonacci_sphere(n_patches, R), a, n_theta, n_phi, n_rings, n_sectors, walks)
    return Workload("sphere_exterior_R3", geom, data, batch, epsilon=1e-4, seed=0)


def thin_disk(b: float = 1.0, truncation: float = 1e5) -> tuple:
    """Test 4 of Sec. 4.1.3: space outside the thin disk of radius b in the plane
    z = 0 about the origin, the disk held at potential 1 (constant data), u = 0
    at infinity; walks that leave the sphere of radius `truncation` have gone
    to infinity.  Returns (Geometry, Dirichlet)."""
    geom = Geometry(GEOM_DISK_EXTERIOR, center=(0.0, 0.0, 0.0), radius=b, truncation=truncation)
    data = Dirichlet(DATA_CONSTANT, constant=1.0)
    return geom, data


def targets_in_ball(n: int, radius: float, margin: float, seed: int = 3) -> np.ndarray:
    """n points uniform in the ball |x| <= radius - margin (PCG64(seed))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = (radius - margin) * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    return v * r[:, None]


def targets_outside_ball(n: int, radius: float, margin: float, seed: int = 4) -> np.ndarray:
    """n points in the shell radius+margin <= |x| <= 2 radius."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = rng.uniform(radius + margin, 2.0 * radius, n)
    return v * r[:, None]


def points_in_box(n: int, lo, hi, margin: float, seed: int = 5) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(lo) + margin
    hi = np.asarray(hi) - margin
    return rng.uniform(lo, hi, size=(n, 3))


# ---------------------------------------------------------------- panel sets for the potential

def sphere_panels(n: int, radius: float = 1.0) -> tuple:
    """n equal-area panels of a sphere: collocation points on the Fibonacci
    lattice, outward normals, area 4 pi radius^2 / n each.  Returns (xyz,
    normals, areas)."""
    y = fibonacci_sphere(n, radius)
    return y, y / radius, np.full(n, 4.0 * math.pi * radius * radius / n)


def box_surface_panels(boxes: np.ndarray, h: float) -> tuple:
    """Square panels of side about h on the six faces of every box (rows lo, hi)
    with outward normals and areas.  Returns (xyz, normals, areas)."""
    xs, ns, ar = [], [], []
    for lo, hi in zip(boxes[:, :3], boxes[:, 3:]):
        for axis in range(3):
            u, v = [a for a in range(3) if a != axis]
            nu = max(1, int(round((hi[u] - lo[u]) / h)))
            nv = max(1, int(round((hi[v] - lo[v]) / h)))
            du, dv = (hi[u] - lo[u]) / nu, (hi[v] - lo[v]) / nv
            cu = lo[u] + du * (np.arange(nu) + 0.5)
            cv = lo[v] + dv * (np.arange(nv) + 0.5)
            gu, gv = np.meshgrid(cu, cv, indexing="ij")
            for side, val in ((-1.0, lo[axis]), (1.0, hi[axis])):
                p = np.empty((nu * nv, 3))
                p[:, axis] = val
                p[:, u] = gu.ravel()
                p[:, v] = gv.ravel()
                nrm = np.zeros((nu * nv, 3))
                nrm[:, axis] = side
                xs.append(p)
                ns.append(nrm)
                ar.append(np.full(nu * nv, du * dv))
    return np.concatenate(xs), np.concatenate(ns), np.concatenate(ar)


def panel_values(n: int, seed: int = 11) -> tuple:
    """Seeded N(0, 1) Neumann and Dirichlet values for n panels (PCG64(seed))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(n), rng.standard_normal(n)
