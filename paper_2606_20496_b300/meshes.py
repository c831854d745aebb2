"""Seeded synthetic inputs: hexahedral meshes, element partitions, right-hand sides.

This module holds no arithmetic of the coarse-grid method itself; it only lays
out vertex coordinates, element connectivity, the element partition into
subdomains and random right-hand sides.  Both the CUDA path and the CPU oracle
take their inputs from here, so parity never depends on a random generator.

Conventions
-----------
* ``xyz``  : float64 array (nv, 3) of vertex coordinates.
* ``conn`` : int32 array (E, 8); local vertex k = a + 2b + 4c addresses the
  corner (a, b, c) in {0,1}^3 of the reference hexahedron (lexicographic, the
  ordering the paper uses for element-local data, Sec. 1).
* ``part`` : int32 array (E,) subdomain id of each element (Omega_p, Sec. 3).
* ``eijk`` : int32 array (E, 3) structured index of each element (kept for
  tests; the method never reads it).

The workloads stand in for the paper's production meshes (T-junction and
pebble beds, Sec. 5), which are not available: unstructured hex meshes with
27-64 dof local blocks and a reduced space of a few thousand unknowns.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    xyz: np.ndarray
    conn: np.ndarray
    part: np.ndarray
    eijk: np.ndarray
    boxes: tuple
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def ne(self) -> int:
        return int(self.conn.shape[0])


def segments(n: int, mode: str = "two") -> list:
    """Split n element layers into partition segments along one axis.

    mode "two":   blocks of 2, a final block of 1 when n is odd.
    mode "mixed": as many 3-blocks as leave an even remainder, then 2-blocks
                  (4 -> 2+2, 5 -> 3+2, 7 -> 3+2+2); n = 1 gives [1].
    """
    if n <= 0:
        return []
    if mode == "two":
        s = [2] * (n // 2)
        if n % 2:
            s.append(1)
        return s
    if mode == "mixed":
        if n == 1:
            return [1]
        t = n // 3
        while t >= 0 and (n - 3 * t) % 2:
            t -= 1
        return [3] * t + [2] * ((n - 3 * t) // 2)
    raise ValueError(mode)


def _segment_ids(n: int, mode: str) -> np.ndarray:
    ids = np.empty(n, dtype=np.int64)
    pos = 0
    for s_id, s in enumerate(segments(n, mode)):
        ids[pos:pos + s] = s_id
        pos += s
    return ids


def _block_partition(eijk: np.ndarray, dims, mode: str) -> np.ndarray:
    sx, sy, sz = (_segment_ids(d, mode) for d in dims)
    nbx = int(sx.max()) + 1
    nby = int(sy.max()) + 1
    p = sx[eijk[:, 0]] + nbx * (sy[eijk[:, 1]] + nby * sz[eijk[:, 2]])
    return p.astype(np.int32)


def _hex_conn(dims, periodic_y: bool = False):
    """Connectivity of a structured nx*ny*nz brick of hexes (lexicographic)."""
    nx, ny, nz = dims
    vx, vy = nx + 1, (ny if periodic_y else ny + 1)
    ei, ej, ek = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ei, ej, ek = (a.transpose(2, 1, 0).ravel() for a in (ei, ej, ek))  # i fastest
    conn = np.empty((ei.size, 8), dtype=np.int64)
    for c in range(2):
        for b in range(2):
            for a in range(2):
                jj = (ej + b) % vy if periodic_y else ej + b
                conn[:, a + 2 * b + 4 * c] = (ei + a) + vx * (jj + vy * (ek + c))
    eijk = np.stack([ei, ej, ek], axis=1).astype(np.int32)
    return conn.astype(np.int32), eijk


def _grid_points(dims):
    nx, ny, nz = dims
    i, j, k = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    return (a.transpose(2, 1, 0).ravel() for a in (i, j, k))


def cube(dims, perturb: float = 0.0, seed=None, deform: bool = False,
         permute_seed=None, part_mode: str = "two", boxes=None, name: str = "cube") -> Mesh:
    """Unit-cube brick of nx*ny*nz trilinear hexes.

    perturb : interior vertices move by U(-perturb*h, +perturb*h) per
              coordinate, h the element size along that axis; the nv*3
              draws come from ``default_rng(seed)`` and only interior
              vertices use theirs.
    deform  : the smooth map x += 0.1 sin(pi y) sin(pi z) and its cyclic
              permutations, evaluated on the undeformed coordinates.
    permute_seed : renumber elements by ``default_rng(permute_seed).permutation(E)``
              so that the connectivity carries no structure.
    """
    if np.isscalar(dims):
        dims = (int(dims),) * 3
    dims = tuple(int(d) for d in dims)
    nx, ny, nz = dims
    conn, eijk = _hex_conn(dims)
    i, j, k = _grid_points(dims)
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    xyz = np.stack([i * h[0], j * h[1], k * h[2]], axis=1).astype(np.float64)
    if perturb:
        rng = np.random.default_rng(seed)
        noise = rng.uniform(-1.0, 1.0, size=xyz.shape) * (perturb * h)
        interior = (i > 0) & (i < nx) & (j > 0) & (j < ny) & (k > 0) & (k < nz)
        xyz[interior] += noise[interior]
    if deform:
        x, y, z = xyz[:, 0].copy(), xyz[:, 1].copy(), xyz[:, 2].copy()
        xyz[:, 0] = x + 0.1 * np.sin(np.pi * y) * np.sin(np.pi * z)
        xyz[:, 1] = y + 0.1 * np.sin(np.pi * z) * np.sin(np.pi * x)
        xyz[:, 2] = z + 0.1 * np.sin(np.pi * x) * np.sin(np.pi * y)
    part = _block_partition(eijk, dims, part_mode)
    if permute_seed is not None:
        perm = np.random.default_rng(permute_seed).permutation(conn.shape[0])
        conn, eijk, part = conn[perm], eijk[perm], part[perm]
    if boxes is None:
        boxes = tuple(int(min(max(-(-d // 4), 2), 16)) for d in dims)
    return Mesh(xyz=xyz, conn=np.ascontiguousarray(conn), part=np.ascontiguousarray(part),
                eijk=np.ascontiguousarray(eijk), boxes=tuple(boxes), name=name,
                meta={"dims": dims})


def cylinder(nr: int = 64, nt: int = 128, nz: int = 128, r_in: float = 1.0, r_out: float = 2.0,
             grading: float = 1.05, aspect: float = 100.0, boxes=(16, 16, 16),
             part_mode: str = "two", name: str = "cylinder") -> Mesh:
    """Hollow cylinder r_in <= r <= r_out, periodic in azimuth.

    Radial sizes grow geometrically, h_k = h_0 * grading**k, summing to
    r_out - r_in.  The axial length is nz * aspect * h_0, so the axial/radial
    aspect ratio of the innermost elements equals ``aspect``.  Vertex index
    ir + (nr+1) * (it + nt * iz); element corners follow (r, theta, z), a
    right-handed frame, so every element has a positive Jacobian.
    """
    if grading == 1.0:
        h0 = (r_out - r_in) / nr
        radii = r_in + h0 * np.arange(nr + 1)
    else:
        h0 = (r_out - r_in) * (grading - 1.0) / (grading ** nr - 1.0)
        radii = r_in + h0 * (grading ** np.arange(nr + 1) - 1.0) / (grading - 1.0)
        radii[-1] = r_out
    length = nz * aspect * h0
    dims = (nr, nt, nz)
    conn, eijk = _hex_conn(dims, periodic_y=True)
    ir, it, iz = np.meshgrid(np.arange(nr + 1), np.arange(nt), np.arange(nz + 1), indexing="ij")
    ir, it, iz = (a.transpose(2, 1, 0).ravel() for a in (ir, it, iz))
    theta = 2.0 * np.pi * it / nt
    r = radii[ir]
    xyz = np.stack([r * np.cos(theta), r * np.sin(theta), iz * (length / nz)], axis=1)
    part = _block_partition(eijk, dims, part_mode)
    return Mesh(xyz=xyz.astype(np.float64), conn=conn, part=part, eijk=eijk, boxes=tuple(boxes),
                name=name, meta={"dims": dims, "h0": h0, "length": length})


def outflow_dirichlet(mesh, axis: int = 2) -> np.ndarray:
    """Dirichlet mask for Neumann boundaries everywhere except an outflow cap:
    the vertices at the largest coordinate along `axis` (the end of the
    cylinder or the top of a cube), as uint8 (1 = Dirichlet)."""
    c = mesh.xyz[:, axis]
    return (c >= c.max() - 1e-12 * max(abs(c.max()), 1.0)).astype(np.uint8)


def rhs(nv: int, seed, count: int | None = None) -> np.ndarray:
    """i.i.d. N(0,1) right-hand side(s) of length nv from ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    if count is None:
        return rng.standard_normal(nv)
    return rng.standard_normal((count, nv))


# ---------------------------------------------------------------------------
# The five workloads.  Where the workload text is silent (seeds for config 2
# and 3, cylinder radii and length, box counts of the batched meshes), the
# readings are the ones listed with the input recipe in the design notes.
# ---------------------------------------------------------------------------

def workload_cube8() -> tuple:
    """8^3 perturbed unit cube (729 vertices), 4^3 boxes, RHS seed 1."""
    m = cube(8, perturb=0.15, seed=0, boxes=(4, 4, 4), name="cube8_perturbed")
    return m, rhs(m.nv, 1)


def workload_cube32() -> tuple:
    """32^3 smoothly deformed cube, elements randomly renumbered, 8^3 boxes."""
    m = cube(32, deform=True, permute_seed=4, boxes=(8, 8, 8), name="cube32_deformed_permuted")
    return m, rhs(m.nv, 5)


def workload_cylinder(scale: int = 1) -> tuple:
    """Hollow cylinder 64 x 128 x 128 (1,073,280 vertices), 16^3 boxes.

    ``scale`` > 1 divides each element count by ``scale`` (a reduced twin with
    the same grading over the same radial span and the same 1:100 aspect).
    """
    nr, nt, nz = 64 // scale, 128 // scale, 128 // scale
    grading = 1.05 ** scale
    m = cylinder(nr, nt, nz, grading=grading, aspect=100.0, boxes=(16, 16, 16) if scale == 1 else
                 tuple(max(2, 16 // scale) for _ in range(3)),
                 name="hollow_cylinder" if scale == 1 else f"hollow_cylinder_div{scale}")
    return m, rhs(m.nv, 6)


def workload_batch(count: int = 256, seed: int = 2) -> list:
    """Batched cubes: edge n_e ~ U{4..24} (seed 2), perturbation seed [2, i],
    mixed 2/3-element subdomain segments, 4 right-hand sides each."""
    n_e = np.random.default_rng(seed).integers(4, 25, count)
    out = []
    for i, n in enumerate(n_e):
        m = cube(int(n), perturb=0.15, seed=[seed, i], part_mode="mixed", name=f"batch{i}_n{int(n)}")
        out.append((m, rhs(m.nv, [seed, i, 1], count=4)))
    return out


# ---------------------------------------------------------------------------
# The p-multigrid wrap: spectral elements of order N on the same hexahedra.
# Its nodes are numbered differently by every implementation, so the
# right-hand side is a function of the node coordinates, not a list.
# ---------------------------------------------------------------------------

def sem_rhs(coords: np.ndarray, seed: int = 9, waves: int = 24, kmax: float = 40.0) -> np.ndarray:
    """f(x) = sum_m a_m sin(k_m . x + phi_m) at the points coords (n, 3):
    ``waves`` plane waves with wave numbers up to ``kmax`` (smooth and rough
    components together), amplitudes N(0,1), phases U(0, 2 pi), all drawn
    from ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(-kmax, kmax, size=(waves, 3))
    a = rng.standard_normal(waves)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=waves)
    return np.sin(np.asarray(coords, dtype=np.float64) @ k.T + phi) @ a


def workload_sem() -> tuple:
    """The 32^3 smoothly deformed cube with spectral elements of order 7 and
    the schedule 7 -> 3 -> 1 (11,390,625 nodes at order 7); the order-1 level
    is the 35,937-vertex coarse problem with its 8^3 boxes."""
    m, _ = workload_cube32()
    return m, (7, 3)


def workload_sem_small() -> tuple:
    """The 8^3 perturbed cube at order 7, schedule 7 -> 3 -> 1 (185,193 nodes)."""
    m, _ = workload_cube8()
    return m, (7, 3)
