"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only draws numbers and lays out meshes; it holds none of the
method's arithmetic (no basis, no geometric factors, no contractions).  Both
sides receive exactly the same arrays from here.

Generator: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based generator: draw i of
stream `seed` is mix64(seed + (i + 1) * 0x9E3779B97F4A7C15), and the top 53
bits give a double in [0, 1).

Mesh recipe (the paper's test meshes are cubes of 512 and 4096 hexahedra,
Section 3): an nx x ny x nz structured grid of the unit cube, spacing
h = 1/nx (per direction), every interior vertex coordinate moved
independently by U[-0.1h, 0.1h], boundary vertices fixed, elements mapped
trilinearly (Section 4: each hexahedron is the image of the bi-unit cube
under a trilinear map).  Element e = ex + nx*(ey + ny*ez).  Corner
c = cr + 2*cs + 4*ct (cr, cs, ct in {0,1} meaning r, s, t = -1 or +1) stores
x, y, z innermost: verts[e, c, d].
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_MESH = 1
SEED_Q = 2
SEED_BATCH = 3
SEED_SERVE = 4


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of stream `seed` as uint64."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, lo: float = 0.0, hi: float = 1.0,
            offset: int = 0) -> np.ndarray:
    """count doubles uniform in [lo, hi) from stream `seed`."""
    u = (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64)
    u *= 2.0 ** -53
    return lo + (hi - lo) * u


def box_mesh(nx: int, ny: int | None = None, nz: int | None = None,
             jitter: float = 0.1, seed: int = SEED_MESH,
             extent=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Vertices (E, 8, 3) float64 of a jittered structured hex mesh of a box.

    jitter is the fraction of the local spacing by which each interior vertex
    coordinate is moved, uniformly in [-jitter*h, jitter*h].
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    ex, ey, ez = extent
    gx = np.linspace(0.0, ex, nx + 1)
    gy = np.linspace(0.0, ey, ny + 1)
    gz = np.linspace(0.0, ez, nz + 1)
    Z, Y, X = np.meshgrid(gz, gy, gx, indexing="ij")
    P = np.stack([X, Y, Z], axis=-1)  # (nz+1, ny+1, nx+1, 3)
    if jitter:
        h = np.array([ex / nx, ey / ny, ez / nz])
        d = uniform(seed, P.size, -1.0, 1.0).reshape(P.shape) * jitter * h
        interior = np.zeros(P.shape[:3], dtype=bool)
        interior[1:-1, 1:-1, 1:-1] = True
        # a vertex on a face of the box keeps its normal coordinate but may
        # slide within the face only if it is interior to that face; the
        # recipe keeps every boundary vertex fixed, so only interior ones move
        P = P + d * interior[..., None]
    E = nx * ny * nz
    V = np.empty((nz, ny, nx, 8, 3))
    for c in range(8):
        cr, cs, ct = c & 1, (c >> 1) & 1, (c >> 2) & 1
        V[:, :, :, c, :] = P[ct:ct + nz, cs:cs + ny, cr:cr + nx, :]
    return np.ascontiguousarray(V.reshape(E, 8, 3))


def near_cube_dims(E: int) -> tuple[int, int, int]:
    """nx, ny, nz with nx*ny*nz == E and the box as close to a cube as the
    factors of E allow (used for the mixed-size mesh batches)."""
    best = None
    for nz in range(1, int(round(E ** (1 / 3))) + 2):
        if E % nz:
            continue
        rest = E // nz
        for ny in range(nz, int(rest ** 0.5) + 2):
            if rest % ny:
                continue
            nx = rest // ny
            dims = tuple(sorted((nx, ny, nz)))
            spread = dims[2] / dims[0]
            if best is None or spread < best[0]:
                best = (spread, dims)
    return best[1]


def field(seed: int, E: int, npts: int, lo: float = -1.0, hi: float = 1.0,
          offset: int = 0) -> np.ndarray:
    """Element-local field (E, npts) uniform in [lo, hi)."""
    return uniform(seed, E * npts, lo, hi, offset).reshape(E, npts)


def batch_workload(count: int = 64, seed: int = SEED_BATCH, nmin: int = 2, nmax: int = 10,
                   emin: int = 64, emax: int = 8192):
    """Mixed-order batch recipe: `count` independent meshes, degree N uniform
    in nmin..nmax, element count log-uniform in [emin, emax] rounded to a
    near-cubic nx x ny x nz box of the unit cube, each jittered by its own
    seed.  Returns a list of dicts (N, nx, ny, nz, E, mesh_seed)."""
    u = uniform(seed, 2 * count)
    out = []
    for i in range(count):
        N = nmin + min(int(u[2 * i] * (nmax - nmin + 1)), nmax - nmin)
        target = float(np.exp(np.log(emin) + u[2 * i + 1] * (np.log(emax) - np.log(emin))))
        nx = max(1, int(round(target ** (1.0 / 3.0))))
        ny = max(1, int(round((target / nx) ** 0.5)))
        nz = max(1, int(round(target / (nx * ny))))
        out.append({"N": N, "nx": nx, "ny": ny, "nz": nz, "E": nx * ny * nz,
                    "mesh_seed": seed * 1000 + i})
    return out


def serve_workload(count: int, seed: int = SEED_SERVE, rate: float = 200.0, nmin: int = 3, nmax: int = 9,
                   emin: int = 512, emax: int = 32768):
    """Request stream recipe: Poisson arrivals (exponential gaps of mean
    1/rate seconds), operator BP3.0 or BP3.5 and precision mode (FP64 or
    mixed) each with probability 1/2, degree N uniform in nmin..nmax, element
    count log-uniform in [emin, emax] as a near-cubic box of the unit cube.
    Returns dicts (t, op, N, nx, ny, nz, E, mixed, mesh_seed, rhs_seed); op is
    3 for BP3.0 and 2 for BP3.5."""
    u = uniform(seed, 5 * count)
    t = 0.0
    out = []
    for i in range(count):
        t += -np.log(1.0 - u[5 * i]) / rate
        op = 3 if u[5 * i + 1] < 0.5 else 2
        N = nmin + min(int(u[5 * i + 2] * (nmax - nmin + 1)), nmax - nmin)
        target = float(np.exp(np.log(emin) + u[5 * i + 3] * (np.log(emax) - np.log(emin))))
        nx = max(1, int(round(target ** (1.0 / 3.0))))
        ny = max(1, int(round((target / nx) ** 0.5)))
        nz = max(1, int(round(target / (nx * ny))))
        out.append({"t": t, "op": op, "N": N, "nx": nx, "ny": ny, "nz": nz, "E": nx * ny * nz,
                    "mixed": bool(u[5 * i + 4] < 0.5), "mesh_seed": seed * 100000 + 2 * i,
                    "rhs_seed": seed * 100000 + 2 * i + 1})
    return out
