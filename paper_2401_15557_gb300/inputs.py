"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only *generates problem data*: triangulations, boundary edge lists,
coefficient fields and analytic source/boundary/exact functions.  It holds none
of the primal hybrid method's arithmetic (no topology tables, no element
matrices, no solve), so the CPU oracle and the CUDA path can both consume it
without sharing any code of the method.

Conventions (paper Section 2.1, Table 1):
  * ``xy``  float64 [nV, 2]  vertex coordinates (``coordinates.dat``),
  * ``tri`` int32  [nT, 3]  counter-clockwise triangles, 0-based (``elements.dat``),
  * ``dirichlet`` / ``neumann`` int32 [n, 2] boundary edges as vertex pairs,
    listed counter-clockwise along the boundary (``Dirichlet.dat``/``Neumann.dat``).

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014): the state is
advanced by the golden-gamma constant and mixed by two xor-shift-multiply
rounds; a uniform double takes the top 53 bits.  Seeds follow
``0x5048464D00000000 + 1000*workload + index``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 0x5048464D00000000
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def seed_for(workload: int, index: int = 0) -> int:
    return (SEED_BASE + 1000 * workload + index) & 0xFFFFFFFFFFFFFFFF


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first ``n`` outputs of SplitMix64 started from state ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int) -> np.ndarray:
    """``n`` doubles uniform in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """``n`` standard normals by Box-Muller on SplitMix64 uniforms."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:n]


@dataclass
class Mesh:
    xy: np.ndarray
    tri: np.ndarray
    dirichlet: np.ndarray
    neumann: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nV(self) -> int:
        return int(self.xy.shape[0])

    @property
    def nT(self) -> int:
        return int(self.tri.shape[0])


def _as_pairs(lst) -> np.ndarray:
    if len(lst) == 0:
        return np.zeros((0, 2), dtype=np.int32)
    return np.ascontiguousarray(np.asarray(lst, dtype=np.int32).reshape(-1, 2))


# ----------------------------------------------------------------------------
# Structured unit-square meshes
# ----------------------------------------------------------------------------

def fan_mesh(n: int) -> Mesh:
    """n triangles around one vertex: ring vertices 0..n-1 on the unit circle,
    the centre last (vertex n, so every spoke has it as its larger vertex),
    triangles (ring i, ring i+1, centre) counter-clockwise; the ring edges are
    Dirichlet.  The centre has valence n."""
    ang = 2.0 * np.pi * np.arange(n) / n
    xy = np.concatenate([np.stack([np.cos(ang), np.sin(ang)], axis=1), np.zeros((1, 2))]).astype(np.float64)
    i = np.arange(n)
    tri = np.stack([i, (i + 1) % n, np.full(n, n)], axis=1).astype(np.int32)
    dirichlet = np.stack([i, (i + 1) % n], axis=1).astype(np.int32)
    return Mesh(xy, tri, dirichlet, np.zeros((0, 2), np.int32), name="fan")


def square_mesh(n: int, dirichlet_sides=("left", "right"), x0=0.0, y0=0.0, size=1.0) -> Mesh:
    """n x n squares on [x0, x0+size] x [y0, y0+size]; every square is split by
    the diagonal from its lower-left to its upper-right corner.  Squares are
    numbered row-major (x fastest) and each contributes the triangles
    (ll, lr, ur) and (ll, ur, ul).  Sides not in ``dirichlet_sides`` are Neumann.
    """
    h = size / n
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    xy = np.stack([x0 + ii.ravel() * h, y0 + jj.ravel() * h], axis=1).astype(np.float64)
    # exact end coordinates (avoid x0 + n*h != x0 + size by rounding)
    xy[ii.ravel() == n, 0] = x0 + size
    xy[jj.ravel() == n, 1] = y0 + size

    def vid(i, j):
        return j * (n + 1) + i

    si, sj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    si = si.ravel()
    sj = sj.ravel()
    ll, lr, ur, ul = vid(si, sj), vid(si + 1, sj), vid(si + 1, sj + 1), vid(si, sj + 1)
    t1 = np.stack([ll, lr, ur], axis=1)
    t2 = np.stack([ll, ur, ul], axis=1)
    tri = np.empty((2 * n * n, 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2
    sides = {
        "bottom": [(vid(i, 0), vid(i + 1, 0)) for i in range(n)],
        "right": [(vid(n, j), vid(n, j + 1)) for j in range(n)],
        "top": [(vid(i + 1, n), vid(i, n)) for i in range(n)],
        "left": [(vid(0, j + 1), vid(0, j)) for j in range(n)],
    }
    dl, nl = [], []
    for s in ("bottom", "right", "top", "left"):
        (dl if s in dirichlet_sides else nl).extend(sides[s])
    return Mesh(xy, tri, _as_pairs(dl), _as_pairs(nl), name=f"square{n}", meta={"n": n, "h": h})


def criss_cross_level0() -> Mesh:
    """The level-0 triangulation of the unit square printed in Table 1 of the
    paper (converted to 0-based vertex numbers): four triangles around the
    centre, Dirichlet on y=0 and x=1, Neumann on y=1 and x=0."""
    xy = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [0.5, 0.5]], dtype=np.float64)
    tri = np.array([[5, 1, 2], [5, 3, 1], [5, 4, 3], [5, 2, 4]], dtype=np.int32) - 1
    dirichlet = np.array([[1, 2], [2, 4]], dtype=np.int32) - 1
    neumann = np.array([[4, 3], [3, 1]], dtype=np.int32) - 1
    return Mesh(xy, tri, dirichlet, neumann, name="crisscross0", meta={"level": 0})


def red_refine(m: Mesh) -> Mesh:
    """Uniform red refinement with the child layout of Listing 4 (Section 2.3):
    the first nT children are the middle triangles [M1 M2 M3], then for every
    parent t the corner children [P1 M3 M2], [P2 M1 M3], [P3 M2 M1] at positions
    nT+3t, nT+3t+1, nT+3t+2, where Mk is the midpoint of the edge opposite Pk.
    Boundary edges (a, b) become (a, m) in the first half of the list and (m, b)
    in the second half.  New midpoint vertices are appended after the old ones,
    numbered by the generator's own (min vertex, max vertex) order of the edges
    (vertex numbering does not change any result of the method).
    """
    tri = m.tri.astype(np.int64)
    nT, nV = tri.shape[0], m.nV
    # the three edges opposite P1, P2, P3
    ea = np.stack([tri[:, 1], tri[:, 2], tri[:, 0]], axis=1)
    eb = np.stack([tri[:, 2], tri[:, 0], tri[:, 1]], axis=1)
    lo = np.minimum(ea, eb).ravel()
    hi = np.maximum(ea, eb).ravel()
    key = lo * nV + hi
    ukey, inv = np.unique(key, return_inverse=True)
    mid_id = (nV + inv).reshape(nT, 3)
    ulo, uhi = ukey // nV, ukey % nV
    new_xy = 0.5 * (m.xy[ulo] + m.xy[uhi])
    xy = np.concatenate([m.xy, new_xy], axis=0)
    M1, M2, M3 = mid_id[:, 0], mid_id[:, 1], mid_id[:, 2]
    P1, P2, P3 = tri[:, 0], tri[:, 1], tri[:, 2]
    out = np.empty((4 * nT, 3), dtype=np.int64)
    out[:nT] = np.stack([M1, M2, M3], axis=1)
    out[nT + 0::3] = np.stack([P1, M3, M2], axis=1)
    out[nT + 1::3] = np.stack([P2, M1, M3], axis=1)
    out[nT + 2::3] = np.stack([P3, M2, M1], axis=1)

    def refine_edges(pairs):
        if len(pairs) == 0:
            return _as_pairs([])
        pairs = pairs.astype(np.int64)
        a, b = pairs[:, 0], pairs[:, 1]
        k = np.minimum(a, b) * nV + np.maximum(a, b)
        pos = np.searchsorted(ukey, k)
        if np.any(pos >= ukey.size) or np.any(ukey[np.minimum(pos, ukey.size - 1)] != k):
            raise ValueError("a boundary pair is not an edge of the mesh")
        mid = nV + pos
        return _as_pairs(np.concatenate([np.stack([a, mid], 1), np.stack([mid, b], 1)], 0))

    meta = dict(m.meta)
    meta["level"] = meta.get("level", 0) + 1
    if "h" in meta:
        meta["h"] = meta["h"] / 2
    return Mesh(xy, out.astype(np.int32), refine_edges(m.dirichlet), refine_edges(m.neumann),
                name=m.name.rstrip("0123456789r") + f"r{meta['level']}", meta=meta)


def criss_cross(level: int) -> Mesh:
    """Level ``level`` of the paper's experiments: the Table 1 mesh red-refined
    ``level`` times (4**(level+1) triangles, h = 2**-level)."""
    m = criss_cross_level0()
    for _ in range(level):
        m = red_refine(m)
    m.meta["level"] = level
    return m


# ----------------------------------------------------------------------------
# L-shaped domain [-1,1]^2 minus (0,1]^2 with jittered interior vertices
# ----------------------------------------------------------------------------

def lshape_mesh(n: int = 32, jitter: float = 0.2, seed: int | None = None, levels: int = 0) -> Mesh:
    """Three unit squares of n x n squares (h = 1/n) covering [-1,1]^2 minus
    (0,1]^2, each square split like :func:`square_mesh`.  Interior vertices are
    moved by r*(cos t, sin t)*jitter*h with r ~ U[0,1), t ~ U[0,2pi) (boundary
    vertices stay).  Dirichlet on the outer boundary, Neumann on the two
    re-entrant sides.  ``levels`` red refinements follow."""
    if seed is None:
        seed = seed_for(1, 0)
    N = 2 * n
    h = 1.0 / n
    gi, gj = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="xy")
    gi, gj = gi.ravel(), gj.ravel()
    keep = ~((gi > n) & (gj > n))
    vid = -np.ones((N + 1) * (N + 1), dtype=np.int64)
    vid[keep] = np.arange(int(keep.sum()))
    X = -1.0 + gi[keep] * h
    Y = -1.0 + gj[keep] * h
    X[gi[keep] == n] = 0.0
    Y[gj[keep] == n] = 0.0
    X[gi[keep] == N] = 1.0
    Y[gj[keep] == N] = 1.0
    xy = np.stack([X, Y], axis=1)

    def V(i, j):
        return vid[j * (N + 1) + i]

    si, sj = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    si, sj = si.ravel(), sj.ravel()
    sq = ~((si >= n) & (sj >= n))
    si, sj = si[sq], sj[sq]
    ll, lr, ur, ul = V(si, sj), V(si + 1, sj), V(si + 1, sj + 1), V(si, sj + 1)
    tri = np.empty((2 * si.size, 3), dtype=np.int64)
    tri[0::2] = np.stack([ll, lr, ur], 1)
    tri[1::2] = np.stack([ll, ur, ul], 1)

    # boundary, counter-clockwise
    outer, reent = [], []
    for i in range(N):                     # bottom y=-1
        outer.append((V(i, 0), V(i + 1, 0)))
    for j in range(n):                     # right x=1, y in [-1,0]
        outer.append((V(N, j), V(N, j + 1)))
    for i in range(N, n, -1):              # re-entrant y=0, x from 1 to 0
        reent.append((V(i, n), V(i - 1, n)))
    for j in range(n, N):                  # re-entrant x=0, y from 0 to 1
        reent.append((V(n, j), V(n, j + 1)))
    for i in range(n, 0, -1):              # top y=1, x from 0 to -1
        outer.append((V(i, N), V(i - 1, N)))
    for j in range(N, 0, -1):              # left x=-1
        outer.append((V(0, j), V(0, j - 1)))

    bnd = np.zeros(xy.shape[0], dtype=bool)
    for a, b in outer + reent:
        bnd[a] = bnd[b] = True
    u = uniform(seed, 2 * xy.shape[0])
    r, t = u[0::2], 2 * np.pi * u[1::2]
    move = ~bnd
    xy = xy.copy()
    xy[move, 0] += r[move] * np.cos(t[move]) * jitter * h
    xy[move, 1] += r[move] * np.sin(t[move]) * jitter * h
    m = Mesh(xy, tri.astype(np.int32), _as_pairs(outer), _as_pairs(reent), name=f"lshape{n}",
             meta={"n": n, "h": h, "level": 0, "seed": seed})
    for _ in range(levels):
        m = red_refine(m)
    return m


# ----------------------------------------------------------------------------
# Coefficients
# ----------------------------------------------------------------------------

def coeff_lshape(x, y):
    """a(x, y) = 1 + 0.5 sin(2 pi x) sin(2 pi y) of the L-shaped workload."""
    return 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)


@dataclass
class FourierField:
    alpha: np.ndarray
    k: np.ndarray
    phi: np.ndarray

    def z(self, x, y):
        out = np.zeros(np.broadcast(x, y).shape)
        for a, (kx, ky), p in zip(self.alpha, self.k, self.phi):
            out = out + a * np.cos(2 * np.pi * (kx * x + ky * y) + p)
        return out

    def a(self, x, y):
        return np.exp(0.5 * self.z(x, y))


def fourier_field(seed: int, modes: int = 8) -> FourierField:
    """z = sum_m alpha_m cos(2 pi k_m.(x,y) + phi_m), alpha ~ N(0,1)/sqrt(8),
    k_m integer in [-4,4]^2 minus {0}, phi ~ U[0, 2pi)."""
    alpha = normal(seed, modes) / math.sqrt(modes)
    u = uniform(seed ^ 0xA5A5A5A5A5A5A5A5, 4 * modes)
    ks = []
    j = 0
    while len(ks) < modes:
        if j + 1 >= u.size:
            u = np.concatenate([u, uniform(seed ^ (0x1234 + j), 4 * modes)])
        kx = int(np.floor(u[j] * 9)) - 4
        ky = int(np.floor(u[j + 1] * 9)) - 4
        j += 2
        if kx == 0 and ky == 0:
            continue
        ks.append((kx, ky))
    phi = 2 * np.pi * uniform(seed ^ 0x5A5A5A5A5A5A5A5A, modes)
    return FourierField(alpha, np.array(ks, dtype=np.int64), phi)


def element_mean_at_midpoints(xy: np.ndarray, tri: np.ndarray, func) -> np.ndarray:
    """Per-triangle coefficient a_T = mean of ``func`` at the three edge
    midpoints (the midpoint quadrature of the paper's load term, applied to a
    variable coefficient)."""
    P = xy[tri]
    m23 = 0.5 * (P[:, 1] + P[:, 2])
    m13 = 0.5 * (P[:, 0] + P[:, 2])
    m12 = 0.5 * (P[:, 0] + P[:, 1])
    return (func(m23[:, 0], m23[:, 1]) + func(m13[:, 0], m13[:, 1]) + func(m12[:, 0], m12[:, 1])) / 3.0


# ----------------------------------------------------------------------------
# Problem data (analytic functions).  g takes the outward unit normal.
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    """Data of -div(a grad u) + p.grad u + delta u = f, u = uD on Gamma_D,
    grad u . nu = g on Gamma_N (A = a I).  ``u``/``grad`` are the exact
    solution where known.  Time-dependent problems take an extra ``t``."""
    f: object
    g: object
    uD: object
    u: object = None
    grad: object = None
    delta: float = 0.0
    p: tuple = (0.0, 0.0)
    A: np.ndarray | None = None
    u0: object = None


def problem_sine_exp() -> Problem:
    """u = sin(pi x) e^y on the unit square; -Lap u = (pi^2 - 1) u."""
    pi = np.pi
    u = lambda x, y: np.sin(pi * x) * np.exp(y)
    grad = lambda x, y: (pi * np.cos(pi * x) * np.exp(y), np.sin(pi * x) * np.exp(y))
    f = lambda x, y: (pi * pi - 1.0) * np.sin(pi * x) * np.exp(y)

    def g(x, y, nx, ny):
        gx, gy = grad(x, y)
        return gx * nx + gy * ny

    return Problem(f=f, g=g, uD=u, u=u, grad=grad, delta=0.0)


def problem_linear(cx=0.7, cy=-0.4, c0=0.3, delta=0.0) -> Problem:
    """Patch test data: u = c0 + cx x + cy y, a = 1, f = delta u."""
    u = lambda x, y: c0 + cx * x + cy * y
    grad = lambda x, y: (cx + 0 * x, cy + 0 * y)
    f = lambda x, y: delta * u(x, y)
    g = lambda x, y, nx, ny: cx * nx + cy * ny
    return Problem(f=f, g=g, uD=u, u=u, grad=grad, delta=delta)


def problem_paper_example1() -> Problem:
    """Example 1 of Section 3: A = I, p = (1,1), delta = 1,
    u = (x - x^2)(y - y^2); f includes +p.grad u; g = (grad u + u p).nu."""
    u = lambda x, y: (x - x * x) * (y - y * y)
    grad = lambda x, y: ((1 - 2 * x) * (y - y * y), (x - x * x) * (1 - 2 * y))

    def f(x, y):
        return (2 * (y - y * y) + 2 * (x - x * x) + (1 - 2 * x) * (y - y * y)
                + (x - x * x) * (1 - 2 * y) + u(x, y))

    def g(x, y, nx, ny):
        return (1 - x - x * x) * (y - y * y) * nx + (x - x * x) * (1 - y - y * y) * ny

    return Problem(f=f, g=g, uD=lambda x, y: 0 * x, u=u, grad=grad, delta=1.0, p=(1.0, 1.0))


def problem_paper_example2() -> Problem:
    """Example 2 of Section 4: u = t (x - x^2)(y - y^2), A = I, p = (1,1),
    delta = 1, u0 = 0, uD = 0."""
    s = lambda x, y: (x - x * x) * (y - y * y)
    u = lambda x, y, t: t * s(x, y)
    grad = lambda x, y, t: (t * (1 - 2 * x) * (y - y * y), t * (x - x * x) * (1 - 2 * y))

    def f(x, y, t):
        return (s(x, y) + 2 * t * (y - y * y) + 2 * t * (x - x * x) + t * (1 - 2 * x) * (y - y * y)
                + t * (x - x * x) * (1 - 2 * y) + u(x, y, t))

    def g(x, y, nx, ny, t):
        return t * ((1 - x - x * x) * (y - y * y) * nx + (x - x * x) * (1 - y - y * y) * ny)

    return Problem(f=f, g=g, uD=lambda x, y, t: 0 * x, u=u, grad=grad, delta=1.0, p=(1.0, 1.0),
                   u0=lambda x, y: 0 * x)


def problem_heat_sine() -> Problem:
    """u = e^{-t} sin(pi x) sin(pi y) with u_t - Lap u = f, f = (2 pi^2 - 1) u;
    Dirichlet 0 on x = 0, 1; g = -pi e^{-t} sin(pi x) on y = 0 and y = 1."""
    pi = np.pi
    u = lambda x, y, t: np.exp(-t) * np.sin(pi * x) * np.sin(pi * y)
    grad = lambda x, y, t: (pi * np.exp(-t) * np.cos(pi * x) * np.sin(pi * y),
                            pi * np.exp(-t) * np.sin(pi * x) * np.cos(pi * y))
    f = lambda x, y, t: (2 * pi * pi - 1.0) * u(x, y, t)

    def g(x, y, nx, ny, t):
        gx, gy = grad(x, y, t)
        return gx * nx + gy * ny

    return Problem(f=f, g=g, uD=lambda x, y, t: 0 * x, u=u, grad=grad, delta=0.0,
                   u0=lambda x, y: u(x, y, 0.0))


# ----------------------------------------------------------------------------
# Workload recipes
# ----------------------------------------------------------------------------

def batch_sides(count: int = 4096, seed: int | None = None, lo: int = 8, hi: int = 256) -> np.ndarray:
    """Side counts n_i = round(exp(U[ln lo, ln hi])) of the batched workload."""
    if seed is None:
        seed = seed_for(3, 0)
    u = uniform(seed, count)
    return np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def batch_member(i: int, n: int, workload: int = 3):
    """Mesh i of the batched workload: an n x n unit square (Dirichlet x=0,1,
    Neumann y=0,1), a_T from a = exp(0.5 z) with a seeded Fourier field z,
    reaction delta ~ U[0,2], f = 1, homogeneous boundary data."""
    seed = seed_for(workload, i + 1)
    m = square_mesh(int(n))
    fld = fourier_field(seed)
    aT = element_mean_at_midpoints(m.xy, m.tri, fld.a)
    delta = 2.0 * float(uniform(seed ^ 0xDE17A, 1)[0])
    return m, aT, delta


def poisson_arrivals(count: int, rate: float, seed: int | None = None) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given mean rate."""
    if seed is None:
        seed = seed_for(4, 0)
    u = uniform(seed, count)
    return np.cumsum(-np.log(1.0 - u) / rate)


# ----------------------------------------------------------------------------
# Problem data at the edges of a numbered mesh
# ----------------------------------------------------------------------------

def edge_data(xy: np.ndarray, ed2el: np.ndarray, eclass: np.ndarray, f, g=None, uD=None, t=None):
    """Sample the problem data at the midpoints of the edges of a mesh whose
    edge table ``ed2el`` ([initial, end, T+, T-]) and classes (0 interior,
    1 Dirichlet, 2 Neumann) are given: ``f_mid`` = f(m_E) on every edge and
    ``bc_mid`` = u_D(m_E) on Dirichlet edges, g(m_E, nu) on Neumann edges with
    nu the outward unit normal (initial -> end runs counter-clockwise around
    the only triangle of a boundary edge), 0 elsewhere."""
    a = xy[ed2el[:, 0]]
    b = xy[ed2el[:, 1]]
    mid = 0.5 * (a + b)
    x, y = mid[:, 0], mid[:, 1]
    targs = () if t is None else (t,)
    f_mid = np.broadcast_to(np.asarray(f(x, y, *targs), dtype=np.float64), x.shape).copy()
    bc = np.zeros(x.shape)
    D = eclass == 1
    N = eclass == 2
    if uD is not None and D.any():
        bc[D] = uD(x[D], y[D], *targs)
    if g is not None and N.any():
        d = b[N] - a[N]
        L = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
        bc[N] = g(x[N], y[N], d[:, 1] / L, -d[:, 0] / L, *targs)
    return f_mid, bc
