"""ORACLE for the lowest-order primal hybrid FEM -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 CPU restatement of "Vectorized implementation of primal
hybrid FEM in MATLAB" (Nagula Mallesham, Porwal, Valdman, Acharya;
arXiv 2401.15557).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in ``oracle/``; the
product (the CUDA library and its Python binding) never does, and this module
imports nothing from the product.  It shares no code with the CUDA path: the
two only consume the same seeded inputs.

What it computes, in the paper's order and notation:
  * uniform red refinement (Section 2.3, redrefine_vec) and the prolongation
    of Crouzeix-Raviart functions from a mesh to its refinement (the coarse
    piecewise-linear function evaluated at the fine edge midpoints);
  * topology (Section 2.2, Eqs. n2el/n2ed/ed2el, Listings 1-3): nodes2element,
    nodes2edge (edges numbered by the column-major order of triu(B)),
    edge2element = [initial, end, T+, T-] with T+ the first element (element-major
    order of the directed edges P1P2, P2P3, P3P1) that holds the edge, led/ledTN;
  * local matrices (Definition 3.1): B_T, D_T, M_T, C_T with the rows R_k;
  * load and boundary data (Eqs. right_b, right_g, DirichletEqn);
  * the saddle-point system Mvec Wvec = Fvec (Section 3.5) and its direct solve;
  * Crank-Nicolson (Section 4, Eq. MatrixformParabolic) M+ W^n = M- W^{n-1} + F;
  * the condensed edge ("Crouzeix-Raviart") system obtained by eliminating the
    element unknowns with u_T = R^{-1} w_T (the equivalence stated in the
    introduction; the multiplier constraint forces midpoint continuity), its
    recovery of U and Lambda, and a plain Jacobi-PCG for large meshes;
  * the multiplier ("flux") Schur complement C K^{-1} C' of the same saddle
    system (reaction delta > 0) and its recovery of U;
  * error norms: L2, broken H1 seminorm, and a mesh M-norm of kappa - kappa_h.

Readings of passages that are ambiguous:
  * Convection uses the listing's column-constant D_T[r, c] = |T|/3 p.grad(lambda_c)
    (the test function is the row), which is the sign that Example 1's f needs.
  * The Neumann datum g is the scalar normal flux; the outward normal of a
    boundary edge is that of its only triangle.
  * In Crank-Nicolson the matrix multiplying (1 +- k delta/2) is the pure mass
    matrix (delta scales only the reaction part); sources are averaged by the
    trapezoid rule (F^n + F^{n-1})/2 as printed; U^0 = R^{-1}[u0(m_E)] per
    element, Lambda^0 given (default 0).
  * The M-norm of the multiplier error is computed as
    sqrt(sum_{E not Neumann} |E| int_E (kappa - kappa_h,E)^2) (the paper does
    not print PHerror).  The formula is pinned by values worked out by hand on
    the two-triangle square; the paper's M-norm column is not reproduced by it
    (only its rate is).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# Rows R_k of Definition 3.1: R_k[j] = lambda_j(m_{E_k}); E_k is opposite P_k.
R = np.array([[0.0, 0.5, 0.5],
              [0.5, 0.0, 0.5],
              [0.5, 0.5, 0.0]])


# ---------------------------------------------------------------------------
# Topology: Section 2.2, Listings 1-3
# ---------------------------------------------------------------------------

def nodes2element(tri: np.ndarray, nV: int) -> sp.csr_matrix:
    """Eq. (n2el): entry (k, l) = j (1-based) if k -> l is a directed edge of
    element j, for the directed edges P1->P2, P2->P3, P3->P1 of each element."""
    nT = tri.shape[0]
    I = tri.ravel()
    J = tri[:, [1, 2, 0]].ravel()
    S = np.repeat(np.arange(1, nT + 1), 3)
    A = sp.coo_matrix((S, (I, J)), shape=(nV, nV)).tocsr()
    # a directed edge owned by two elements would have been summed: reject
    ones = sp.coo_matrix((np.ones_like(S), (I, J)), shape=(nV, nV)).tocsr()
    if ones.nnz and ones.data.max() > 1:
        raise ValueError("a directed edge belongs to two elements (orientation clash)")
    return A


def nodes2edge(n2el: sp.csr_matrix) -> tuple[sp.csr_matrix, np.ndarray, np.ndarray]:
    """Eq. (n2ed), Listing 2: the nonzeros of triu(n2el + n2el') enumerated in
    column-major order get the edge numbers 1..nrEdges.  Returns the symmetric
    sparse map (1-based values) and the (row, col) node pair of every edge."""
    nV = n2el.shape[0]
    Bm = (n2el + n2el.T).tocsr()
    U = sp.triu(Bm, k=1).tocsc()
    U.sort_indices()
    col = np.repeat(np.arange(nV), np.diff(U.indptr))
    row = U.indices.copy()
    num = np.arange(1, row.size + 1)
    half = sp.coo_matrix((num, (row, col)), shape=(nV, nV))
    n2ed = (half + half.T).tocsr()
    return n2ed, row, col


def _lookup(M: sp.csr_matrix, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    if i.size == 0:
        return np.zeros(0, dtype=np.int64)
    return np.asarray(M[i, j]).ravel().astype(np.int64)


def edge_tables(tri: np.ndarray, nV: int) -> dict:
    """Listing 3 / Eq. (ed2el).  0-based outputs:
    ed2el[e] = [initial node, end node, T+, T- (-1 on the boundary)],
    led/ledTN = local edge index (0, 1, 2 for E1, E2, E3) in T+ / T-,
    t2e[m, k] = edge opposite local vertex k of element m, sigma[m, k] = +1 if
    m is T+ of that edge else -1."""
    tri = np.asarray(tri, dtype=np.int64)
    nT = tri.shape[0]
    n2el = nodes2element(tri, nV)
    n2ed, row, col = nodes2edge(n2el)
    nE = row.size
    # directed edges in the element-major order of Inode/Enode (Listing 3)
    Inode = tri.ravel()
    Enode = tri[:, [1, 2, 0]].ravel()
    p2 = _lookup(n2ed, Inode, Enode) - 1
    occ = np.arange(3 * nT)
    first = np.full(nE, 3 * nT, dtype=np.int64)
    np.minimum.at(first, p2, occ)
    ed2el = np.empty((nE, 4), dtype=np.int64)
    ed2el[:, 0] = Inode[first]
    ed2el[:, 1] = Enode[first]
    ed2el[:, 2] = first // 3
    # T- is the element owning the reverse directed edge (4th column of Q)
    ed2el[:, 3] = _lookup(n2el, Enode[first], Inode[first]) - 1
    localE = np.tile(np.array([2, 0, 1]), nT)  # P1P2 -> E3, P2P3 -> E1, P3P1 -> E2
    led = localE[first]
    ledTN = led.copy()
    last = np.full(nE, -1, dtype=np.int64)
    np.maximum.at(last, p2, occ)
    inter = ed2el[:, 3] >= 0
    ledTN[inter] = localE[last[inter]]
    count = np.bincount(p2, minlength=nE)
    if count.max(initial=0) > 2:
        raise ValueError("an edge belongs to more than two elements")
    t2e = np.empty((nT, 3), dtype=np.int64)
    t2e[occ // 3, localE] = p2
    sigma = np.where(ed2el[t2e, 2] == np.arange(nT)[:, None], 1, -1).astype(np.int64)
    return dict(n2el=n2el, n2ed=n2ed, ed2el=ed2el, led=led, ledTN=ledTN, t2e=t2e,
                sigma=sigma, nE=nE, intE=np.flatnonzero(inter), extE=np.flatnonzero(~inter))


def boundary_sets(topo: dict, dirichlet: np.ndarray, neumann: np.ndarray) -> dict:
    """Dbed, Nbed (edge numbers of the listed boundary pairs, Main.m), Redges =
    all edges except Neumann ones in increasing order (the multiplier index set
    E_Omega u E_D), and the free edges (all but Dirichlet) of the condensed
    system, also increasing."""
    n2ed = topo["n2ed"]
    nE = topo["nE"]
    d = np.asarray(dirichlet, dtype=np.int64).reshape(-1, 2)
    n = np.asarray(neumann, dtype=np.int64).reshape(-1, 2)
    Dbed = _lookup(n2ed, d[:, 0], d[:, 1]) - 1
    Nbed = _lookup(n2ed, n[:, 0], n[:, 1]) - 1
    if (Dbed < 0).any() or (Nbed < 0).any():
        raise ValueError("a listed boundary pair is not an edge")
    ext = set(topo["extE"].tolist())
    if not set(Dbed.tolist()) <= ext or not set(Nbed.tolist()) <= ext:
        raise ValueError("a listed boundary pair is an interior edge")
    if set(Dbed.tolist()) & set(Nbed.tolist()):
        raise ValueError("an edge is both Dirichlet and Neumann")
    if len(set(Dbed.tolist()) | set(Nbed.tolist())) != len(ext):
        raise ValueError("a boundary edge is neither Dirichlet nor Neumann")
    isN = np.zeros(nE, dtype=bool)
    isN[Nbed] = True
    isD = np.zeros(nE, dtype=bool)
    isD[Dbed] = True
    Redges = np.flatnonzero(~isN)
    free = np.flatnonzero(~isD)
    lam_id = -np.ones(nE, dtype=np.int64)
    lam_id[Redges] = np.arange(Redges.size)
    free_id = -np.ones(nE, dtype=np.int64)
    free_id[free] = np.arange(free.size)
    eclass = np.zeros(nE, dtype=np.int64)  # 0 interior, 1 Dirichlet, 2 Neumann
    eclass[isD] = 1
    eclass[isN] = 2
    return dict(Dbed=Dbed, Nbed=Nbed, Redges=Redges, free=free, lam_id=lam_id,
                free_id=free_id, isD=isD, isN=isN, eclass=eclass)


def redrefine(xy: np.ndarray, tri: np.ndarray, dirichlet: np.ndarray, neumann: np.ndarray):
    """Uniform red refinement of Section 2.3 (redrefine_vec): the midpoint of
    edge e (the edge numbering of Eq. n2ed) becomes vertex nV + e at
    (initial + end) / 2; element t becomes its middle child [M1 M2 M3] (Mk the
    new vertex on the edge opposite Pk) at position t, and its corner children
    [P1 M3 M2], [P2 M1 M3], [P3 M2 M1] are appended at nT + 3t, nT + 3t + 1,
    nT + 3t + 2.  A listed boundary pair (a, b) with new vertex m becomes
    (a, m) at its own position and (m, b) at position (list length + its own)."""
    xy = np.asarray(xy, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    nV, nT = xy.shape[0], tri.shape[0]
    topo = edge_tables(tri, nV)
    ed2el, t2e, n2ed = topo["ed2el"], topo["t2e"], topo["n2ed"]
    marker = nV + np.arange(topo["nE"])
    new_xy = np.concatenate([xy, (xy[ed2el[:, 0]] + xy[ed2el[:, 1]]) / 2], axis=0)
    M1, M2, M3 = marker[t2e[:, 0]], marker[t2e[:, 1]], marker[t2e[:, 2]]
    P1, P2, P3 = tri[:, 0], tri[:, 1], tri[:, 2]
    out = np.empty((4 * nT, 3), dtype=np.int64)
    out[:nT] = np.stack([M1, M2, M3], axis=1)
    out[nT::3] = np.stack([P1, M3, M2], axis=1)
    out[nT + 1::3] = np.stack([P2, M1, M3], axis=1)
    out[nT + 2::3] = np.stack([P3, M2, M1], axis=1)

    def refine_edges(pairs):
        pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
        if pairs.shape[0] == 0:
            return pairs
        base = _lookup(n2ed, pairs[:, 0], pairs[:, 1]) - 1
        if (base < 0).any():
            raise ValueError("a listed boundary pair is not an edge")
        m = marker[base]
        return np.concatenate([np.stack([pairs[:, 0], m], axis=1), np.stack([m, pairs[:, 1]], axis=1)], axis=0)

    return new_xy, out, refine_edges(dirichlet), refine_edges(neumann)


def cr_prolongation(xy_c, tri_c, xy_f, tri_f) -> sp.csr_matrix:
    """Prolongation of Crouzeix-Raviart functions (values at edge midpoints)
    from a mesh to its red refinement (redrefine): the coarse function
    v = sum_k v_{E_k} (1 - 2 lambda_k) on each coarse triangle, evaluated at
    every fine edge midpoint, and averaged over the (one or two) coarse
    triangles whose closure holds that midpoint.  Fine vertex nV_c + E is the
    midpoint of coarse edge E.  Returns the (nE_f x nE_c) matrix."""
    xy_c = np.asarray(xy_c, dtype=np.float64)
    xy_f = np.asarray(xy_f, dtype=np.float64)
    tri_c = np.asarray(tri_c, dtype=np.int64)
    nVc = xy_c.shape[0]
    tc = edge_tables(tri_c, nVc)
    tf = edge_tables(np.asarray(tri_f, dtype=np.int64), xy_f.shape[0])
    t2e_c, ed2el_c = tc["t2e"], tc["ed2el"]
    # coarse triangle holding each pair of its edges
    owner = {}
    for t in range(tri_c.shape[0]):
        for k in range(3):
            a, b = t2e_c[t, (k + 1) % 3], t2e_c[t, (k + 2) % 3]
            owner[(min(a, b), max(a, b))] = t
    rows, cols, vals = [], [], []
    for f in range(tf["nE"]):
        a, b = tf["ed2el"][f, 0], tf["ed2el"][f, 1]
        x = 0.5 * (xy_f[a] + xy_f[b])
        if a >= nVc and b >= nVc:       # inside one coarse triangle
            e1, e2 = a - nVc, b - nVc
            tris = [owner[(min(e1, e2), max(e1, e2))]]
        else:                           # half of a coarse edge
            E = max(a, b) - nVc
            tris = [t for t in ed2el_c[E, 2:4] if t >= 0]
        for t in tris:
            P = xy_c[tri_c[t]]
            # barycentric coordinates of x in t
            Tm = np.array([[P[1, 0] - P[0, 0], P[2, 0] - P[0, 0]], [P[1, 1] - P[0, 1], P[2, 1] - P[0, 1]]])
            l12 = np.linalg.solve(Tm, x - P[0])
            lam = np.array([1.0 - l12[0] - l12[1], l12[0], l12[1]])
            for k in range(3):
                rows.append(f)
                cols.append(t2e_c[t, k])
                vals.append((1.0 - 2.0 * lam[k]) / len(tris))
    return sp.coo_matrix((vals, (rows, cols)), shape=(tf["nE"], tc["nE"])).tocsr()


# ---------------------------------------------------------------------------
# Geometry and local matrices: Definition 3.1
# ---------------------------------------------------------------------------

def element_geometry(xy: np.ndarray, tri: np.ndarray) -> dict:
    """Barycentric coordinates from their definition (lambda_i affine with
    lambda_i(P_j) = delta_ij, i.e. the inverse of [1 x y] at the vertices),
    area |T|, edge lengths |E_k| and edge midpoints m_{E_k}."""
    P = xy[tri]                                   # (nT, 3, 2)
    V = np.concatenate([np.ones(P.shape[:2] + (1,)), P], axis=2)   # rows [1, x_j, y_j]
    coef = np.linalg.inv(V)                       # column i: coefficients of lambda_i
    grads = np.transpose(coef[:, 1:, :], (0, 2, 1))  # (nT, 3, 2): grad lambda_i
    area = 0.5 * np.linalg.det(V)
    if (area <= 0).any():
        raise ValueError("triangles must be counter-clockwise and non-degenerate")
    opp = np.array([[1, 2], [2, 0], [0, 1]])      # E_k = conv{P_{k+1}, P_{k+2}}
    ends = P[:, opp, :]                           # (nT, 3, 2, 2)
    elen = np.linalg.norm(ends[:, :, 1] - ends[:, :, 0], axis=2)
    mid = 0.5 * (ends[:, :, 0] + ends[:, :, 1])   # (nT, 3, 2)
    return dict(P=P, grads=grads, area=area, elen=elen, mid=mid, coef=coef)


def local_matrices(geo: dict, aT=None, A=None, p=(0.0, 0.0), delta=0.0) -> dict:
    """Definition 3.1 with A_T = a_T * I (per element) or a constant SPD A:
    (B_T)_{ij} = |T| (A grad lambda_j).grad lambda_i,
    (D_T)_{rc} = |T|/3 p.grad lambda_c   (listing's column-constant form),
    M0_T = integral of lambda_i lambda_j = |T|/12 (I + J),  M_T = delta M0_T."""
    G = geo["grads"]
    area = geo["area"]
    nT = area.size
    if A is not None:
        A = np.asarray(A, dtype=np.float64)
        BT = area[:, None, None] * np.einsum("tik,kl,tjl->tij", G, A, G)
    else:
        a = np.ones(nT) if aT is None else np.broadcast_to(np.asarray(aT, dtype=np.float64), (nT,))
        BT = (area * a)[:, None, None] * np.einsum("tik,tjk->tij", G, G)
    pv = np.asarray(p, dtype=np.float64)
    pg = np.einsum("tck,k->tc", G, pv)            # p . grad lambda_c
    DT = (area / 3.0)[:, None, None] * np.broadcast_to(pg[:, None, :], (nT, 3, 3))
    M0 = (area / 12.0)[:, None, None] * (np.eye(3) + np.ones((3, 3)))[None]
    return dict(B=BT, D=DT, M0=M0, M=delta * M0)


def local_C(geo: dict, sigma: np.ndarray) -> np.ndarray:
    """C_T row k = sigma_k |E_k| R_k (Definition 3.1)."""
    return (sigma * geo["elen"])[:, :, None] * R[None, :, :]


def _eval_g(g, x, y, nx, ny, t=None):
    return g(x, y, nx, ny) if t is None else g(x, y, nx, ny, t)


def _eval(fn, x, y, t=None):
    return fn(x, y) if t is None else fn(x, y, t)


def edge_midpoints(xy: np.ndarray, ed2el: np.ndarray):
    a = xy[ed2el[:, 0]]
    b = xy[ed2el[:, 1]]
    mid = 0.5 * (a + b)
    d = b - a
    L = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
    # initial -> end is counter-clockwise in T+, so (dy, -dx)/|E| points out of T+
    nrm = np.stack([d[:, 1], -d[:, 0]], axis=1) / L[:, None]
    return mid, L, nrm


def load_vectors(xy, tri, topo, bsets, geo, f, g, uD, t=None) -> dict:
    """Eq. (right_b): b_j = sum_T |T|/3 sum_i f(m_{E_i}) phi_j(m_{E_i});
    Eq. (right_g): LN_j = sum_{E in E_N} |E| g(m_E) phi_j(m_E) on T+ of E;
    Eq. (DirichletEqn): b_D,l = -|E_l| u_D(m_{E_l}) on Dirichlet rows of Lambda."""
    nT = tri.shape[0]
    mid = geo["mid"]
    fm = _eval(f, mid[..., 0], mid[..., 1], t)             # (nT, 3): f(m_{E_i})
    bT = (geo["area"] / 3.0)[:, None] * (fm @ R)           # sum_i f_i R_i[j]
    b = bT.reshape(3 * nT)
    ed2el = topo["ed2el"]
    emid, elen, enrm = edge_midpoints(xy, ed2el)
    LN = np.zeros(3 * nT)
    for e in bsets["Nbed"]:
        m, k = ed2el[e, 2], topo["led"][e]
        gv = _eval_g(g, emid[e, 0], emid[e, 1], enrm[e, 0], enrm[e, 1], t)
        LN[3 * m:3 * m + 3] += elen[e] * gv * R[k]
    L = bsets["Redges"].size
    bD = np.zeros(L)
    Db = bsets["Dbed"]
    bD[bsets["lam_id"][Db]] = -elen[Db] * _eval(uD, emid[Db, 0], emid[Db, 1], t)
    return dict(b=b, LN=LN, bD=bD, bT=bT)


def global_blocks(tri, topo, bsets, geo, loc) -> dict:
    """Global B, D, M, M0 (block diagonal over the element-major DOFs 3m+j,
    rho/theta index vectors of Listing 5) and C (L x N) of Listing 6."""
    nT = tri.shape[0]
    N = 3 * nT
    r = (3 * np.arange(nT))[:, None, None] + np.arange(3)[None, :, None]
    c = (3 * np.arange(nT))[:, None, None] + np.arange(3)[None, None, :]
    rr = np.broadcast_to(r, (nT, 3, 3)).ravel()
    cc = np.broadcast_to(c, (nT, 3, 3)).ravel()

    def blk(vals):
        return sp.csr_matrix((vals.ravel(), (rr, cc)), shape=(N, N))

    ed2el = topo["ed2el"]
    Redges = bsets["Redges"]
    rows, cols, vals = [], [], []
    elen = np.empty(topo["nE"])
    elen[topo["t2e"].ravel()] = geo["elen"].ravel()
    for l, e in enumerate(Redges):
        Tp, kp = ed2el[e, 2], topo["led"][e]
        rows += [l] * 3
        cols += list(3 * Tp + np.arange(3))
        vals += list(elen[e] * R[kp])
        Tm = ed2el[e, 3]
        if Tm >= 0:
            km = topo["ledTN"][e]
            rows += [l] * 3
            cols += list(3 * Tm + np.arange(3))
            vals += list(-elen[e] * R[km])
    C = sp.csr_matrix((vals, (rows, cols)), shape=(Redges.size, N))
    return dict(B=blk(loc["B"]), D=blk(loc["D"]), M=blk(loc["M"]), M0=blk(loc["M0"]), C=C)


# ---------------------------------------------------------------------------
# Elliptic problem: the saddle-point system of Section 3.5 and its solve
# ---------------------------------------------------------------------------

def setup(mesh, problem=None, aT=None, A=None):
    """Topology, boundary sets, geometry and local matrices of a mesh."""
    xy = np.asarray(mesh.xy, dtype=np.float64)
    tri = np.asarray(mesh.tri, dtype=np.int64)
    topo = edge_tables(tri, xy.shape[0])
    bsets = boundary_sets(topo, mesh.dirichlet, mesh.neumann)
    geo = element_geometry(xy, tri)
    p = (0.0, 0.0) if problem is None else problem.p
    delta = 0.0 if problem is None else problem.delta
    if A is None and problem is not None and problem.A is not None:
        A = problem.A
    loc = local_matrices(geo, aT=aT, A=A, p=p, delta=delta)
    return dict(xy=xy, tri=tri, topo=topo, bsets=bsets, geo=geo, loc=loc)


def saddle_system(st, problem, t=None):
    """Mvec = [B + D + M, -C'; -C, 0] and Fvec = [b + LN; b_D] (Section 3.5)."""
    glob = global_blocks(st["tri"], st["topo"], st["bsets"], st["geo"], st["loc"])
    lv = load_vectors(st["xy"], st["tri"], st["topo"], st["bsets"], st["geo"],
                      problem.f, problem.g, problem.uD, t)
    K = glob["B"] + glob["D"] + glob["M"]
    C = glob["C"]
    L = C.shape[0]
    Mvec = sp.bmat([[K, -C.T], [-C, sp.csr_matrix((L, L))]], format="csc")
    Fvec = np.concatenate([lv["b"] + lv["LN"], lv["bD"]])
    return Mvec, Fvec, glob, lv


def solve_saddle(mesh, problem, aT=None, A=None, return_all=False):
    """Wvec = Mvec \\ Fvec with a sparse direct solver (the paper's Main.m).
    Returns U (3 nT, element-major) and Lambda (in Redges order)."""
    st = setup(mesh, problem, aT=aT, A=A)
    Mvec, Fvec, glob, lv = saddle_system(st, problem)
    W = spla.spsolve(Mvec, Fvec)
    N = 3 * st["tri"].shape[0]
    out = dict(U=W[:N], Lambda=W[N:], st=st)
    if return_all:
        out.update(Mvec=Mvec, Fvec=Fvec, glob=glob, lv=lv)
    return out


# ---------------------------------------------------------------------------
# Condensed edge system (trace / Crouzeix-Raviart form)
# ---------------------------------------------------------------------------

def condensed_local(st, lv=None):
    """K^CR_T = R^{-T} K_T R^{-1} and F^CR_T = R^{-T} F_T with K_T = B_T + D_T + M_T
    and F_T = b_T + LN_T: substituting u_T = R^{-1} w_T (w_T = the values at the
    three edge midpoints) into the element rows of the saddle system and
    multiplying by R^{-T} turns the multiplier term into -diag(sigma |E|) Lambda_T,
    which cancels between T+ and T- on interior edges."""
    loc = st["loc"]
    Rinv = np.linalg.inv(R)
    KT = loc["B"] + loc["D"] + loc["M"]
    KCR = np.einsum("ji,tjk,kl->til", Rinv, KT, Rinv)
    out = dict(KCR=KCR, Rinv=Rinv)
    if lv is not None:
        nT = st["tri"].shape[0]
        FT = (lv["b"] + lv["LN"]).reshape(nT, 3)
        out["FCR"] = np.einsum("ji,tj->ti", Rinv, FT)
    return out


def condensed_system(mesh, problem, aT=None, A=None, st=None):
    """Assemble the condensed SPD system over the free edges (interior and
    Neumann), ordered by increasing edge number: S w_f = rhs with
    rhs = F^CR_f - S_fd u_D(m_d).  Every element adds its 3x3 block K^CR_T to
    the (free, free) pairs of its edges; duplicates are summed and every
    structural entry is kept (also exact zeros), columns sorted (CSR)."""
    if st is None:
        st = setup(mesh, problem, aT=aT, A=A)
    lv = load_vectors(st["xy"], st["tri"], st["topo"], st["bsets"], st["geo"],
                      problem.f, problem.g, problem.uD)
    cl = condensed_local(st, lv)
    t2e = st["topo"]["t2e"]
    free_id = st["bsets"]["free_id"]
    nE = st["topo"]["nE"]
    emid, elen, enrm = edge_midpoints(st["xy"], st["topo"]["ed2el"])
    wD = np.zeros(nE)
    Db = st["bsets"]["Dbed"]
    wD[Db] = problem.uD(emid[Db, 0], emid[Db, 1])
    nF = st["bsets"]["free"].size
    KCR, FCR = cl["KCR"], cl["FCR"]
    fi = free_id[t2e]                                   # (nT, 3)
    rows = np.broadcast_to(fi[:, :, None], KCR.shape)
    cols = np.broadcast_to(fi[:, None, :], KCR.shape)
    keep = (rows >= 0) & (cols >= 0)
    S = sp.coo_matrix((KCR[keep], (rows[keep], cols[keep])), shape=(nF, nF)).tocsr()
    S.sort_indices()
    # lifting of the Dirichlet values and the element loads
    lift = np.einsum("tij,tj->ti", KCR, np.where(fi < 0, wD[t2e], 0.0))
    contrib = FCR - lift
    rhs = np.zeros(nF)
    ok = fi >= 0
    np.add.at(rhs, fi[ok], contrib[ok])
    return dict(S=S, rhs=rhs, row_ptr=S.indptr.astype(np.int64), col=S.indices.astype(np.int64),
                val=S.data.copy(), wD=wD, st=st, lv=lv, cl=cl)


def recover(st, cl, w_all, lv=None):
    """U and Lambda from the edge-midpoint values w (all edges, Dirichlet ones
    set to u_D): u_T = R^{-1} w_T, and from the element rows
    K^CR_T w_T - F^CR_T = diag(sigma |E|) Lambda_T, read on T+ (sigma = +1).
    Also returns the same quantity read on T- for interior edges, and the
    element residual on Neumann edges (which must vanish)."""
    t2e = st["topo"]["t2e"]
    sigma = st["topo"]["sigma"]
    wT = w_all[t2e]                               # (nT, 3)
    U = np.einsum("ij,tj->ti", cl["Rinv"], wT).reshape(-1)
    res = np.einsum("tij,tj->ti", cl["KCR"], wT) - cl["FCR"]
    lam_id = st["bsets"]["lam_id"]
    L = st["bsets"]["Redges"].size
    val = res / (sigma * st["geo"]["elen"])
    li = lam_id[t2e]
    Lam_plus = np.full(L, np.nan)
    Lam_minus = np.full(L, np.nan)
    plus = (li >= 0) & (sigma > 0)
    minus = (li >= 0) & (sigma < 0)
    Lam_plus[li[plus]] = val[plus]
    Lam_minus[li[minus]] = val[minus]
    return dict(U=U, Lambda=Lam_plus, Lambda_minus=Lam_minus, neumann_residual=res[li < 0])


def solve_condensed(mesh, problem, aT=None, A=None, method="direct", rtol=1e-13, maxiter=100000):
    """Condensed solve (direct, or plain Jacobi-PCG for large meshes) followed by
    the recovery of U and Lambda."""
    cs = condensed_system(mesh, problem, aT=aT, A=A)
    if method == "direct":
        wf = spla.spsolve(cs["S"].tocsc(), cs["rhs"])
        info = dict(iterations=0)
    else:
        wf, info = pcg(cs["S"], cs["rhs"], rtol=rtol, maxiter=maxiter)
    w = cs["wD"].copy()
    w[cs["st"]["bsets"]["free"]] = wf
    rec = recover(cs["st"], cs["cl"], w)
    rec.update(w=w, wf=wf, info=info, cs=cs)
    return rec


def flux_system(mesh, problem, aT=None, A=None):
    """Multiplier ("flux") Schur complement of the saddle system of Section 3.5:
    the element rows K U - C' Lambda = F give U = K^{-1} (F + C' Lambda), and the
    constraint rows -C U = b_D then read
        (C K^{-1} C') Lambda = -b_D - C K^{-1} F.
    K = B + D + M is block diagonal over the elements; each 3x3 block is
    inverted on its own (it is invertible only when the reaction delta > 0).
    Rows and columns are the multipliers in Redges order (interior and
    Dirichlet edges)."""
    st = setup(mesh, problem, aT=aT, A=A)
    glob = global_blocks(st["tri"], st["topo"], st["bsets"], st["geo"], st["loc"])
    lv = load_vectors(st["xy"], st["tri"], st["topo"], st["bsets"], st["geo"],
                      problem.f, problem.g, problem.uD)
    loc = st["loc"]
    KT = loc["B"] + loc["D"] + loc["M"]
    nT = KT.shape[0]
    Kinv_T = np.linalg.inv(KT)                    # raises on a singular block
    r = (3 * np.arange(nT))[:, None, None] + np.arange(3)[None, :, None]
    c = (3 * np.arange(nT))[:, None, None] + np.arange(3)[None, None, :]
    Kinv = sp.csr_matrix((Kinv_T.ravel(), (np.broadcast_to(r, (nT, 3, 3)).ravel(),
                                           np.broadcast_to(c, (nT, 3, 3)).ravel())),
                         shape=(3 * nT, 3 * nT))
    C = glob["C"].tocsr()
    F = lv["b"] + lv["LN"]
    S = (C @ Kinv @ C.T).tocsr()
    rhs = -lv["bD"] - C @ (Kinv @ F)
    return dict(S=S, rhs=rhs, Kinv=Kinv, C=C, F=F, st=st)


def flux_recover(fs, Lambda):
    """U = K^{-1} (F + C' Lambda) (the element rows of Section 3.5)."""
    return fs["Kinv"] @ (fs["F"] + fs["C"].T @ Lambda)


def relative_residual(S, b, x) -> float:
    """||b - S x||_2 / ||b||_2 of the condensed free-edge system, evaluated in
    difference form r_i = b_i - sum_j S_ij (x_j - x_i) - (sum_j S_ij) x_i.
    Differences of neighbouring values are exact or nearly so, which keeps the
    FP64 evaluation accurate where the plain row product loses about 1/h^2
    digits to cancellation (the reading of the "1e-10 relative residual"
    criterion: the residual of the FP64 matrix, evaluated accurately)."""
    S = S.tocsr()
    row = np.repeat(np.arange(S.shape[0]), np.diff(S.indptr))
    terms = S.data * (x[S.indices] - x[row])
    Sx = np.bincount(row, weights=terms, minlength=S.shape[0])
    rowsum = np.bincount(row, weights=S.data, minlength=S.shape[0])
    r = b - (Sx + rowsum * x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def pcg(S, b, rtol=1e-13, maxiter=100000, x0=None):
    """Plain Jacobi-preconditioned conjugate gradients in FP64 (Hestenes-Stiefel
    recurrences), stopped on ||b - S x||_2 <= rtol ||b||_2 of the recursive
    residual."""
    d = S.diagonal()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - S @ x
    z = r / d
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    it = 0
    while np.linalg.norm(r) > rtol * nb and it < maxiter:
        q = S @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = r / d
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, dict(iterations=it, rel_residual=np.linalg.norm(b - S @ x) / nb)


# ---------------------------------------------------------------------------
# Crank-Nicolson (Section 4)
# ---------------------------------------------------------------------------

def cn_solve(mesh, problem, k, nsteps, aT=None, A=None, Lambda0=None, keep_history=False):
    """M+ W^n = M- W^{n-1} + F (Eq. MatrixformParabolic) with
    M+- = [(1 +- k delta/2) M0 +- k/2 B +- k/2 D, -+ k/2 C'; -+ 1/2 C, 0],
    F = [k (F^n + F^{n-1})/2 ; (b_D^n + b_D^{n-1})/2], t_n = n k.
    U^0 = R^{-1}[u0(m_{E_k})] per element; Lambda^0 = given or 0.
    Returns U^n, Lambda^n and Lambda^{n-1/2} = (Lambda^n + Lambda^{n-1})/2."""
    st = setup(mesh, problem, aT=aT, A=A)
    glob = global_blocks(st["tri"], st["topo"], st["bsets"], st["geo"], st["loc"])
    delta = problem.delta
    M0, B, D, C = glob["M0"], glob["B"], glob["D"], glob["C"]
    L = C.shape[0]
    Z = sp.csr_matrix((L, L))
    Mp = sp.bmat([[(1 + 0.5 * k * delta) * M0 + 0.5 * k * B + 0.5 * k * D, -0.5 * k * C.T],
                  [-0.5 * C, Z]], format="csc")
    Mm = sp.bmat([[(1 - 0.5 * k * delta) * M0 - 0.5 * k * B - 0.5 * k * D, 0.5 * k * C.T],
                  [0.5 * C, Z]], format="csr")
    lu = spla.splu(Mp)

    def forcing(t):
        lv = load_vectors(st["xy"], st["tri"], st["topo"], st["bsets"], st["geo"],
                          problem.f, problem.g, problem.uD, t)
        return lv["b"] + lv["LN"], lv["bD"]

    mid = st["geo"]["mid"]
    u0m = problem.u0(mid[..., 0], mid[..., 1])            # (nT, 3): u0(m_{E_k})
    U0 = (u0m @ np.linalg.inv(R).T).reshape(-1)
    Lam = np.zeros(L) if Lambda0 is None else np.asarray(Lambda0, dtype=np.float64).copy()
    W = np.concatenate([U0, Lam])
    N = U0.size
    Fprev, bDprev = forcing(0.0)
    hist = []
    lam_half = np.zeros(L)
    for n in range(1, nsteps + 1):
        Fn, bDn = forcing(n * k)
        rhs = Mm @ W + np.concatenate([k * 0.5 * (Fn + Fprev), 0.5 * (bDn + bDprev)])
        Wn = lu.solve(rhs)
        lam_half = 0.5 * (Wn[N:] + W[N:])
        W = Wn
        Fprev, bDprev = Fn, bDn
        if keep_history:
            hist.append(W.copy())
    return dict(U=W[:N], Lambda=W[N:], Lambda_half=lam_half, st=st, history=hist, U0=U0)


# ---------------------------------------------------------------------------
# Errors (the paper's PHerror is not printed; these follow Section 3.1's norms)
# ---------------------------------------------------------------------------

def _gauss_legendre01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def errors(st, U, u, grad, t=None, nq=6) -> dict:
    """||u - u_h||_{L2}, broken ||grad_h(u - u_h)||_{L2} and the full broken H1
    norm, by a Duffy-collapsed nq x nq Gauss-Legendre rule on every triangle."""
    P = st["geo"]["P"]
    G = st["geo"]["grads"]
    area = st["geo"]["area"]
    Ue = np.asarray(U).reshape(-1, 3)
    xi, wi = _gauss_legendre01(nq)
    s = xi[:, None] * np.ones(nq)[None, :]
    tt = xi[None, :] * (1.0 - xi[:, None])
    w = (wi[:, None] * wi[None, :]) * (1.0 - xi[:, None])
    s, tt, w = s.ravel(), tt.ravel(), w.ravel()
    lam = np.stack([1.0 - s - tt, s, tt], axis=1)           # (q, 3)
    X = np.einsum("qj,tjk->tqk", lam, P)                     # (nT, q, 2)
    uh = np.einsum("qj,tj->tq", lam, Ue)
    guh = np.einsum("tj,tjk->tk", Ue, G)                     # constant per element
    ue = u(X[..., 0], X[..., 1]) if t is None else u(X[..., 0], X[..., 1], t)
    gx, gy = grad(X[..., 0], X[..., 1]) if t is None else grad(X[..., 0], X[..., 1], t)
    jac = 2.0 * area
    l2 = np.sum(jac[:, None] * w[None, :] * (ue - uh) ** 2)
    h1s = np.sum(jac[:, None] * w[None, :] * ((gx - guh[:, None, 0]) ** 2 + (gy - guh[:, None, 1]) ** 2))
    return dict(L2=np.sqrt(l2), H1semi=np.sqrt(h1s), H1=np.sqrt(l2 + h1s))


def exact_flux(st, grad, t=None, A=None, a=None):
    """kappa = (A grad u).nu_E at the midpoints of the multiplier edges (Redges
    order), nu_E the outward normal of T+ (Eq. exactLagrange).  With the
    listing's convection form (test function on the row) the convective term
    is not integrated by parts, so u p does not enter the multiplier."""
    Redges = st["bsets"]["Redges"]
    emid, elen, enrm = edge_midpoints(st["xy"], st["topo"]["ed2el"])
    return _flux(grad, emid[Redges], enrm[Redges], t, A, a)


def _flux(grad, X, nrm, t=None, A=None, a=None):
    x, y = X[..., 0], X[..., 1]
    gx, gy = grad(x, y) if t is None else grad(x, y, t)
    if A is not None:
        gx, gy = A[0, 0] * gx + A[0, 1] * gy, A[1, 0] * gx + A[1, 1] * gy
    if a is not None:
        av = a(x, y)
        gx, gy = av * gx, av * gy
    return gx * nrm[..., 0] + gy * nrm[..., 1]


def m_norm_error(st, Lambda, grad, t=None, A=None, nq=6) -> float:
    """Mesh M-norm of kappa - kappa_h (the paper does not print PHerror):
    sqrt(sum over multiplier edges E of |E| * int_E (kappa - Lambda_E)^2), the
    edge integral by nq-point Gauss-Legendre; it decreases like h.  Pinned by
    hand-worked values on the two-triangle square (constant offsets, a flux
    linear along an edge, Neumann edges left out), not by the paper's column."""
    Redges = st["bsets"]["Redges"]
    ed2el = st["topo"]["ed2el"]
    a = st["xy"][ed2el[Redges, 0]]
    b = st["xy"][ed2el[Redges, 1]]
    d = b - a
    Ln = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
    nrm = np.stack([d[:, 1], -d[:, 0]], axis=1) / Ln[:, None]
    xg, wg = _gauss_legendre01(nq)
    X = a[:, None, :] + xg[None, :, None] * d[:, None, :]
    kap = _flux(grad, X, nrm[:, None, :], t, A)
    e2 = ((kap - np.asarray(Lambda)[:, None]) ** 2 * wg[None, :]).sum(axis=1) * Ln
    return float(np.sqrt(np.sum(Ln * e2)))


def mesh_h(st) -> float:
    """h of Main.m: sqrt(2 det[1 1 1; P]) of the first element = 2 sqrt(|T_1|)."""
    return float(2.0 * np.sqrt(st["geo"]["area"][0]))
