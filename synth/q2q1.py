"""Seeded synthetic Q2-Q1 (Taylor-Hood) Stokes / Oseen systems on uniform meshes.

This module produces the INPUTS of the solver: the discrete block system of
Section 2 (eq. stokes_block_system for Stokes, eq. ns_block_system for the
Oseen linearisation), node coordinates, the pressure-to-velocity co-location
map and seeded right-hand sides.  It holds no arithmetic of the multigrid
method itself; the CUDA path and the oracle both receive what it returns.

Definitions (Section 2.1 and 2.2):
  * velocity: biquadratic (triquadratic) nodal basis phi_i on a uniform n^d
    element mesh, (2n+1)^d nodes; pressure: bilinear (trilinear) psi_k,
    (n+1)^d nodes, sitting at the element vertices (Fig. 1), so every pressure
    node is co-located with a velocity node.
  * A_hat[i, j] = int grad(phi_i) . grad(phi_j)                (Section 2.1)
  * K_hat[i, j] = int (w . grad(phi_j)) phi_i                   (Section 2.2)
    and the Oseen velocity block is nu * A_hat + K_hat.
  * B = [B_x  B_y (B_z)], B_c[k, i] = - int psi_k d(phi_i)/dx_c.
    The paper writes B with a plus sign, which with its weak form gives
    [A -B^T; B 0]; the minus sign used here gives the symmetric [A B^T; B 0]
    of eq. stokes_block_system (the negated continuity row has a zero RHS).
  * Numbering: lexicographic from the lower-left corner, x fastest (the
    "natural ordering" of Section 6.1); dofs ordered [u_x | u_y (| u_z) | p].
  * Integrals use the 3-point Gauss rule per direction, exact for A_hat, B
    and for K_hat with a polynomial wind of degree <= 2 per direction.
  * Dirichlet velocity on every boundary node (all components); values are
    lifted into the RHS, Dirichlet rows become identity rows and Dirichlet
    columns are zeroed, so A_hat stays shared by all components.
  * Optional pinned pressure node: its B row is zeroed, its (2,2) diagonal
    entry is 1 and its RHS is 0.  Without a pin the pressure is determined up
    to a constant (Section 2.1) and b_p is projected to zero mean.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from .rng import uniform_pm1

# 1D reference basis on s in [0, 1]
_GAUSS_S = np.array([0.5 - np.sqrt(0.15), 0.5, 0.5 + np.sqrt(0.15)])
_GAUSS_W = np.array([5.0, 8.0, 5.0]) / 18.0


def _q2(s):
    return np.array([2 * s * s - 3 * s + 1, 4 * s - 4 * s * s, 2 * s * s - s])


def _dq2(s):
    return np.array([4 * s - 3, 4 - 8 * s, 4 * s - 1])


def _q1(s):
    return np.array([1 - s, s])


@dataclasses.dataclass
class Problem:
    dim: int
    n: int
    n_v: int               # velocity nodes (per component)
    n_p: int               # pressure nodes
    A: sp.csr_matrix       # scalar velocity block (n_v x n_v), shared by components
    B: sp.csr_matrix       # divergence block (n_p x dim*n_v), component-major columns
    vcoords: np.ndarray    # (n_v, dim)
    pcoords: np.ndarray    # (n_p, dim)
    p2v: np.ndarray        # (n_p,) velocity node co-located with each pressure node
    v_dirichlet: np.ndarray  # (n_v,) bool
    pinned: int            # pinned pressure node, -1 if none
    symmetric: bool
    b: np.ndarray          # (N, nrhs) right-hand sides, N = dim*n_v + n_p
    name: str = ""

    @property
    def N(self) -> int:
        return self.dim * self.n_v + self.n_p

    def full_matrix(self) -> sp.csr_matrix:
        """The whole block matrix [I_d (x) A, B^T; B, C] (C = pin diagonal)."""
        Av = sp.kron(sp.identity(self.dim, format="csr"), self.A, format="csr")
        C = sp.csr_matrix((self.n_p, self.n_p))
        if self.pinned >= 0:
            C = sp.csr_matrix(([1.0], ([self.pinned], [self.pinned])), shape=(self.n_p, self.n_p))
        return sp.bmat([[Av, self.B.T], [self.B, C]], format="csr")


def _canonical(M) -> sp.csr_matrix:
    M = sp.csr_matrix(M)
    M.sum_duplicates()
    M.eliminate_zeros()
    M.sort_indices()
    M.indices = M.indices.astype(np.int32)
    M.indptr = M.indptr.astype(np.int32) if M.nnz < 2**31 - 1 else M.indptr
    return M


def _reference_tables(dim):
    """Basis values/gradients at the 3^dim Gauss points of the unit element."""
    nq1 = 3
    Q = nq1 ** dim
    nv_loc, np_loc = 3 ** dim, 2 ** dim
    phi = np.ones((Q, nv_loc))
    dphi = np.ones((Q, dim, nv_loc))   # d/ds_k on the unit element
    psi = np.ones((Q, np_loc))
    wq = np.ones(Q)
    spts = np.zeros((Q, dim))
    for q in range(Q):
        qi = [(q // nq1 ** k) % nq1 for k in range(dim)]
        for k in range(dim):
            s = _GAUSS_S[qi[k]]
            spts[q, k] = s
            wq[q] *= _GAUSS_W[qi[k]]
        for a in range(nv_loc):
            ai = [(a // 3 ** k) % 3 for k in range(dim)]
            for k in range(dim):
                phi[q, a] *= _q2(spts[q, k])[ai[k]]
            for kd in range(dim):
                for k in range(dim):
                    f = _dq2(spts[q, k])[ai[k]] if k == kd else _q2(spts[q, k])[ai[k]]
                    dphi[q, kd, a] *= f
        for b in range(np_loc):
            bi = [(b // 2 ** k) % 2 for k in range(dim)]
            for k in range(dim):
                psi[q, b] *= _q1(spts[q, k])[bi[k]]
    return phi, dphi, psi, wq, spts


def element_matrices(dim: int, h: float):
    """Element stiffness (3^d x 3^d) and divergence blocks (d x 2^d x 3^d) on a cube of side h."""
    phi, dphi, psi, wq, _ = _reference_tables(dim)
    W = wq * h ** dim
    g = dphi / h
    Ae = np.einsum("q,qki,qkj->ij", W, g, g)
    Be = -np.einsum("q,qp,qki->kpi", W, psi, g)
    return Ae, Be


def _element_nodes(n, dim):
    """Global velocity/pressure node ids per element, (E, 3^d) and (E, 2^d)."""
    nv1, np1 = 2 * n + 1, n + 1
    E = n ** dim
    e = np.arange(E)
    emi = [(e // n ** k) % n for k in range(dim)]
    vloc = np.zeros((E, 3 ** dim), dtype=np.int64)
    for a in range(3 ** dim):
        ai = [(a // 3 ** k) % 3 for k in range(dim)]
        vloc[:, a] = sum((2 * emi[k] + ai[k]) * nv1 ** k for k in range(dim))
    ploc = np.zeros((E, 2 ** dim), dtype=np.int64)
    for b in range(2 ** dim):
        bi = [(b // 2 ** k) % 2 for k in range(dim)]
        ploc[:, b] = sum((emi[k] + bi[k]) * np1 ** k for k in range(dim))
    return vloc, ploc, emi


def mass_matrices(n: int, dim: int = 2, lo: float = 0.0, hi: float = 1.0):
    """Q2 velocity mass matrix (one component, n_v x n_v) and Q1 pressure mass matrix
    (n_p x n_p) on the uniform n^dim mesh: integrals of products of basis functions,
    exact with the 3-point Gauss rule."""
    h = (hi - lo) / n
    phi, _, psi, wq, _ = _reference_tables(dim)
    W = wq * h ** dim
    Mv_e = np.einsum("q,qi,qj->ij", W, phi, phi)
    Mp_e = np.einsum("q,qi,qj->ij", W, psi, psi)
    vloc, ploc, _ = _element_nodes(n, dim)
    n_v, n_p = (2 * n + 1) ** dim, (n + 1) ** dim
    def build(loc, Me, size):
        k = loc.shape[1]
        r = np.repeat(loc, k, axis=1).ravel()
        c = np.tile(loc, (1, k)).ravel()
        v = np.tile(Me.ravel(), loc.shape[0])
        return sp.csr_matrix((v, (r, c)), shape=(size, size))
    return build(vloc, Mv_e, n_v), build(ploc, Mp_e, n_p)


def _grid_coords(m, dim, lo, hi):
    """Coordinates of an m^dim lexicographic grid of nodes spanning [lo, hi]^dim."""
    i = np.arange(m ** dim)
    X = np.zeros((m ** dim, dim))
    for k in range(dim):
        X[:, k] = lo + (hi - lo) * ((i // m ** k) % m) / (m - 1)
    return X


def recirculating_wind(x):
    """w = (2y(1-x^2), -2x(1-y^2)): divergence free, tangential on [-1,1]^2."""
    return np.stack([2 * x[..., 1] * (1 - x[..., 0] ** 2), -2 * x[..., 0] * (1 - x[..., 1] ** 2)], axis=-1)


def assemble(n: int, dim: int = 2, lo: float = 0.0, hi: float = 1.0, nu: float = 1.0, wind=None, wind_nodal=None):
    """Unconstrained velocity block (nu*A_hat [+ K_hat]) and B on the uniform n^dim mesh.
    The convection wind is a function of the point (wind) or a discrete Q2 field given by
    its nodal values, shape (dim, n_v) (wind_nodal), evaluated at the quadrature points."""
    h = (hi - lo) / n
    nv1, np1 = 2 * n + 1, n + 1
    n_v, n_p = nv1 ** dim, np1 ** dim
    vloc, ploc, emi = _element_nodes(n, dim)
    Ae, Be = element_matrices(dim, h)
    nvl, npl = vloc.shape[1], ploc.shape[1]
    rows = np.repeat(vloc, nvl, axis=1).ravel()
    cols = np.tile(vloc, (1, nvl)).ravel()
    vals = np.tile((nu * Ae).ravel(), vloc.shape[0])
    if wind is not None or wind_nodal is not None:
        phi, dphi, _, wq, spts = _reference_tables(dim)
        if wind_nodal is not None:
            wn = np.asarray(wind_nodal, dtype=np.float64).reshape(dim, n_v)
            wv = np.einsum("qa,kea->eqk", phi, wn[:, vloc])                 # (E, Q, dim)
        else:
            origin = np.stack([lo + h * emi[k] for k in range(dim)], axis=1)   # (E, dim)
            xq = origin[:, None, :] + h * spts[None, :, :]                     # (E, Q, dim)
            wv = wind(xq)                                                      # (E, Q, dim)
        Ke = np.einsum("q,qi,eqk,qkj->eij", wq * h ** dim, phi, wv, dphi / h)
        vals = vals + Ke.reshape(-1)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n_v, n_v))
    Bblocks = []
    for k in range(dim):
        r = np.repeat(ploc, nvl, axis=1).ravel()
        c = np.tile(vloc, (1, npl)).ravel()
        v = np.tile(Be[k].ravel(), vloc.shape[0])
        Bblocks.append(sp.csr_matrix((v, (r, c)), shape=(n_p, n_v)))
    B = sp.hstack(Bblocks, format="csr")
    vcoords = _grid_coords(nv1, dim, lo, hi)
    pcoords = _grid_coords(np1, dim, lo, hi)
    pmi = [(np.arange(n_p) // np1 ** k) % np1 for k in range(dim)]
    p2v = sum(2 * pmi[k] * nv1 ** k for k in range(dim)).astype(np.int32)
    vmi = [(np.arange(n_v) // nv1 ** k) % nv1 for k in range(dim)]
    bnd = np.zeros(n_v, dtype=bool)
    for k in range(dim):
        bnd |= (vmi[k] == 0) | (vmi[k] == nv1 - 1)
    top = vmi[dim - 1] == nv1 - 1
    return _canonical(A), _canonical(B), vcoords, pcoords, p2v, bnd, top


def make_problem(n: int, dim: int = 2, lo: float = 0.0, hi: float = 1.0, bc: str = "zero",
                 pin: bool = False, nu: float = 1.0, wind=None, nrhs: int = 1, seed: int = 0,
                 body: str = "uniform", name: str = "", wind_nodal=None) -> Problem:
    """Assemble, apply Dirichlet BCs / pin, and draw nrhs seeded right-hand sides.

    bc: "zero" (homogeneous Dirichlet) or "lid" (u_x = 1 on the top face
    including its edges and corners, the leaky lid of Section 6.1; every other
    boundary value 0).  body: "uniform" puts i.i.d. uniform[-1,1] draws on the
    non-Dirichlet velocity rows (RHS j drawn from splitmix64 seed 1000*seed+j,
    one draw per velocity dof in dof order); "none" is the zero body force.
    """
    A, B, vcoords, pcoords, p2v, bnd, top = assemble(n, dim, lo, hi, nu, wind, wind_nodal)
    n_v, n_p = A.shape[0], B.shape[0]
    N = dim * n_v + n_p
    g = np.zeros((dim, n_v))
    if bc == "lid":
        g[0, top] = 1.0
    elif bc != "zero":
        raise ValueError(bc)
    # lifting of the Dirichlet values into the right-hand side
    lift_u = np.stack([-(A @ g[c]) for c in range(dim)])
    lift_p = -(B @ g.reshape(-1))
    D = np.flatnonzero(bnd)
    keep = np.ones(n_v)
    keep[D] = 0.0
    Kd = sp.diags(keep)
    A = Kd @ A @ Kd + sp.diags(1.0 - keep)
    B = B @ sp.diags(np.tile(keep, dim))
    pinned = -1
    if pin:
        pinned = 0
        rk = np.ones(n_p)
        rk[pinned] = 0.0
        B = sp.diags(rk) @ B
    A, B = _canonical(A), _canonical(B)
    b = np.zeros((N, nrhs))
    for j in range(nrhs):
        bu = lift_u.copy()
        if body == "uniform":
            draws = uniform_pm1(1000 * seed + j, dim * n_v).reshape(dim, n_v)
            bu += draws
        elif body != "none":
            raise ValueError(body)
        bu[:, D] = g[:, D]
        bp = lift_p.copy()
        if pinned >= 0:
            bp[pinned] = 0.0
        else:
            bp -= bp.mean()
        b[: dim * n_v, j] = bu.reshape(-1)
        b[dim * n_v:, j] = bp
    return Problem(dim=dim, n=n, n_v=n_v, n_p=n_p, A=A, B=B, vcoords=vcoords, pcoords=pcoords,
                   p2v=p2v, v_dirichlet=bnd, pinned=pinned, symmetric=wind is None and wind_nodal is None, b=b,
                   name=name)


# ----------------------------------------------------------------------------
# The workloads, each named by what it is.

def stokes_pinned_2d(n=16, nrhs=1, seed=0):
    """Unit square, nu=1, homogeneous Dirichlet, pressure node 0 pinned, uniform body load."""
    return make_problem(n, 2, 0.0, 1.0, bc="zero", pin=True, nrhs=nrhs, seed=seed,
                        name=f"stokes2d_pinned_{n}x{n}")


def stokes_lid_2d(n=256, nrhs=8, seed=0, body="uniform", lo=0.0, hi=1.0):
    """Leaky lid-driven cavity, nu=1, pressure up to a constant, nrhs seeded body loads."""
    return make_problem(n, 2, lo, hi, bc="lid", pin=False, nrhs=nrhs, seed=seed, body=body,
                        name=f"stokes2d_lid_{n}x{n}")


def oseen_recirculating_2d(n=512, Re=10.0, nrhs=32, seed=0):
    """[-1,1]^2, recirculating wind, nu = 2/Re, homogeneous Dirichlet, seeded body loads."""
    return make_problem(n, 2, -1.0, 1.0, bc="zero", pin=False, nu=2.0 / Re,
                        wind=recirculating_wind, nrhs=nrhs, seed=seed,
                        name=f"oseen2d_Re{Re:g}_{n}x{n}")


def stokes_lid_3d(n=48, nrhs=1, seed=0):
    """Unit cube, lid (1,0,0) on z=1 including its edges, nu=1."""
    return make_problem(n, 3, 0.0, 1.0, bc="lid", pin=False, nrhs=nrhs, seed=seed,
                        name=f"stokes3d_lid_{n}^3")


def with_perturbed_coordinates(p: Problem, amplitude: float = 0.35, seed: int = 100) -> Problem:
    """The same matrices and right-hand sides with the node coordinates the
    coarsening reads (Alg. 3's distance heuristics, Alg. 4's mid-point test)
    moved by seeded uniform offsets of up to `amplitude` times the velocity node
    spacing per direction; a pressure node keeps its co-located velocity node's
    position.  On a uniform mesh Alg. 3 packs the coarse pressures perfectly and
    no F-point is badly covered; the perturbed positions change which candidate
    wins each step, so find_extra_dist3_Cpoints has F-points to convert.  Only
    the coordinate inputs change: the block system is the uniform mesh's."""
    lo, hi = float(p.vcoords.min()), float(p.vcoords.max())
    h = (hi - lo) / (2 * p.n)
    off = uniform_pm1(seed, p.n_v * p.dim).reshape(p.n_v, p.dim) * (amplitude * h)
    vX = p.vcoords + off
    return dataclasses.replace(p, vcoords=vX, pcoords=vX[p.p2v], name=p.name + f"_perturbed{seed}")
