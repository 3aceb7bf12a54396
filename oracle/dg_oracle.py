"""FP64 CPU oracle: SIPDG Poisson problems on a uniform auxiliary mesh and the
exchange matrix K built from their solutions.

TEST INFRASTRUCTURE ONLY -- never imported by the product path.

What is restated here, and from where (arXiv 2510.21213):

* Degree-q nodal Lagrange basis on the tensor Gauss-Legendre points of each
  element; the same points define the quadrature rule (Sec. 6.2, eq.
  density_approx; Sec. 6.3).
* SIPDG bilinear form, Sec. 3.4 eq. sip_bilinear: element volume gradients plus,
  on every interior face, -[[u]].{grad v} - {grad u}.[[v]] + sigma [[u]].[[v]],
  with the jump [[f]] = f^- n^- + f^+ n^+ and average {f} = (f^- + f^+)/2 of
  Sec. 3.1.
* Penalty sigma from Sec. 3.5 (eqs. Cprop, Csquared, pen_poly). The paper's units are
  inconsistent (sigma >= C^2/(eps h) with C^2 = (p+1)^2/h); form 0 reads it as
  sigma = (p+1)^2/(eps h), form 1 keeps the literal (p+1)^2/(eps h^2).
  eps = 1/8 as in Sec. 3.5.
* Poisson problem -Lap u = 4 pi f in Omega with the inhomogeneous Dirichlet
  data u(r) = int_Omega f(r')/|r - r'| dr' on the boundary, evaluated with the
  grid's Gauss quadrature (Sec. 6.3). The paper does not state the
  weak form of the Dirichlet condition; the symmetric Nitsche terms
  -u d_n v - d_n u v + sigma u v on boundary faces (and the matching load
  sigma g v - g d_n v) are used, i.e. the boundary face is treated as a face
  whose exterior trace is zero.
* Right-hand sides evaluated pointwise at the quadrature nodes (Sec. 6.1.2):
  f = psi_i psi_j for the exchange problems (eq. fock_poisson),
  f = rho = sum_k psi_k^2 for the Hartree problem (eq. hartree_poisson,
  with rho from eq. HF in Sec. 2.3.1).
* K_ij = sum_q W_q psi_i(q) sum_s psi_s(q) v_sj(q) from eq. fock_exchange
  (Sec. 6.1.2) with phi_i -> psi_i and u -> psi_j, each distinct pair
  solved once (v_sj = v_js).
* E_H = 1/2 sum_q W_q rho v_H and E_X = -1/2 tr K (HF energy, Sec. 2.3.1).

Orderings (shared with the C-ABI): elements x-fastest, e = ex + nx (ey + ny ez);
nodes inside an element lexicographic x-fastest, local = a + n1 (b + n1 c).
Boundary data of the face normal to axis d is a 2-D array indexed by the
global node indices of the two other axes in increasing axis order.

Parity: the solvers here are direct (dense Cholesky or exact fast
diagonalisation of the Kronecker-sum operator), so they give the exact
solution of the discrete problem that the multigrid-preconditioned CG of the
GPU path converges to.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.sparse

FOUR_PI = 4.0 * math.pi


# ---------------------------------------------------------------------------
# Mesh
# ---------------------------------------------------------------------------
class Mesh:
    """Uniform hexahedral box mesh with degree-p tensor GL nodal elements."""

    def __init__(self, lo, hi, n, p):
        self.lo = np.asarray(lo, dtype=np.float64).reshape(3)
        self.hi = np.asarray(hi, dtype=np.float64).reshape(3)
        if np.isscalar(n):
            n = (n, n, n)
        self.n = tuple(int(v) for v in n)
        self.p = int(p)
        self.n1 = self.p + 1
        self.h = (self.hi - self.lo) / np.asarray(self.n, dtype=np.float64)
        self.E = self.n[0] * self.n[1] * self.n[2]
        self.npe = self.n1 ** 3
        self.Nq = self.E * self.npe
        self.L = tuple(self.n[d] * self.n1 for d in range(3))

    def __repr__(self):
        return f"Mesh(lo={self.lo.tolist()}, hi={self.hi.tolist()}, n={self.n}, p={self.p})"


# ---------------------------------------------------------------------------
# 1-D ingredients
# ---------------------------------------------------------------------------
def gauss_legendre(npts):
    """Gauss-Legendre nodes and weights on [-1, 1] (library routine)."""
    x, w = np.polynomial.legendre.leggauss(int(npts))
    return x.astype(np.float64), w.astype(np.float64)


def lagrange_eval(nodes, x):
    """Values and first derivatives of the Lagrange basis on `nodes` at points x.

    Returns (L, dL) with L[k, i] = l_i(x_k) and dL[k, i] = l_i'(x_k), from the
    product formula l_i(x) = prod_{m != i} (x - x_m) / (x_i - x_m).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(nodes)
    L = np.ones((len(x), m))
    dL = np.zeros((len(x), m))
    for i in range(m):
        for k in range(len(x)):
            val = 1.0
            for j in range(m):
                if j != i:
                    val *= (x[k] - nodes[j]) / (nodes[i] - nodes[j])
            L[k, i] = val
            der = 0.0
            for j in range(m):
                if j == i:
                    continue
                term = 1.0 / (nodes[i] - nodes[j])
                for l in range(m):
                    if l != i and l != j:
                        term *= (x[k] - nodes[l]) / (nodes[i] - nodes[l])
                der += term
            dL[k, i] = der
    return L, dL


def penalty(p, h, form=0, eps=0.125):
    """Face penalty sigma (Sec. 3.5, eq. pen_poly). form 0: (p+1)^2/(eps h); 1: (p+1)^2/(eps h^2)."""
    if form == 0:
        return (p + 1) ** 2 / (eps * h)
    if form == 1:
        return (p + 1) ** 2 / (eps * h * h)
    raise ValueError("penalty form must be 0 or 1")


def sipdg_1d(n, p, lo, hi, sigma, nq_extra=2):
    """Global 1-D SIPDG matrix and (diagonal) mass on n elements of degree p.

    Volume term int u' v' and every face term are assembled element by element
    with a Gauss rule of p+1+nq_extra points (exact). Interior faces carry
    -[[u]]{v'} - {u'}[[v]] + sigma [[u]][[v]] with n^- = +1, n^+ = -1; the two
    domain ends carry the Nitsche terms -u d_n v - d_n u v + sigma u v.
    Returns (A1 [L, L], M1 [L]) with L = n (p+1); M1 is the collocated GL mass
    w_a h / 2.
    """
    n1 = p + 1
    h = (hi - lo) / n
    xi, w = gauss_legendre(n1)
    xq, wq = gauss_legendre(n1 + nq_extra)
    _, dLq = lagrange_eval(xi, xq)
    Lm, dLm = lagrange_eval(xi, [-1.0])
    Lp, dLp = lagrange_eval(xi, [1.0])
    Lm, dLm, Lp, dLp = Lm[0], dLm[0] * (2.0 / h), Lp[0], dLp[0] * (2.0 / h)
    L = n * n1
    A = np.zeros((L, L))
    for e in range(n):
        s = slice(e * n1, (e + 1) * n1)
        dphys = dLq * (2.0 / h)
        A[s, s] += dphys.T @ (wq[:, None] * (h / 2.0) * dphys)
    # interior faces between element e-1 (minus side) and e (plus side)
    for e in range(1, n):
        idx = np.concatenate([np.arange((e - 1) * n1, e * n1), np.arange(e * n1, (e + 1) * n1)])
        jump = np.concatenate([Lp * (+1.0), Lm * (-1.0)])
        avg = np.concatenate([0.5 * dLp, 0.5 * dLm])
        loc = -np.outer(jump, avg) - np.outer(avg, jump) + sigma * np.outer(jump, jump)
        A[np.ix_(idx, idx)] += loc
    # boundary faces: exterior trace zero, one-sided average
    for e, val, der, nrm in ((0, Lm, dLm, -1.0), (n - 1, Lp, dLp, +1.0)):
        idx = np.arange(e * n1, (e + 1) * n1)
        jump = val * nrm
        avg = der
        loc = -np.outer(jump, avg) - np.outer(avg, jump) + sigma * np.outer(jump, jump)
        A[np.ix_(idx, idx)] += loc
    M1 = np.tile(w * (h / 2.0), n)
    return A, M1


# ---------------------------------------------------------------------------
# Nodes, weights, orderings
# ---------------------------------------------------------------------------
def _element_xyz(mesh, e):
    nx, ny, _ = mesh.n
    return e % nx, (e // nx) % ny, e // (nx * ny)


def global_indices(mesh):
    """Global 1-D node indices (X, Y, Z) of every node in element-blocked order."""
    n1 = mesh.n1
    e = np.arange(mesh.E)
    ex, ey, ez = e % mesh.n[0], (e // mesh.n[0]) % mesh.n[1], e // (mesh.n[0] * mesh.n[1])
    loc = np.arange(mesh.npe)
    a, b, c = loc % n1, (loc // n1) % n1, loc // (n1 * n1)
    X = (ex[:, None] * n1 + a[None, :]).ravel()
    Y = (ey[:, None] * n1 + b[None, :]).ravel()
    Z = (ez[:, None] * n1 + c[None, :]).ravel()
    return X, Y, Z


def lex_of_eb(mesh):
    """Map element-blocked node index -> lexicographic index X + Lx (Y + Ly Z)."""
    X, Y, Z = global_indices(mesh)
    return X + mesh.L[0] * (Y + mesh.L[1] * Z)


def axis_nodes(mesh, d):
    """Physical coordinates of the global 1-D GL nodes along axis d."""
    xi, _ = gauss_legendre(mesh.n1)
    e = np.arange(mesh.n[d])
    return (mesh.lo[d] + mesh.h[d] * (e[:, None] + (xi[None, :] + 1.0) / 2.0)).ravel()


def axis_weights(mesh, d):
    _, w = gauss_legendre(mesh.n1)
    return np.tile(w * mesh.h[d] / 2.0, mesh.n[d])


def node_coords(mesh):
    """[Nq, 3] coordinates of all nodes, element-blocked order."""
    X, Y, Z = global_indices(mesh)
    return np.stack([axis_nodes(mesh, 0)[X], axis_nodes(mesh, 1)[Y], axis_nodes(mesh, 2)[Z]], axis=1)


def quad_weights(mesh):
    """[Nq] quadrature weights W_q = w_a w_b w_c (hx/2)(hy/2)(hz/2)."""
    X, Y, Z = global_indices(mesh)
    return axis_weights(mesh, 0)[X] * axis_weights(mesh, 1)[Y] * axis_weights(mesh, 2)[Z]


# ---------------------------------------------------------------------------
# Operator assembly
# ---------------------------------------------------------------------------
def level_sigmas(mesh, penalty_form=0, eps=0.125):
    return [penalty(mesh.p, mesh.h[d], penalty_form, eps) for d in range(3)]


def assemble_kron(mesh, penalty_form=0, eps=0.125):
    """3-D SIPDG matrix as the Kronecker sum Ax(x)My(x)Mz + Mx(x)Ay(x)Mz + Mx(x)My(x)Az
    (the tensor-product reduction of Sec. 3.5), returned in element-blocked order
    as a scipy CSR matrix."""
    sig = level_sigmas(mesh, penalty_form, eps)
    A1, M1 = [], []
    for d in range(3):
        a, m = sipdg_1d(mesh.n[d], mesh.p, mesh.lo[d], mesh.hi[d], sig[d])
        A1.append(scipy.sparse.csr_matrix(a))
        M1.append(scipy.sparse.diags(m))
    k = scipy.sparse.kron
    A_lex = (k(M1[2], k(M1[1], A1[0])) + k(M1[2], k(A1[1], M1[0])) + k(A1[2], k(M1[1], M1[0]))).tocsr()
    perm = lex_of_eb(mesh)
    return A_lex[perm][:, perm].tocsr()


def _basis_1d_tables(xi, pts):
    L, dL = lagrange_eval(xi, pts)
    return L, dL


def assemble_dense(mesh, penalty_form=0, eps=0.125, nq_extra=2):
    """3-D SIPDG matrix assembled directly from eq. sip_bilinear with explicit 3-D
    gradients, normals, jumps and averages, element by element and face by
    face, using Gauss rules of p+1+nq_extra points. Tiny meshes only."""
    n1, p = mesh.n1, mesh.p
    xi, _ = gauss_legendre(n1)
    xq, wq = gauss_legendre(n1 + nq_extra)
    Lq, dLq = _basis_1d_tables(xi, xq)
    Lb, dLb = _basis_1d_tables(xi, [-1.0, 1.0])  # rows: xi=-1, xi=+1
    sig = level_sigmas(mesh, penalty_form, eps)
    h = mesh.h
    A = np.zeros((mesh.Nq, mesh.Nq))
    npe = mesh.npe
    loc = np.arange(npe)
    la, lb, lc = loc % n1, (loc // n1) % n1, loc // (n1 * n1)
    nq = len(xq)

    def eval_basis(ref_pts_per_axis):
        """ref_pts_per_axis: three (L, dL) table pairs, each [npts_d, n1] in
        reference coordinates. Returns phi [P, npe] and grad [P, npe, 3] on the
        tensor grid of points (x fastest)."""
        (Lx, dLx), (Ly, dLy), (Lz, dLz) = ref_pts_per_axis
        px, py, pz = Lx.shape[0], Ly.shape[0], Lz.shape[0]
        phi = np.zeros((pz, py, px, npe))
        grad = np.zeros((pz, py, px, npe, 3))
        for k in range(pz):
            for j in range(py):
                for i in range(px):
                    phi[k, j, i] = Lx[i, la] * Ly[j, lb] * Lz[k, lc]
                    grad[k, j, i, :, 0] = dLx[i, la] * (2.0 / h[0]) * Ly[j, lb] * Lz[k, lc]
                    grad[k, j, i, :, 1] = Lx[i, la] * dLy[j, lb] * (2.0 / h[1]) * Lz[k, lc]
                    grad[k, j, i, :, 2] = Lx[i, la] * Ly[j, lb] * dLz[k, lc] * (2.0 / h[2])
        return phi.reshape(-1, npe), grad.reshape(-1, npe, 3)

    # volume terms
    _, gvol = eval_basis([(Lq, dLq)] * 3)
    wvol = (wq[None, None, :] * wq[None, :, None] * wq[:, None, None]).ravel() * (h[0] * h[1] * h[2] / 8.0)
    Kvol = np.einsum("q,qid,qjd->ij", wvol, gvol, gvol)
    for e in range(mesh.E):
        s = slice(e * npe, (e + 1) * npe)
        A[s, s] += Kvol

    def face_tables(d, side):
        """Basis traces on the face xi_d = side of an element; tangential
        directions sampled at the nq-point rule."""
        tab = []
        for ax in range(3):
            if ax == d:
                r = 0 if side < 0 else 1
                tab.append((Lb[r:r + 1], dLb[r:r + 1]))
            else:
                tab.append((Lq, dLq))
        phi, grad = eval_basis(tab)
        t = [ax for ax in range(3) if ax != d]
        wf = (wq[None, :] * wq[:, None]).ravel() * (h[t[0]] * h[t[1]] / 4.0)
        return phi, grad, wf

    stride = (1, mesh.n[0], mesh.n[0] * mesh.n[1])
    for d in range(3):
        nrm = np.zeros(3)
        nrm[d] = 1.0
        phi_m, grad_m, wf = face_tables(d, +1)  # minus element: face at its xi_d = +1
        phi_p, grad_p, _ = face_tables(d, -1)  # plus element: face at its xi_d = -1
        for e in range(mesh.E):
            exyz = _element_xyz(mesh, e)
            # interior face towards +d
            if exyz[d] + 1 < mesh.n[d]:
                ep = e + stride[d]
                idx = np.concatenate([np.arange(e * npe, (e + 1) * npe), np.arange(ep * npe, (ep + 1) * npe)])
                jump = np.concatenate([phi_m[:, :, None] * nrm, phi_p[:, :, None] * (-nrm)], axis=1)
                avg = np.concatenate([0.5 * grad_m, 0.5 * grad_p], axis=1)
                loc_m = (
                    -np.einsum("q,qid,qjd->ij", wf, jump, avg)
                    - np.einsum("q,qid,qjd->ij", wf, avg, jump)
                    + sig[d] * np.einsum("q,qid,qjd->ij", wf, jump, jump)
                )
                A[np.ix_(idx, idx)] += loc_m
            # boundary faces (exterior trace zero, one-sided gradient)
            for side, at_bdry in ((-1, exyz[d] == 0), (+1, exyz[d] == mesh.n[d] - 1)):
                if not at_bdry:
                    continue
                phi_b, grad_b = (phi_p, grad_p) if side < 0 else (phi_m, grad_m)
                idx = np.arange(e * npe, (e + 1) * npe)
                jump = phi_b[:, :, None] * (side * nrm)
                avg = grad_b
                loc_b = (
                    -np.einsum("q,qid,qjd->ij", wf, jump, avg)
                    - np.einsum("q,qid,qjd->ij", wf, avg, jump)
                    + sig[d] * np.einsum("q,qid,qjd->ij", wf, jump, jump)
                )
                A[np.ix_(idx, idx)] += loc_b
    return A


# ---------------------------------------------------------------------------
# Boundary data and right-hand side
# ---------------------------------------------------------------------------
def boundary_face_nodes(mesh):
    """List of 6 arrays [T1, T2, 3]: coordinates of the GL nodes of the faces
    -x, +x, -y, +y, -z, +z; (T1, T2) are the global node indices of the two
    tangential axes in increasing axis order."""
    out = []
    for d in range(3):
        t = [ax for ax in range(3) if ax != d]
        c1, c2 = axis_nodes(mesh, t[0]), axis_nodes(mesh, t[1])
        for side in (0, 1):
            pts = np.zeros((len(c1), len(c2), 3))
            pts[:, :, d] = mesh.lo[d] if side == 0 else mesh.hi[d]
            pts[:, :, t[0]] = c1[:, None]
            pts[:, :, t[1]] = c2[None, :]
            out.append(pts)
    return out


def boundary_data_direct(mesh, f, chunk=64, node_stride=1):
    """Dirichlet data of Sec. 6.3: g(x_b) = sum_q W_q f(x_q)/|x_b - x_q|
    at every boundary face node, by direct Gauss quadrature.

    f: [Nq] or [nf, Nq]. Returns a list of 6 arrays [nf, T1, T2] (or [T1, T2]).
    node_stride > 1 evaluates only every node_stride-th node of each face
    (flattened order) and returns flat arrays [nf, n_eval]; used to time a
    bounded sample of the full evaluation.
    """
    f = np.asarray(f, dtype=np.float64)
    single = f.ndim == 1
    F = (np.atleast_2d(f) * quad_weights(mesh)[None, :]).T  # [Nq, nf]
    xq = node_coords(mesh)
    out = []
    for pts in boundary_face_nodes(mesh):
        shp = pts.shape[:2]
        P = pts.reshape(-1, 3)
        if node_stride > 1:
            P = P[::node_stride]
            shp = (P.shape[0],)
        g = np.zeros((P.shape[0], F.shape[1]))
        for s in range(0, P.shape[0], chunk):
            blk = P[s:s + chunk]
            dx = blk[:, None, 0] - xq[None, :, 0]
            dy = blk[:, None, 1] - xq[None, :, 1]
            dz = blk[:, None, 2] - xq[None, :, 2]
            G = 1.0 / np.sqrt(dx * dx + dy * dy + dz * dz)
            g[s:s + chunk] = G @ F
        g = g.T.reshape(F.shape[1], *shp)
        out.append(g[0] if single else g)
    return out


def gauss_sum_1_over_r(rmin, rmax, tol):
    """Coefficients of 1/r ~ sum_k c_k exp(-a_k r^2) on [rmin, rmax] (Sec. 5.2).

    Trapezoidal rule in t for 1/r = (2/sqrt(pi)) int exp(-r^2 e^(2t) + t) dt:
    c_k = (2/sqrt(pi)) h e^(t_k), a_k = e^(2 t_k). The t-range drops tails
    below tol at both ends; the step h is halved from 1 until the maximum
    relative error on 4000 log-spaced radii is below tol."""
    from scipy.special import erfc
    t_lo = math.log(tol * math.sqrt(math.pi) / (2.0 * rmax))
    x = 0.5
    while erfc(x) > 0.5 * tol:
        x += 0.01
    t_hi = math.log(x / rmin)
    r = np.exp(np.linspace(math.log(rmin), math.log(rmax), 4000))
    h = 1.0
    while h > 1e-3:
        t = np.arange(t_lo, t_hi + h, h)
        c = 2.0 / math.sqrt(math.pi) * h * np.exp(t)
        a = np.exp(2.0 * t)
        err = np.abs((np.exp(-np.outer(r * r, a)) @ c) * r - 1.0).max()
        if err <= tol:
            return c, a, err
        h *= 0.5
    raise RuntimeError("Gaussian-sum step search failed")


def boundary_data_gausssum(mesh, f, tol=1e-12, chunk=8):
    """Dirichlet data of Sec. 6.3 with 1/r replaced by the Gaussian sum of
    Sec. 5.2, evaluated on the tensor grid as three 1-D contractions per term
    and face. f: [nf, Nq]. Returns the same layout as boundary_data_direct.
    Sources are processed chunk at a time (memory only; every source's sums
    are the same)."""
    f = np.atleast_2d(np.asarray(f, dtype=np.float64))
    if f.shape[0] > chunk:
        parts = [boundary_data_gausssum(mesh, f[i:i + chunk], tol, chunk) for i in range(0, f.shape[0], chunk)]
        return [np.concatenate([pp[face] for pp in parts]) for face in range(6)]
    xq = [axis_nodes(mesh, d) for d in range(3)]
    xi, _ = gauss_legendre(mesh.n1)
    rmin = min((1.0 - xi[-1]) * mesh.h[d] / 2.0 for d in range(3))
    rmax = float(np.linalg.norm(mesh.hi - mesh.lo))
    c, a, _ = gauss_sum_1_over_r(0.999 * rmin, 1.001 * rmax, tol)
    perm = lex_of_eb(mesh)
    Lx, Ly, Lz = mesh.L
    out = [np.zeros((f.shape[0], mesh.L[[ax for ax in range(3) if ax != d][0]],
                     mesh.L[[ax for ax in range(3) if ax != d][1]])) for d in range(3) for _ in range(2)]
    W = quad_weights(mesh)
    nf = f.shape[0]
    F = np.empty((nf, mesh.Nq))
    F[:, perm] = W[None, :] * f
    F = F.reshape(nf, Lz, Ly, Lx)  # [source, Z, Y, X]
    for d in range(3):
        t = [ax for ax in range(3) if ax != d]
        for side in range(2):
            face = mesh.lo[d] if side == 0 else mesh.hi[d]
            GN = np.exp(-np.outer(a, (xq[d] - face) ** 2))  # [k, L_d]
            # contraction along the normal axis for all terms k at once
            if d == 0:
                T = np.tensordot(F, GN, axes=([3], [1])).transpose(0, 3, 2, 1)  # [src, k, y, z]
            elif d == 1:
                T = np.tensordot(F, GN, axes=([2], [1])).transpose(0, 3, 2, 1)  # [src, k, x, z]
            else:
                T = np.tensordot(F, GN, axes=([1], [1])).transpose(0, 3, 2, 1)  # [src, k, x, y]
            # every source accumulates its terms k in ascending order
            acc = np.zeros((nf, mesh.L[t[0]], mesh.L[t[1]]))
            for k in range(len(c)):
                G1 = np.exp(-a[k] * (xq[t[0]][:, None] - xq[t[0]][None, :]) ** 2)
                G2 = np.exp(-a[k] * (xq[t[1]][:, None] - xq[t[1]][None, :]) ** 2)
                acc += c[k] * (G1[None, :, :] @ T[:, k] @ G2.T[None, :, :])
            out[2 * d + side][:] = acc
    return out


def rhs(mesh, f, g, penalty_form=0, eps=0.125):
    """Load vector of the Nitsche-SIPDG Poisson problem.

    b = 4 pi W f (pointwise quadrature of 4 pi int f v) plus, on each boundary
    face, int_F g (sigma v - d_n v) with g interpolated at the face GL nodes and
    integrated with the face GL rule. f: [Nq]; g: list of 6 face arrays as
    returned by boundary_data_direct (or None for zero data)."""
    n1 = mesh.n1
    xi, w = gauss_legendre(n1)
    Lb, dLb = lagrange_eval(xi, [-1.0, 1.0])
    sig = level_sigmas(mesh, penalty_form, eps)
    b = FOUR_PI * quad_weights(mesh) * np.asarray(f, dtype=np.float64)
    if g is None:
        return b
    X, Y, Z = global_indices(mesh)
    G = (X, Y, Z)
    wts = [axis_weights(mesh, d) for d in range(3)]
    for d in range(3):
        t = [ax for ax in range(3) if ax != d]
        for side in (0, 1):
            gface = np.asarray(g[2 * d + side])
            r = 0 if side == 0 else 1
            nrm = -1.0 if side == 0 else 1.0
            # per local node index along d: sigma l_a(+-1) - d_n l_a(+-1)
            coef = sig[d] * Lb[r] - nrm * dLb[r] * (2.0 / mesh.h[d])
            e_d = G[d] // n1
            a_d = G[d] % n1
            on_face = e_d == (0 if side == 0 else mesh.n[d] - 1)
            idx = np.nonzero(on_face)[0]
            T1, T2 = G[t[0]][idx], G[t[1]][idx]
            b[idx] += coef[a_d[idx]] * wts[t[0]][T1] * wts[t[1]][T2] * gface[T1, T2]
    return b


# ---------------------------------------------------------------------------
# Solvers
# ---------------------------------------------------------------------------
def solve_dense(A, b):
    """Dense Cholesky solve (A SPD)."""
    A = A.toarray() if scipy.sparse.issparse(A) else np.asarray(A)
    c = scipy.linalg.cho_factor(A, lower=True)
    return scipy.linalg.cho_solve(c, b)


def fdm_factors(mesh, penalty_form=0, eps=0.125):
    """Generalised eigen-decompositions A_d S_d = M_d S_d Lambda_d of the 1-D
    operators (S_d^T M_d S_d = I)."""
    sig = level_sigmas(mesh, penalty_form, eps)
    out = []
    for d in range(3):
        a, m = sipdg_1d(mesh.n[d], mesh.p, mesh.lo[d], mesh.hi[d], sig[d])
        lam, S = scipy.linalg.eigh(a, np.diag(m))
        out.append((lam, S))
    return out


def solve_fdm(mesh, b, penalty_form=0, eps=0.125, factors=None):
    """Exact solve of the Kronecker-sum system by fast diagonalisation:
    v = (Sz(x)Sy(x)Sx) diag(1/(lx_i + ly_j + lz_k)) (Sz(x)Sy(x)Sx)^T b.
    b: [Nq] or [nb, Nq] (element-blocked)."""
    if factors is None:
        factors = fdm_factors(mesh, penalty_form, eps)
    (lx, Sx), (ly, Sy), (lz, Sz) = factors
    b = np.asarray(b, dtype=np.float64)
    single = b.ndim == 1
    B = np.atleast_2d(b)
    perm = lex_of_eb(mesh)
    Lx, Ly, Lz = mesh.L
    out = np.empty_like(B)
    denom = lz[:, None, None] + ly[None, :, None] + lx[None, None, :]
    for r in range(B.shape[0]):
        blex = np.empty(mesh.Nq)
        blex[perm] = B[r]
        t = blex.reshape(Lz, Ly, Lx)
        # (Sz (x) Sy (x) Sx)^T b, one axis at a time: t[k, j, i] = sum S_z[z,k] S_y[y,j] S_x[x,i] b[z,y,x]
        t = np.tensordot(t, Sx, axes=([2], [0]))            # [z, y, i]
        t = np.tensordot(t, Sy, axes=([1], [0]))            # [z, i, j]
        t = np.tensordot(t, Sz, axes=([0], [0]))            # [i, j, k]
        t = t.transpose(2, 1, 0) / denom                    # [k, j, i]
        t = np.tensordot(t, Sx, axes=([2], [1]))            # [k, j, x]
        t = np.tensordot(t, Sy, axes=([1], [1]))            # [k, x, y]
        t = np.tensordot(t, Sz, axes=([0], [1]))            # [x, y, z]
        out[r] = t.transpose(2, 1, 0).ravel()[perm]
    return out[0] if single else out


def solve(mesh, b, penalty_form=0, eps=0.125, method="auto"):
    """Exact solution of A v = b. method: 'dense', 'fdm' or 'auto'."""
    if method == "auto":
        method = "dense" if mesh.Nq <= 4000 else "fdm"
    if method == "dense":
        A = assemble_dense(mesh, penalty_form, eps) if mesh.Nq <= 1000 else assemble_kron(mesh, penalty_form, eps)
        b2 = np.atleast_2d(b)
        x = solve_dense(A, b2.T).T
        return x[0] if np.ndim(b) == 1 else x
    return solve_fdm(mesh, b, penalty_form, eps)


# ---------------------------------------------------------------------------
# Exchange build
# ---------------------------------------------------------------------------
def pair_list(N):
    """Distinct orbital pairs (i, j), i <= j, upper-triangular row-major."""
    return [(i, j) for i in range(N) for j in range(i, N)]


def poisson(mesh, f, penalty_form=0, eps=0.125, method="auto", g=None):
    """v solving -Lap v = 4 pi f with the Coulomb-quadrature Dirichlet data.
    f: [nf, Nq]. Returns (v [nf, Nq], g)."""
    f = np.atleast_2d(np.asarray(f, dtype=np.float64))
    if g is None:
        g = boundary_data_direct(mesh, f)
    B = np.stack([rhs(mesh, f[r], [gf[r] for gf in g], penalty_form, eps) for r in range(f.shape[0])])
    v = np.atleast_2d(solve(mesh, B, penalty_form, eps, method))
    return v, g


def exchange_partial(mesh, psi, src_begin, src_end, penalty_form=0, eps=0.125, method="auto", g_route="direct",
                     with_self=False):
    """The part of the exchange build that sources [src_begin, src_end) of the
    list (0 = Hartree density rho, then the pairs of pair_list) contribute:
    K_part[i, j] = sum_q W_q psi_i(q) sum_{pairs (s, j) in range} psi_s(q) v_sj(q)
    (eq. fock_exchange, Sec. 6.1.2, summed over the listed pairs only; K is
    linear in the pair potentials, so disjoint ranges add up to K) and E_H
    (Sec. 2.3.1) if source 0 is in the range, else 0. g_route "gausssum"
    takes the Dirichlet data from boundary_data_gausssum at 1e-12 instead of
    the direct quadrature (for meshes where the direct sum is too slow).
    with_self: also return the sources' self-energies (f|f) = sum_q W_q f v."""
    psi = np.asarray(psi, dtype=np.float64)
    N = psi.shape[0]
    Wq = quad_weights(mesh)
    pairs = pair_list(N)
    idx = list(range(int(src_begin), int(src_end)))
    if not idx:
        return np.zeros((N, N)), 0.0
    rho = np.sum(psi * psi, axis=0)
    sources = np.stack([rho if k == 0 else psi[pairs[k - 1][0]] * psi[pairs[k - 1][1]] for k in idx])
    g = boundary_data_gausssum(mesh, sources, tol=1e-12) if g_route == "gausssum" else None
    v, _ = poisson(mesh, sources, penalty_form, eps, method, g=g)
    Wacc = np.zeros_like(psi)
    E_H = 0.0
    for row, k in enumerate(idx):
        if k == 0:
            E_H = 0.5 * float(np.sum(Wq * rho * v[row]))
            continue
        s_, j = pairs[k - 1]
        Wacc[j] += psi[s_] * v[row]
        if s_ != j:
            Wacc[s_] += psi[j] * v[row]
    K_part = (psi * Wq[None, :]) @ Wacc.T
    if with_self:
        return K_part, E_H, np.sum(Wq[None, :] * sources * v, axis=1)
    return K_part, E_H


def exchange_build(mesh, psi, penalty_form=0, eps=0.125, method="auto", keep_potentials=False, g_route="direct"):
    """Hartree potential, pair potentials, K, E_H and E_X for orbitals psi [N, Nq].
    g_route "gausssum": Dirichlet data from boundary_data_gausssum at 1e-12
    (pinned against the direct quadrature) instead of the direct sum."""
    psi = np.asarray(psi, dtype=np.float64)
    N = psi.shape[0]
    Wq = quad_weights(mesh)
    pairs = pair_list(N)
    rho = np.sum(psi * psi, axis=0)
    sources = np.stack([rho] + [psi[i] * psi[j] for (i, j) in pairs])
    g = boundary_data_gausssum(mesh, sources, tol=1e-12) if g_route == "gausssum" else None
    v, _ = poisson(mesh, sources, penalty_form, eps, method, g=g)
    vH, vpair = v[0], v[1:]
    Wacc = np.zeros_like(psi)
    for k, (s, j) in enumerate(pairs):
        Wacc[j] += psi[s] * vpair[k]
        if s != j:
            Wacc[s] += psi[j] * vpair[k]
    K = (psi * Wq[None, :]) @ Wacc.T
    E_H = 0.5 * float(np.sum(Wq * rho * vH))
    E_X = -0.5 * float(np.trace(K))
    # Coulomb self-energy of every source (Sec. 2.3.1): (f|f) = int f v, by the
    # same pointwise quadrature; for a pair density the integral (ij|ij), for
    # the density (rho|rho) = 2 E_H
    self_e = np.sum(Wq[None, :] * sources * v, axis=1)
    out = {"K": K, "E_H": E_H, "E_X": E_X, "v_H": vH, "W": Wacc, "pairs": pairs, "self": self_e}
    if keep_potentials:
        out["v_pairs"] = vpair
    return out


def ace_apply(build, Wq, U):
    """Adaptively compressed exchange operator of an exchange build (the
    compressed V_X of Sec. 2.3.1 eq. exchange that the HF SCF of Sec. 7.2
    applies): V_X^ACE u = -W Ks^-1 (W^T diag(Wq) u), Ks = (K + K^T) / 2, with W
    the build's exchange accumulation W_j = sum_s psi_s v_sj (= -V_X psi_j)
    and K_ij = <psi_i, W_j>. U: [m, Nq]; returns [m, Nq]."""
    W = np.asarray(build["W"], dtype=np.float64)
    K = np.asarray(build["K"], dtype=np.float64)
    Ks = 0.5 * (K + K.T)
    C = W @ (np.asarray(U, dtype=np.float64) * Wq[None, :]).T  # [N, m]
    Z = np.linalg.solve(Ks, C)
    return -(W.T @ Z).T


def jk_apply(mesh, psi, U, penalty_form=0, eps=0.125, method="auto", hartree=True, exchange=True):
    """Hartree and exchange operators of Sec. 2.3.1 applied to trial functions
    u_k given by their values at the fine-level nodes (the action an
    eigensolver needs, Sec. 6.1: the same auxiliary-grid Poisson solves as the
    exchange build, with the trial function in place of the second orbital):
      (J u_k)(q) = v_H(q) u_k(q),             -lap v_H  = 4 pi sum_j psi_j^2
      (X u_k)(q) = -sum_j psi_j(q) v_jk(q),   -lap v_jk = 4 pi psi_j u_k
    Each v solves the discrete SIPDG problem of Sec. 6.3 / 6.4 exactly, with the
    source's own Coulomb boundary data. psi: [N, Nq]; U: [m, Nq]. Returns
    (JU, XU), each [m, Nq], or None for an operator not asked for."""
    psi = np.asarray(psi, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    N, m = psi.shape[0], U.shape[0]
    JU = XU = None
    if hartree:
        rho = np.sum(psi * psi, axis=0)
        vH, _ = poisson(mesh, rho[None, :], penalty_form, eps, method)
        JU = vH[0][None, :] * U
    if exchange:
        XU = np.zeros_like(U)
        for k in range(m):
            sources = psi * U[k][None, :]  # row j: psi_j u_k
            v, _ = poisson(mesh, sources, penalty_form, eps, method)
            for j in range(N):  # j ascending
                XU[k] -= psi[j] * v[j]
    return JU, XU


def transfer_matrix(fine, coarse):
    """Prolongation P [fine.Nq, coarse.Nq] between nested levels of the hp
    hierarchy (Sec. 6.4): a coarse DG function, given by its values at the
    coarse GL nodes, evaluated at the fine nodes. Each fine node lies inside
    one coarse element (the fine elements are the coarse ones or their
    children); its row holds the coarse element's tensor Lagrange basis at the
    node's reference coordinates (sparse: n1c^3 entries per row). Restriction
    is P^T."""
    xf = node_coords(fine)
    xi, _ = gauss_legendre(coarse.n1)
    hc = np.asarray(coarse.h, dtype=np.float64)
    ec = np.floor((xf - coarse.lo[None, :]) / hc[None, :]).astype(np.int64)
    ec = np.clip(ec, 0, np.asarray(coarse.n)[None, :] - 1)
    L = []
    for d in range(3):
        t = 2.0 * (xf[:, d] - (coarse.lo[d] + ec[:, d] * hc[d])) / hc[d] - 1.0
        Ld, _ = lagrange_eval(xi, t)
        L.append(Ld)  # [Nq_f, n1c]
    n1 = coarse.n1
    e = ec[:, 0] + coarse.n[0] * (ec[:, 1] + coarse.n[1] * ec[:, 2])
    rows, cols, vals = [], [], []
    for k in range(n1):
        for j in range(n1):
            for i in range(n1):
                rows.append(np.arange(fine.Nq))
                cols.append(e * coarse.npe + i + n1 * (j + n1 * k))
                vals.append(L[0][:, i] * L[1][:, j] * L[2][:, k])
    return scipy.sparse.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                   shape=(fine.Nq, coarse.Nq))
