"""Adaptive octree auxiliary mesh with 2:1 nonconforming faces, and the SIPDG
operator and load on it (Sec. 6.2: the auxiliary mesh is refined where a
quadrature indicator of the density exceeds a threshold; Sec. 3.4 eq.
sip_bilinear and Sec. 6.3 on a mesh whose faces may meet a neighbour's face
in a quarter).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: plain, slow, dense.

Readings (where the paper leaves the details open):
* The leaves are boxes of the uniform root grid n^3 split isotropically into
  8 children (the paper also allows splits along fewer axes); the tree is
  kept 2:1 balanced across faces.
* A face between leaves of different size is integrated on the smaller face
  with the smaller element's Gauss points; both traces are evaluated there.
  The penalty uses the smaller element's size: sigma_F = (p+1)^2/(eps h_F).
* The refinement indicator of a leaf is Q = |I_K(rho) - sum_children I_C(rho)|
  with I the degree-p Gauss-Legendre rule of the leaf or child; a leaf is split
  while Q > delta and its level is below max_level.
"""

from __future__ import annotations

import math

import numpy as np

from .dg_oracle import FOUR_PI, gauss_legendre, lagrange_eval, penalty


class OctreeMesh:
    """Leaves of an octree over [lo, hi]: the uniform n^3 root grid (level 0)
    refined by 8-child splits. A leaf is (level, ix, iy, iz) in the level's
    integer grid of n_d 2^level cells per axis; every leaf carries degree-p
    tensor GL nodes."""

    def __init__(self, lo, hi, n, p):
        self.lo = np.asarray(lo, dtype=np.float64).reshape(3)
        self.hi = np.asarray(hi, dtype=np.float64).reshape(3)
        if np.isscalar(n):
            n = (n, n, n)
        self.n = tuple(int(v) for v in n)
        self.p = int(p)
        self.n1 = self.p + 1
        self.npe = self.n1 ** 3
        self.H = (self.hi - self.lo) / np.asarray(self.n, dtype=np.float64)
        self.leaves = {(0, ix, iy, iz) for iz in range(self.n[2]) for iy in range(self.n[1]) for ix in range(self.n[0])}

    # geometry ------------------------------------------------------------
    def h(self, key):
        return self.H / (2 ** key[0])

    def origin(self, key):
        return self.lo + np.asarray(key[1:], dtype=np.float64) * self.h(key)

    def extent(self, level, d):
        return self.n[d] * 2 ** level

    # structure -----------------------------------------------------------
    def leaf_list(self):
        """Leaves in a fixed order: by root cell (x fastest), then level and
        position; without refinement this is the uniform mesh's element order."""

        def sort_key(k):
            lv, ix, iy, iz = k
            r = (ix >> lv, iy >> lv, iz >> lv)
            return (r[0] + self.n[0] * (r[1] + self.n[1] * r[2]), lv, iz, iy, ix)

        return sorted(self.leaves, key=sort_key)

    @property
    def E(self):
        return len(self.leaves)

    @property
    def Nq(self):
        return self.E * self.npe

    def refine(self, keys):
        for k in list(keys):
            if k not in self.leaves:
                continue
            self.leaves.remove(k)
            lv, ix, iy, iz = k
            for c in range(8):
                self.leaves.add((lv + 1, 2 * ix + (c & 1), 2 * iy + ((c >> 1) & 1), 2 * iz + (c >> 2)))

    def leaf_covering(self, level, ix, iy, iz):
        """The leaf that contains the cell (level, ix, iy, iz), if the cell is
        not refined further; None when finer leaves cover it."""
        for lv in range(level, -1, -1):
            s = level - lv
            k = (lv, ix >> s, iy >> s, iz >> s)
            if k in self.leaves:
                return k
        return None

    def neighbour_cell(self, key, d, side):
        """The same-level cell across face (d, side) of leaf `key`, or None at
        the domain boundary."""
        lv = key[0]
        c = list(key[1:])
        c[d] += side
        if c[d] < 0 or c[d] >= self.extent(lv, d):
            return None
        return (lv, c[0], c[1], c[2])

    def balance(self):
        """Refine until leaves sharing a face differ by at most one level."""
        changed = True
        while changed:
            changed = False
            split = set()
            for k in self.leaves:
                for d in range(3):
                    for side in (-1, 1):
                        nb = self.neighbour_cell(k, d, side)
                        if nb is None:
                            continue
                        L = self.leaf_covering(*nb)
                        if L is not None and L[0] < k[0] - 1:
                            split.add(L)
            if split:
                self.refine(split)
                changed = True

    def is_balanced(self):
        for k in self.leaves:
            for d in range(3):
                for side in (-1, 1):
                    nb = self.neighbour_cell(k, d, side)
                    if nb is None:
                        continue
                    L = self.leaf_covering(*nb)
                    if L is not None and L[0] < k[0] - 1:
                        return False
        return True

    # nodes and weights ---------------------------------------------------
    def node_coords(self):
        xi, _ = gauss_legendre(self.n1)
        loc = np.arange(self.npe)
        a, b, c = loc % self.n1, (loc // self.n1) % self.n1, loc // (self.n1 * self.n1)
        out = []
        for k in self.leaf_list():
            o, h = self.origin(k), self.h(k)
            out.append(np.stack([o[0] + (xi[a] + 1) * h[0] / 2, o[1] + (xi[b] + 1) * h[1] / 2,
                                 o[2] + (xi[c] + 1) * h[2] / 2], axis=1))
        return np.concatenate(out)

    def quad_weights(self):
        _, w = gauss_legendre(self.n1)
        loc = np.arange(self.npe)
        a, b, c = loc % self.n1, (loc // self.n1) % self.n1, loc // (self.n1 * self.n1)
        out = []
        for k in self.leaf_list():
            h = self.h(k)
            out.append(w[a] * w[b] * w[c] * h[0] * h[1] * h[2] / 8.0)
        return np.concatenate(out)


def _basis_on_grid(xi, pts_per_axis, h):
    """Tensor Lagrange basis of the GL nodes xi at the tensor grid of reference
    points (one array per axis, x fastest): phi [P, npe], grad [P, npe, 3]
    (physical gradient for an element of size h)."""
    n1 = len(xi)
    npe = n1 ** 3
    loc = np.arange(npe)
    la, lb, lc = loc % n1, (loc // n1) % n1, loc // (n1 * n1)
    tabs = [lagrange_eval(xi, np.atleast_1d(np.asarray(pp, dtype=np.float64))) for pp in pts_per_axis]
    (Lx, dLx), (Ly, dLy), (Lz, dLz) = tabs
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


def _faces(mesh):
    """Every face once: (K, L, d, s) with K the smaller (or, for equal sizes,
    the -d) leaf, s the side of K's face (+1: K's +d face), L the neighbour or
    None on the boundary."""
    out = []
    for K in mesh.leaf_list():
        for d in range(3):
            for s in (-1, 1):
                nb = mesh.neighbour_cell(K, d, s)
                if nb is None:
                    out.append((K, None, d, s))
                    continue
                L = mesh.leaf_covering(*nb)
                if L is None:
                    continue  # finer neighbours own this face
                if L[0] == K[0] and s < 0:
                    continue  # equal sizes: taken from the -d leaf
                out.append((K, L, d, s))
    return out


def _face_quadrature(mesh, K, d, s, xq, wq):
    """Gauss points on face (d, s) of leaf K as per-axis physical coordinate
    lists, and the tensor weights (x fastest over the two tangential axes)."""
    o, h = mesh.origin(K), mesh.h(K)
    axes = []
    for ax in range(3):
        if ax == d:
            axes.append(np.array([o[ax] + (h[ax] if s > 0 else 0.0)]))
        else:
            axes.append(o[ax] + (xq + 1.0) * h[ax] / 2.0)
    t = [ax for ax in range(3) if ax != d]
    w = (wq[None, :] * wq[:, None]).ravel() * (h[t[0]] * h[t[1]] / 4.0)
    return axes, w


def _ref(mesh, key, axes):
    o, h = mesh.origin(key), mesh.h(key)
    return [2.0 * (axes[ax] - o[ax]) / h[ax] - 1.0 for ax in range(3)]


def assemble(mesh, penalty_form=0, eps=0.125, nq_extra=2):
    """Dense SIPDG matrix on the octree leaves (Sec. 3.4 eq. sip_bilinear with
    symmetric Nitsche boundary terms), element-blocked in leaf_list order."""
    xi, _ = gauss_legendre(mesh.n1)
    xq, wq = gauss_legendre(mesh.n1 + nq_extra)
    leaves = mesh.leaf_list()
    index = {k: i for i, k in enumerate(leaves)}
    npe = mesh.npe
    A = np.zeros((mesh.Nq, mesh.Nq))
    wvol = (wq[None, None, :] * wq[None, :, None] * wq[:, None, None]).ravel()
    for K in leaves:
        h = mesh.h(K)
        _, g = _basis_on_grid(xi, [xq] * 3, h)
        e = index[K]
        s_ = slice(e * npe, (e + 1) * npe)
        A[s_, s_] += np.einsum("q,qid,qjd->ij", wvol * (h[0] * h[1] * h[2] / 8.0), g, g, optimize=True)
    for (K, L, d, s) in _faces(mesh):
        axes, wf = _face_quadrature(mesh, K, d, s, xq, wq)
        nrm = np.zeros(3)
        nrm[d] = 1.0
        hK = mesh.h(K)
        sig = penalty(mesh.p, hK[d], penalty_form, eps)  # K is the smaller (or equal) leaf
        phiK, gradK = _basis_on_grid(xi, _ref(mesh, K, axes), hK)
        iK = np.arange(index[K] * npe, (index[K] + 1) * npe)
        if L is None:
            jump = phiK[:, :, None] * (s * nrm)
            avg = gradK
            idx = iK
        else:
            phiL, gradL = _basis_on_grid(xi, _ref(mesh, L, axes), mesh.h(L))
            iL = np.arange(index[L] * npe, (index[L] + 1) * npe)
            # minus = the leaf on the -d side, plus = the +d side; jump v- n - v+ n
            if s > 0:
                (pm, gm, im), (pp, gp, ip) = (phiK, gradK, iK), (phiL, gradL, iL)
            else:
                (pm, gm, im), (pp, gp, ip) = (phiL, gradL, iL), (phiK, gradK, iK)
            jump = np.concatenate([pm[:, :, None] * nrm, pp[:, :, None] * (-nrm)], axis=1)
            avg = np.concatenate([0.5 * gm, 0.5 * gp], axis=1)
            idx = np.concatenate([im, ip])
        loc = (-np.einsum("q,qid,qjd->ij", wf, jump, avg, optimize=True)
               - np.einsum("q,qid,qjd->ij", wf, avg, jump, optimize=True)
               + sig * np.einsum("q,qid,qjd->ij", wf, jump, jump, optimize=True))
        A[np.ix_(idx, idx)] += loc
    return A


def rhs(mesh, f, g=None, penalty_form=0, eps=0.125, nq_extra=2):
    """Load vector: 4 pi W f (pointwise quadrature at the nodes) plus, on each
    boundary face, int_F g (sigma v - d_n v), with g a callable of [P, 3]
    physical points sampled at the face's GL nodes and interpolated to the
    face's Gauss points, as the uniform oracle does (None: zero data)."""
    b = FOUR_PI * mesh.quad_weights() * np.asarray(f, dtype=np.float64)
    if g is None:
        return b
    xi, _ = gauss_legendre(mesh.n1)
    xq, wq = gauss_legendre(mesh.n1 + nq_extra)
    index = {k: i for i, k in enumerate(mesh.leaf_list())}
    npe = mesh.npe
    for (K, L, d, s) in _faces(mesh):
        if L is not None:
            continue
        axes, wf = _face_quadrature(mesh, K, d, s, xq, wq)
        hK = mesh.h(K)
        phi, grad = _basis_on_grid(xi, _ref(mesh, K, axes), hK)
        # g at the face GL nodes, interpolated to the Gauss points
        o = mesh.origin(K)
        gl = [axes[ax] if ax == d else o[ax] + (xi + 1.0) * hK[ax] / 2.0 for ax in range(3)]
        X, Y, Z = np.meshgrid(gl[0], gl[1], gl[2], indexing="ij")
        pts = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(), Z.transpose(2, 1, 0).ravel()],
                       axis=1)
        t0, t1 = [ax for ax in range(3) if ax != d]
        G = np.asarray(g(pts), dtype=np.float64).reshape(mesh.n1, mesh.n1)  # [t1][t0]
        Lq, _ = lagrange_eval(xi, xq)  # [nq, n1]
        gv = (Lq @ G @ Lq.T).ravel()  # [t1 Gauss][t0 Gauss], t0 fastest
        sig = penalty(mesh.p, hK[d], penalty_form, eps)
        dn = grad[:, :, d] * s
        b[index[K] * npe:(index[K] + 1) * npe] += np.einsum("q,q,qi->i", wf, gv, sig * phi - dn)
    return b


def density_indicator(mesh, key, rho):
    """Q of Sec. 6.2 for one leaf: |I_K(rho) - sum over the 8 children of
    I_C(rho)|, I the leaf's (or child's) tensor GL rule of degree p; rho a
    callable of [P, 3] points."""
    xi, w = gauss_legendre(mesh.n1)

    def integral(o, h):
        X = o[0] + (xi + 1) * h[0] / 2
        Y = o[1] + (xi + 1) * h[1] / 2
        Z = o[2] + (xi + 1) * h[2] / 2
        P = np.stack(np.meshgrid(X, Y, Z, indexing="ij"), axis=-1).reshape(-1, 3)
        W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel() * h[0] * h[1] * h[2] / 8.0
        return float(np.sum(W * rho(P)))

    o, h = mesh.origin(key), mesh.h(key)
    whole = integral(o, h)
    parts = 0.0
    for c in range(8):
        off = np.array([c & 1, (c >> 1) & 1, c >> 2], dtype=np.float64) * h / 2.0
        parts += integral(o + off, h / 2.0)
    return abs(whole - parts)


def refine_to_density(mesh, rho, delta, max_level):
    """Split every leaf whose indicator exceeds delta (below max_level), keep
    the tree 2:1 balanced, and repeat until no leaf is split."""
    while True:
        split = [k for k in mesh.leaves if k[0] < max_level and density_indicator(mesh, k, rho) > delta]
        if not split:
            return mesh
        mesh.refine(split)
        mesh.balance()


def coulomb_boundary_data(mesh, f):
    """The Dirichlet data of Sec. 6.3 as a callable: g(x) = sum_q W_q f_q / |x - x_q|
    over the octree's nodes (the quadrature sum of the free-space potential)."""
    xq = mesh.node_coords()
    wf = mesh.quad_weights() * np.asarray(f, dtype=np.float64)

    def g(P):
        P = np.atleast_2d(P)
        out = np.empty(P.shape[0])
        for i0 in range(0, P.shape[0], 256):
            d = np.linalg.norm(P[i0:i0 + 256, None, :] - xq[None, :, :], axis=2)
            out[i0:i0 + 256] = d ** -1 @ wf
        return out

    return g


def poisson(mesh, f, penalty_form=0, eps=0.125):
    """v solving -Lap v = 4 pi f on the octree with the Coulomb-quadrature
    Dirichlet data (dense Cholesky; small meshes only)."""
    import scipy.linalg

    A = assemble(mesh, penalty_form, eps)
    b = rhs(mesh, f, coulomb_boundary_data(mesh, f), penalty_form, eps)
    return scipy.linalg.cho_solve(scipy.linalg.cho_factor(A), b)


def exchange_build(mesh, psi, penalty_form=0, eps=0.125):
    """Hartree solve, pair solves, W_j = sum_s psi_s v_sj, K = Psi^T diag(W_q) W,
    E_H and E_X (Sec. 6.1, eq. fock_exchange) on the octree; the same source
    list and conventions as the uniform oracle's exchange_build."""
    import scipy.linalg

    psi = np.asarray(psi, dtype=np.float64)
    N = psi.shape[0]
    Wq = mesh.quad_weights()
    A = scipy.linalg.cho_factor(assemble(mesh, penalty_form, eps))

    def solve(f):
        return scipy.linalg.cho_solve(A, rhs(mesh, f, coulomb_boundary_data(mesh, f), penalty_form, eps))

    rho = np.sum(psi * psi, axis=0)
    vH = solve(rho)
    Wacc = np.zeros_like(psi)
    for i in range(N):
        for j in range(i, N):
            v = solve(psi[i] * psi[j])
            Wacc[j] += psi[i] * v
            if i != j:
                Wacc[i] += psi[j] * v
    K = (psi * Wq[None, :]) @ Wacc.T
    return {"K": K, "E_H": 0.5 * float(np.sum(Wq * rho * vH)), "E_X": -0.5 * float(np.trace(K)), "W": Wacc,
            "v_H": vH}
