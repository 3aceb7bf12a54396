"""Seeded synthetic inputs: molecular-like Gaussian orbital systems.

This module holds no arithmetic of the discretisation or of the solver: it
draws atoms, Gaussian primitives and coefficients from a seeded generator and
evaluates the resulting orbitals at whatever node coordinates the caller
passes in (optionally Loewdin-orthonormalised in the discrete inner product
given by the caller's quadrature weights). Both the CUDA path and the CPU
oracle are fed from here, so they see identical inputs.

Recipes (the paper uses Gaussian-type orbitals on molecules, Sec. 4.1.2; the
systems below are synthetic stand-ins with the same structure):

* "tiny":    box [-8, 8]^3, 4^3 elements, p = 4; two normalised s-Gaussians of
             exponent 1 centred at (+-0.7, 0, 0) (not orthonormalised).
* "chain10": box [-12, 12]^3, 8^3 elements, p = 6; 10 atoms on the x axis at
             x = -6.3 + 1.4 k; 10 orbitals, seed 2.
* "mixed64": box [-12, 12]^3, 16^3 elements, p = 7; 32 atoms uniform in
             [-6, 6]^3 with minimum separation 1.8; 64 orbitals, seed 3.
* batched systems: box [-12, 12]^3, n in {4, 6, 8, 10, 12}, p in 4..8,
             N in 2..40 orbitals, ceil(N/2) + 1 atoms, one seed per system.

Each atom carries one s and three Cartesian p primitives sharing one exponent
drawn log-uniformly in [0.2, 5]; orbital coefficients are standard normal;
orbitals are Loewdin-orthonormalised, Psi <- (Psi W Psi^T)^(-1/2) Psi.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class MeshSpec:
    lo: tuple
    hi: tuple
    n: tuple
    p: int

    @property
    def n1(self):
        return self.p + 1

    @property
    def Nq(self):
        return self.n[0] * self.n[1] * self.n[2] * self.n1 ** 3


@dataclass
class SystemSpec:
    mesh: MeshSpec
    atoms: np.ndarray  # [A, 3]
    exponents: np.ndarray  # [A] one shell exponent per atom
    coeffs: np.ndarray  # [N, 4A] coefficients of (s, px, py, pz) per atom
    orthonormalise: bool = True
    kind: str = "gto"
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.coeffs.shape[0]


def _random_atoms(rng, n_atoms, half=6.0, min_sep=1.8, max_tries=200000):
    pts = []
    tries = 0
    while len(pts) < n_atoms:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place atoms with the requested separation")
        c = rng.uniform(-half, half, size=3)
        if all(np.linalg.norm(c - q) >= min_sep for q in pts):
            pts.append(c)
    return np.asarray(pts)


def gto_system(mesh, atoms, n_orb, seed, orthonormalise=True):
    rng = np.random.default_rng(seed + 7919)
    A = atoms.shape[0]
    exps = np.exp(rng.uniform(math.log(0.2), math.log(5.0), size=A))
    coeffs = rng.standard_normal((n_orb, 4 * A))
    return SystemSpec(mesh=mesh, atoms=np.asarray(atoms, float), exponents=exps, coeffs=coeffs,
                      orthonormalise=orthonormalise, seed=seed)


def tiny_system():
    """Two normalised s-Gaussians, exponent 1, at (+-0.7, 0, 0)."""
    mesh = MeshSpec((-8.0,) * 3, (8.0,) * 3, (4, 4, 4), 4)
    atoms = np.array([[-0.7, 0.0, 0.0], [0.7, 0.0, 0.0]])
    return SystemSpec(mesh=mesh, atoms=atoms, exponents=np.array([1.0, 1.0]), coeffs=np.eye(2, 8),
                      orthonormalise=False, kind="s_normalised", seed=0)


def chain_system(seed=2, n=8, p=6, n_orb=10):
    mesh = MeshSpec((-12.0,) * 3, (12.0,) * 3, (n, n, n), p)
    atoms = np.array([[-6.3 + 1.4 * k, 0.0, 0.0] for k in range(10)])
    return gto_system(mesh, atoms, n_orb, seed)


def random_system(seed=3, n=16, p=7, n_orb=64, n_atoms=32):
    mesh = MeshSpec((-12.0,) * 3, (12.0,) * 3, (n, n, n), p)
    rng = np.random.default_rng(seed)
    atoms = _random_atoms(rng, n_atoms)
    return gto_system(mesh, atoms, n_orb, seed)


def batched_system(seed):
    """One system of the uneven batch: n, p, N and atoms drawn from `seed`."""
    rng = np.random.default_rng(seed)
    n = int(rng.choice([4, 6, 8, 10, 12]))
    p = int(rng.integers(4, 9))
    n_orb = int(rng.integers(2, 41))
    n_atoms = (n_orb + 1) // 2 + 1
    mesh = MeshSpec((-12.0,) * 3, (12.0,) * 3, (n, n, n), p)
    atoms = _random_atoms(rng, n_atoms)
    return gto_system(mesh, atoms, n_orb, seed)


def named_system(name, seed=None):
    if name == "tiny":
        return tiny_system()
    if name == "chain10":
        return chain_system(seed=2 if seed is None else seed)
    if name == "mixed64":
        return random_system(seed=3 if seed is None else seed)
    raise KeyError(name)


def eval_primitives(spec, coords):
    """[4A, Nq] values of the (s, px, py, pz) primitives of every atom."""
    coords = np.asarray(coords, dtype=np.float64)
    A = spec.atoms.shape[0]
    out = np.empty((4 * A, coords.shape[0]))
    for a in range(A):
        d = coords - spec.atoms[a][None, :]
        r2 = np.einsum("qi,qi->q", d, d)
        g = np.exp(-spec.exponents[a] * r2)
        out[4 * a] = g
        out[4 * a + 1] = d[:, 0] * g
        out[4 * a + 2] = d[:, 1] * g
        out[4 * a + 3] = d[:, 2] * g
    return out


def lowdin(psi, weights):
    """Psi <- S^(-1/2) Psi with S = Psi diag(weights) Psi^T."""
    S = (psi * weights[None, :]) @ psi.T
    lam, U = np.linalg.eigh(S)
    if lam.min() <= 0:
        raise RuntimeError("orbital overlap is not positive definite")
    return (U @ np.diag(lam ** -0.5) @ U.T) @ psi


def orbitals(spec, coords, weights=None):
    """[N, Nq] orbital values at `coords` ([Nq, 3]). `weights` are the
    quadrature weights of the same nodes (needed when orthonormalising)."""
    coords = np.asarray(coords, dtype=np.float64)
    if spec.kind == "s_normalised":
        out = np.empty((spec.atoms.shape[0], coords.shape[0]))
        for a in range(spec.atoms.shape[0]):
            al = spec.exponents[a]
            d = coords - spec.atoms[a][None, :]
            out[a] = (2.0 * al / math.pi) ** 0.75 * np.exp(-al * np.einsum("qi,qi->q", d, d))
        return out
    psi = spec.coeffs @ eval_primitives(spec, coords)
    if spec.orthonormalise:
        if weights is None:
            raise ValueError("orthonormalisation needs the quadrature weights")
        psi = lowdin(psi, np.asarray(weights, dtype=np.float64))
    return psi


def orbitals_torch(spec, coords, weights=None):
    """orbitals() evaluated with torch on the device of `coords` (float64
    [Nq, 3] tensor; `weights` [Nq] tensor), for generating many large systems
    quickly (network training). Same recipe as orbitals()."""
    import torch

    if spec.kind != "gto":
        raise ValueError("only Gaussian-orbital systems")
    dev = coords.device
    atoms = torch.tensor(spec.atoms, dtype=torch.float64, device=dev)
    exps = torch.tensor(spec.exponents, dtype=torch.float64, device=dev)
    C = torch.tensor(spec.coeffs, dtype=torch.float64, device=dev)
    psi = torch.zeros((C.shape[0], coords.shape[0]), dtype=torch.float64, device=dev)
    for a in range(atoms.shape[0]):
        d = coords - atoms[a]
        g = torch.exp(-exps[a] * (d * d).sum(dim=1))
        prim = torch.stack([g, d[:, 0] * g, d[:, 1] * g, d[:, 2] * g])
        psi += C[:, 4 * a:4 * a + 4] @ prim
    if spec.orthonormalise:
        if weights is None:
            raise ValueError("orthonormalisation needs the quadrature weights")
        # the N x N overlap is decomposed on the host (no device linear-algebra library needed)
        S = ((psi * weights[None, :]) @ psi.T).cpu().numpy()
        lam, U = np.linalg.eigh(S)
        if lam.min() <= 0:
            raise RuntimeError("orbital overlap is not positive definite")
        T = torch.tensor((U * lam ** -0.5) @ U.T, dtype=torch.float64, device=dev)
        psi = T @ psi
    return psi
