"""Tight-binding Hamiltonians H0 and dipole perturbations H1 (orthogonal basis).

Every generator is deterministic in its seed (numpy ``default_rng``) and
returns FP64 arrays. The shapes and value distributions follow the workloads
the method is exercised on: an open 1D chain, periodic simple-cubic lattices
with on-site and bond disorder, a random symmetric banded matrix and a batch
of disordered 3D clusters with three dipole directions.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Problem:
    """One Hamiltonian with D perturbation directions and its solve settings."""

    name: str
    H0: np.ndarray                 # (N, N) symmetric FP64
    H1: np.ndarray                 # (D, N, N) symmetric FP64
    nocc: float                    # target occupation Tr P0
    beta: float                    # inverse electronic temperature
    n: int                         # recursion steps
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.H0.shape[0])

    @property
    def D(self) -> int:
        return int(self.H1.shape[0])


def _symmetric_from_upper(rows, cols, vals, N):
    H = np.zeros((N, N))
    np.add.at(H, (rows, cols), vals)
    np.add.at(H, (cols, rows), vals)
    return H


def chain_1d(N: int = 64, seed: int = 1001, beta: float = 10.0, n: int = 12) -> Problem:
    """Open 1D chain: on-site eps_i ~ U[-1, 1], hopping -1, H1 = diag(i - (N-1)/2)."""
    rng = np.random.default_rng(seed)
    eps = rng.uniform(-1.0, 1.0, size=N)
    H0 = np.diag(eps)
    idx = np.arange(N - 1)
    H0[idx, idx + 1] = -1.0
    H0[idx + 1, idx] = -1.0
    x = np.arange(N, dtype=np.float64) - (N - 1) / 2.0
    H1 = np.diag(x)[None]
    return Problem("chain_1d", H0, H1, nocc=N / 2.0, beta=beta, n=n,
                   meta={"seed": seed})


def cubic_lattice(L=(16, 16, 16), seed: int = 1002, beta: float = 20.0, n: int = 14,
                  onsite_sigma: float = 0.3, bond_disorder: float = 0.1,
                  periodic: bool = True, directions: str = "x") -> Problem:
    """Simple-cubic s-orbital lattice, site index i = (ix * Ly + iy) * Lz + iz.

    On-site eps ~ N(0, onsite_sigma^2); every nearest-neighbour bond gets
    hopping -(1 + U[-bond_disorder, bond_disorder]); periodic wrap when
    ``periodic``. H1 holds one diagonal dipole operator per letter of
    ``directions`` (site coordinate along that axis, centred).
    """
    Lx, Ly, Lz = (int(v) for v in L)
    N = Lx * Ly * Lz
    rng = np.random.default_rng(seed)
    eps = rng.normal(0.0, onsite_sigma, size=N)
    ix, iy, iz = np.meshgrid(np.arange(Lx), np.arange(Ly), np.arange(Lz), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    site = lambda a, b, c: (a * Ly + b) * Lz + c  # noqa: E731
    rows, cols = [], []
    for (dx, dy, dz, Lax, coord) in ((1, 0, 0, Lx, ix), (0, 1, 0, Ly, iy), (0, 0, 1, Lz, iz)):
        if periodic:
            if Lax < 3:
                keep = coord + 1 < Lax
            else:
                keep = np.ones(N, dtype=bool)
        else:
            keep = coord + 1 < Lax
        a = ix[keep]; b = iy[keep]; c = iz[keep]
        rows.append(site(a, b, c))
        cols.append(site((a + dx) % Lx, (b + dy) % Ly, (c + dz) % Lz))
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    hop = -(1.0 + rng.uniform(-bond_disorder, bond_disorder, size=rows.size))
    H0 = _symmetric_from_upper(rows, cols, hop, N) + np.diag(eps)
    coords = {"x": ix - (Lx - 1) / 2.0, "y": iy - (Ly - 1) / 2.0, "z": iz - (Lz - 1) / 2.0}
    H1 = np.stack([np.diag(coords[d].astype(np.float64)) for d in directions])
    return Problem(f"cubic_{Lx}x{Ly}x{Lz}", H0, H1, nocc=N / 2.0, beta=beta, n=n,
                   meta={"seed": seed, "L": (Lx, Ly, Lz)})


def banded_random(N: int = 8192, bandwidth: int = 64, seed: int = 1004, beta: float = 20.0,
                  n: int = 14) -> Problem:
    """Random symmetric banded H0: entries |i-j| <= bandwidth drawn N(0,1)/sqrt(bandwidth)."""
    rng = np.random.default_rng(seed)
    H0 = np.zeros((N, N))
    scale = 1.0 / np.sqrt(bandwidth)
    for d in range(bandwidth + 1):
        v = rng.normal(0.0, 1.0, size=N - d) * scale
        i = np.arange(N - d)
        H0[i, i + d] = v
        H0[i + d, i] = v
    x = np.arange(N, dtype=np.float64) - (N - 1) / 2.0
    return Problem("banded", H0, np.diag(x)[None], nocc=N / 2.0, beta=beta, n=n,
                   meta={"seed": seed, "bandwidth": bandwidth})


def _cluster(Nb: int, seed: int, beta: float, n: int) -> Problem:
    rng = np.random.default_rng(seed)
    side = Nb ** (1.0 / 3.0)
    pos = rng.uniform(0.0, side, size=(Nb, 3))
    eps = rng.normal(0.0, 0.3, size=Nb)
    diff = pos[:, None, :] - pos[None, :, :]
    r = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
    H0 = np.where((r < 2.5) & (r > 0.0), -np.exp(-2.0 * (r - 1.0)), 0.0)
    H0 = 0.5 * (H0 + H0.T)
    H0[np.diag_indices(Nb)] = eps
    centred = pos - pos.mean(axis=0)
    H1 = np.stack([np.diag(centred[:, a]) for a in range(3)])
    return Problem(f"cluster_{Nb}", H0, H1, nocc=float(Nb // 2), beta=beta, n=n,
                   meta={"seed": seed})


def nonorthogonal_cluster(Nb: int = 256, seed: int = 2001, beta: float = 20.0, n: int = 14,
                          s0: float = 0.3, sigma: float = 0.8) -> Problem:
    """Non-orthogonal s-orbital cluster (extended-Hueckel-like), the input of Eq. Fermi_D.

    Sites uniform in a cube of side Nb^(1/3) (unit density). Overlap
    S = (1 - s0) I + s0 G with the Gaussian kernel G_ij = exp(-r_ij^2 / (2 sigma^2)), which
    is positive semidefinite, so S is positive definite with eigenvalues >= 1 - s0. Fockian
    F_ii = eps_i ~ N(0, 0.3^2), F_ij = -4 S_ij. Dipoles in the Mulliken form
    (h1)_ij = S_ij (x_i + x_j) / 2 for x, y, z (centred coordinates). F is returned as H0,
    the dipoles as H1 and S in meta["S"]; N_occ = Nb / 2. For the self-consistent charge
    model, meta["gamma"] = U exp(-r^2 / (2 a^2)) (U = 0.5, a = 1; a positive semidefinite
    Gaussian kernel) and meta["q0"] = 1 per site (neutral at half filling).
    """
    rng = np.random.default_rng(seed)
    side = Nb ** (1.0 / 3.0)
    pos = rng.uniform(0.0, side, size=(Nb, 3))
    eps = rng.normal(0.0, 0.3, size=Nb)
    diff = pos[:, None, :] - pos[None, :, :]
    r2 = np.einsum("ijk,ijk->ij", diff, diff)
    S = (1.0 - s0) * np.eye(Nb) + s0 * np.exp(-r2 / (2.0 * sigma * sigma))
    S = 0.5 * (S + S.T)
    F = -4.0 * S
    F[np.diag_indices(Nb)] = eps
    c = pos - pos.mean(axis=0)
    H1 = np.stack([S * 0.5 * (c[:, a][:, None] + c[:, a][None, :]) for a in range(3)])
    gamma = 0.5 * np.exp(-r2 / 2.0)
    return Problem(f"nonorth_cluster_{Nb}", F, H1, nocc=float(Nb // 2), beta=beta, n=n,
                   meta={"seed": seed, "S": S, "gamma": 0.5 * (gamma + gamma.T),
                         "q0": np.ones(Nb)})


def cluster_sizes(B: int = 96, seed: int = 1005, nmin: int = 128, nmax: int = 1536) -> List[int]:
    """The sizes N_b ~ U{nmin..nmax} that clusters() draws (without building the systems)."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.integers(nmin, nmax + 1, size=B)]


def clusters(B: int = 96, seed: int = 1005, nmin: int = 128, nmax: int = 1536,
             beta: float = 20.0, n: int = 12, sizes: Optional[List[int]] = None) -> List[Problem]:
    """B disordered 3D clusters of uneven size, three dipole directions each."""
    if sizes is None:
        sizes = cluster_sizes(B, seed, nmin, nmax)
    return [_cluster(Nb, seed + b, beta, n) for b, Nb in enumerate(sizes)]


WORKLOADS = {
    # 1D chain, FP64 path
    "chain64": lambda: chain_1d(64, 1001, 10.0, 12),
    # 16^3 periodic lattice at three temperatures
    "cubic16_b5": lambda: cubic_lattice((16, 16, 16), 1002, 5.0, 14),
    "cubic16_b20": lambda: cubic_lattice((16, 16, 16), 1002, 20.0, 14),
    "cubic16_b80": lambda: cubic_lattice((16, 16, 16), 1002, 80.0, 14),
    # mixed-precision sizes
    "cubic20_b20": lambda: cubic_lattice((20, 20, 20), 1003, 20.0, 14),
    "banded8192": lambda: banded_random(8192, 64, 1004, 20.0, 14),
    # adjoint workload: 16x16x8 lattice, n = 16
    "cubic16x16x8": lambda: cubic_lattice((16, 16, 8), 1006, 20.0, 16),
}


def workload(name: str) -> Problem:
    return WORKLOADS[name]()
