"""Seeded synthetic NAO-like (H, S) pairs on a shared sparse pattern.

This module only draws inputs. It holds none of the PEXSI arithmetic (no
pole expansion, no factorisation, no inversion) so that both the CPU oracle
and the CUDA path can consume the same inputs without sharing any code of
the method.

The generators stand in for the SIESTA-produced Hamiltonians of the paper's
test systems (Sec. III, Table I and Table II: DNA chains, C-BN sheets and
liquid water), which are not available here. Recipe (all energies in Ha,
lengths in bohr):

* atoms carry ``norb`` orbitals each (13 for "heavy", 5 for "H", 4 for the
  tiny chain);
* every atom pair (I, J), I != J, whose minimum-image distance r is within
  the cutoff gets an H block of entries N(0,1) * exp(-r / lam) and an S block
  of entries 0.05 * N(0,1) * exp(-r / lam); the (J, I) block is the
  transpose, so H and S are symmetric;
* the on-site block of H has diagonal entries U[-1, 1] and off-diagonal
  entries 0.1 * N(0,1) (symmetrised), which couples all orbitals of one atom
  so that they share one sparsity structure;
* S has an identity on-site block; it is made SPD by diagonal dominance,
  S_ii = 1 + sum_j |S_ij| + 0.1;
* the stored pattern is the full symmetric pattern of H (S's pattern is a
  subset; S is stored as explicit zeros outside its own blocks), 0-based CSC
  with sorted row indices and the diagonal present.

Values come from ``numpy.random.default_rng(seed)`` in a fixed order, so a
(kind, size, seed) triple always gives bit-identical inputs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903


@dataclasses.dataclass
class System:
    """One synthetic system on a shared CSC pattern."""

    name: str
    n: int
    colptr: np.ndarray  # int64, n + 1
    rowind: np.ndarray  # int32, nnz
    H: np.ndarray  # float64, nnz, CSC order
    S: np.ndarray  # float64, nnz, CSC order
    norb: np.ndarray  # int32, orbitals per atom
    positions: np.ndarray  # float64 (natoms, 3), bohr (debug only)
    seed: int
    beta: float
    n_poles: int
    params: dict

    @property
    def nnz(self) -> int:
        return int(self.rowind.shape[0])

    def to_scipy(self, which: str = "H") -> sp.csc_matrix:
        vals = self.H if which == "H" else self.S
        return sp.csc_matrix((vals, self.rowind, self.colptr), shape=(self.n, self.n))


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------

def chain_positions(natoms: int, spacing: float) -> np.ndarray:
    pos = np.zeros((natoms, 3))
    pos[:, 0] = spacing * np.arange(natoms)
    return pos


def honeycomb_positions(ncell: int, bond_angstrom: float = 1.42):
    """Periodic ncell x ncell honeycomb sheet, two atoms per rhombic cell."""
    a = bond_angstrom * math.sqrt(3.0) * BOHR_PER_ANGSTROM  # lattice constant
    a1 = np.array([a, 0.0, 0.0])
    a2 = np.array([0.5 * a, 0.5 * math.sqrt(3.0) * a, 0.0])
    basis = [np.zeros(3), (a1 + a2) / 3.0]
    pos = []
    for i in range(ncell):
        for j in range(ncell):
            for b in basis:
                pos.append(i * a1 + j * a2 + b)
    lattice = np.stack([ncell * a1, ncell * a2, np.array([0.0, 0.0, 1.0e6])])
    return np.asarray(pos), lattice


def fluid_positions(rng: np.random.Generator, natoms: int, box: float, dmin: float) -> np.ndarray:
    """Uniform random positions in a periodic cube with a minimum separation."""
    pos = np.zeros((natoms, 3))
    k = 0
    tries = 0
    while k < natoms:
        cand = rng.uniform(0.0, box, size=3)
        if k:
            d = pos[:k] - cand
            d -= box * np.round(d / box)
            if np.min(np.einsum("ij,ij->i", d, d)) < dmin * dmin:
                tries += 1
                if tries > 200000:
                    raise RuntimeError("fluid packing failed; lower the density")
                continue
        pos[k] = cand
        k += 1
    return pos


def _pairs(pos: np.ndarray, cutoff: float, lattice: np.ndarray | None):
    """All atom pairs I < J with minimum-image distance <= cutoff, sorted."""
    natoms = pos.shape[0]
    inv = np.linalg.inv(lattice) if lattice is not None else None
    I_list, J_list, R_list = [], [], []
    chunk = max(1, 4_000_000 // max(natoms, 1))
    for i0 in range(0, natoms, chunk):
        i1 = min(natoms, i0 + chunk)
        d = pos[None, :, :] - pos[i0:i1, None, :]
        if lattice is not None:
            f = d @ inv
            f -= np.round(f)
            d = f @ lattice
        r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
        ii, jj = np.nonzero(r <= cutoff)
        ii = ii + i0
        keep = jj > ii
        I_list.append(ii[keep]); J_list.append(jj[keep]); R_list.append(r[ii[keep] - i0, jj[keep]])
    I = np.concatenate(I_list); J = np.concatenate(J_list); R = np.concatenate(R_list)
    order = np.lexsort((J, I))
    return I[order], J[order], R[order]


# ----------------------------------------------------------------------------
# matrices
# ----------------------------------------------------------------------------

def _assemble(rng, norb, pos, cutoff, lam, lattice):
    natoms = norb.shape[0]
    first = np.zeros(natoms + 1, dtype=np.int64)
    first[1:] = np.cumsum(norb)
    n = int(first[-1])
    I, J, R = _pairs(pos, cutoff, lattice)

    # --- on-site blocks: diagonal U[-1,1]; off-diagonal 0.1*N(0,1), symmetrised
    onsite_diag = rng.uniform(-1.0, 1.0, size=n)
    osz = norb.astype(np.int64) ** 2
    onsite_raw = 0.1 * rng.standard_normal(int(osz.sum()))
    a_of = np.repeat(np.arange(natoms), osz)
    t = np.arange(int(osz.sum())) - np.repeat(np.cumsum(osz) - osz, osz)
    k_of = norb.astype(np.int64)[a_of]
    li, lj = t // k_of, t % k_of
    o_rows = first[a_of] + li
    o_cols = first[a_of] + lj
    # symmetrise: value(i,j) = (raw(i,j) + raw(j,i)) / 2
    base = np.repeat(np.cumsum(osz) - osz, osz)
    o_h = 0.5 * (onsite_raw + onsite_raw[base + lj * k_of + li])
    diag = li == lj
    o_h[diag] = onsite_diag[o_rows[diag]]
    o_s = np.where(diag, 1.0, 0.0)

    # --- pair blocks in sorted (I, J) order: all H entries, then all S entries
    ka = norb.astype(np.int64)[I]; kb = norb.astype(np.int64)[J]
    psz = ka * kb
    tot = int(psz.sum())
    decay = np.exp(-R / lam)
    hraw = rng.standard_normal(tot)
    sraw = 0.05 * rng.standard_normal(tot)
    p_of = np.repeat(np.arange(I.shape[0]), psz)
    t = np.arange(tot) - np.repeat(np.cumsum(psz) - psz, psz)
    kbp = kb[p_of]
    p_rows = first[I][p_of] + t // kbp
    p_cols = first[J][p_of] + t % kbp
    p_h = hraw * decay[p_of]
    p_s = sraw * decay[p_of]

    rows = np.concatenate([o_rows, p_rows, p_cols])
    cols = np.concatenate([o_cols, p_cols, p_rows])
    hv = np.concatenate([o_h, p_h, p_h])
    sv = np.concatenate([o_s, p_s, p_s])
    # CSC with sorted rows; H and S ride together as the real and imaginary
    # parts of one complex value so they keep identical positions.
    M = sp.coo_matrix((hv + 1j * sv, (rows, cols)), shape=(n, n)).tocsc()
    M.sort_indices()
    rows = M.indices.astype(np.int32)
    cols = np.repeat(np.arange(n), np.diff(M.indptr))
    hv = M.data.real.copy(); sv = M.data.imag.copy()
    # S diagonal dominance: S_ii = 1 + sum_{j != i} |S_ij| + 0.1
    off = rows != cols
    absrow = np.bincount(cols[off], weights=np.abs(sv[off]), minlength=n)
    dpos = ~off
    sv[dpos] = 1.0 + absrow[cols[dpos]] + 0.1
    colptr = M.indptr.astype(np.int64)
    return n, colptr, rows.astype(np.int32), hv.astype(np.float64), sv.astype(np.float64)


def make_chain(natoms: int = 64, seed: int = 0, norb: int = 4, spacing: float = 2.5,
               cutoff: float = 6.0, lam: float = 2.0, beta: float = 1000.0, n_poles: int = 40) -> System:
    """1D chain (the tiny plain-method case: 64 atoms x 4 orbitals, n = 256)."""
    rng = np.random.default_rng(seed)
    pos = chain_positions(natoms, spacing)
    no = np.full(natoms, norb, dtype=np.int32)
    n, cp, ri, H, S = _assemble(rng, no, pos, cutoff, lam, None)
    return System(f"chain{natoms}", n, cp, ri, H, S, no, pos, seed, beta, n_poles,
                  dict(kind="chain", natoms=natoms, spacing=spacing, cutoff=cutoff, lam=lam))


def make_sheet(ncell: int = 32, seed: int = 0, norb: int = 13, cutoff_angstrom: float = 8.0,
               lam: float = 3.0, beta: float = 2000.0, n_poles: int = 60) -> System:
    """Periodic honeycomb sheet (ncell=32: 2048 atoms x 13 orbitals, n = 26,624)."""
    rng = np.random.default_rng(seed)
    pos, lattice = honeycomb_positions(ncell)
    no = np.full(pos.shape[0], norb, dtype=np.int32)
    cutoff = cutoff_angstrom * BOHR_PER_ANGSTROM
    n, cp, ri, H, S = _assemble(rng, no, pos, cutoff, lam, lattice)
    return System(f"sheet{ncell}x{ncell}", n, cp, ri, H, S, no, pos, seed, beta, n_poles,
                  dict(kind="sheet", ncell=ncell, cutoff=cutoff, lam=lam))


def make_fluid(nmol: int = 512, seed: int = 0, cutoff: float = 10.0, lam: float = 3.0,
               beta: float = 1000.0, n_poles: int = 60, dmin: float = 2.0) -> System:
    """Periodic water-like fluid: nmol 'O' (13 orb) + 2 nmol 'H' (5 orb).

    nmol = 512 gives 1536 atoms and n = 11,776 in a cube of side
    46.9 * (nmol / 512)^(1/3) bohr (liquid-water molecular density).
    """
    rng = np.random.default_rng(seed)
    box = 46.9 * (nmol / 512.0) ** (1.0 / 3.0)
    natoms = 3 * nmol
    pos = fluid_positions(rng, natoms, box, dmin)
    no = np.array([13] * nmol + [5] * (2 * nmol), dtype=np.int32)
    lattice = np.diag([box, box, box])
    n, cp, ri, H, S = _assemble(rng, no, pos, cutoff, lam, lattice)
    return System(f"fluid{nmol}", n, cp, ri, H, S, no, pos, seed, beta, n_poles,
                  dict(kind="fluid", nmol=nmol, box=box, cutoff=cutoff, lam=lam))


def hermitian_from(sys: System, seed: int, imag_scale: float = 0.25):
    """Complex Hermitian H and S on the pattern of `sys` (the k-point /
    spin-orbit variant): H' = H + i A and S' = S + i B, with A and B real
    antisymmetric (A_ij = -A_ji, zero diagonal) of magnitude imag_scale |H_ij|
    and imag_scale |S_ij| / 2 times N(0,1). The diagonal of S' is reset to
    1 + sum_{j != i} |S'_ij| + 0.1, so that S' is Hermitian, strictly
    diagonally dominant with a positive diagonal, hence positive definite.
    Returns (H', S') as complex128 arrays of nnz values in CSC order."""
    rng = np.random.default_rng(seed)
    n, colptr, rowind = sys.n, sys.colptr, sys.rowind
    cols = np.repeat(np.arange(n), np.diff(colptr))
    off = rowind != cols

    def antisym(mag):
        raw = np.where(off, mag * rng.standard_normal(sys.nnz), 0.0)
        t = sp.csc_matrix((raw, rowind, colptr), shape=(n, n)).T.tocsc()
        t.sort_indices()
        # the pattern is symmetric, so the transpose has the same CSC structure
        assert np.array_equal(t.indptr, colptr) and np.array_equal(t.indices, rowind)
        return 0.5 * (raw - t.data)

    Hc = sys.H + 1j * antisym(imag_scale * np.abs(sys.H))
    Sc = sys.S + 1j * antisym(0.5 * imag_scale * np.abs(sys.S))
    absrow = np.bincount(cols[off], weights=np.abs(Sc[off]), minlength=n)
    diag = ~off
    Sc[diag] = 1.0 + absrow[cols[diag]] + 0.1
    return Hc.astype(np.complex128), Sc.astype(np.complex128)


def spectral_interval(sys: System, dense_limit: int = 4096, margin: float = 0.05):
    """Bounds [E_min, E_max] of the generalised spectrum of (H, S).

    Exact (dense symmetric-definite eigensolver) up to ``dense_limit``,
    otherwise LOBPCG estimates widened by ``margin`` of the width. This is
    input preparation (choosing mu mid-spectrum and Delta E), not part of
    the method.
    """
    import scipy.linalg as sla
    import scipy.sparse.linalg as spla
    Hm = sys.to_scipy("H"); Sm = sys.to_scipy("S")
    if sys.n <= dense_limit:
        ev = sla.eigh(Hm.toarray(), Sm.toarray(), eigvals_only=True)
        return float(ev[0]), float(ev[-1])
    rng = np.random.default_rng(12345)
    X = rng.standard_normal((sys.n, 4))
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        lo = spla.lobpcg(Hm, X, B=Sm, largest=False, maxiter=120, tol=1e-5)[0][0]
        hi = spla.lobpcg(Hm, X, B=Sm, largest=True, maxiter=120, tol=1e-5)[0][0]
    w = hi - lo
    return float(lo - margin * w), float(hi + margin * w)


def mu_and_delta_e(sys: System, **kw):
    """mu at the centre of the spectral interval, Delta E its half-width +10%."""
    lo, hi = spectral_interval(sys, **kw)
    mu = 0.5 * (lo + hi)
    return mu, 0.55 * (hi - lo)


CONFIGS = {
    "chain": make_chain,
    "sheet": make_sheet,
    "fluid": make_fluid,
}
