"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measured "randomly generated proteins" of 1k-100k atoms (Section III,
Table 1) and argued for the direct sum on elongated DNA/RNA-like structures and
sparse pseudo-atom models (Abstract; Section I-A).  None of its molecules ship,
so these generators stand in for them.  They draw positions, atom types,
form-factor coefficients, q grids and per-atom form-factor tables (an input of
their own, drawn from a recipe stated below, not from the type coefficients):
nothing here evaluates the method's type form factor, a distance or a sinc, so
the CPU oracle and the CUDA library can both be fed from this module without
sharing any of the method's arithmetic.

Every generator takes an explicit integer seed and uses NumPy's PCG64
(``np.random.default_rng``), so a (generator, seed) pair names an input
exactly, on x86 and on Arm alike.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 1306


def seed_for(config: int, index: int = 0) -> int:
    """Seed of input ``index`` of workload family ``config`` (1..5; 6 for Table 1's workload)."""
    return BASE_SEED + 1000 * config + index


@dataclass
class Molecule:
    """One synthetic molecule: positions [n,3] (Å), types [n] int32 in [0, n_types)."""

    coords: np.ndarray
    types: np.ndarray
    n_types: int
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.coords.shape[0])

    def as_f32(self) -> "Molecule":
        return Molecule(self.coords.astype(np.float32), self.types, self.n_types, self.name)


# ----------------------------------------------------------------------------
# form-factor coefficients and q grids
# ----------------------------------------------------------------------------

def form_factor_coefficients(n_types: int, seed: int) -> np.ndarray:
    """Coefficients [n_types, 9] = (a1..a4, b1..b4, c) of the synthetic form factor
    f(q) = sum_k a_k exp(-b_k (q/4pi)^2) + c.

    The paper gives no formula for f_j(q) (Section I-A, after Eq. 1); this
    four-Gaussian-plus-constant shape and its ranges a_k in U[0.5, 3],
    b_k in U[0.5, 40] Å^2, c in U[0, 0.5] are the stated synthetic stand-in.
    Drawn per type in the order a[4], b[4], c.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((n_types, 9), dtype=np.float64)
    for t in range(n_types):
        out[t, 0:4] = rng.uniform(0.5, 3.0, size=4)
        out[t, 4:8] = rng.uniform(0.5, 40.0, size=4)
        out[t, 8] = rng.uniform(0.0, 0.5)
    return out


def atomic_form_factor_table(n: int, q: np.ndarray, seed: int, shell_fraction: float = 0.3) -> np.ndarray:
    """Per-atom form factors ff[k, i] = f_i(q_k), shape [n_q, n], for the per-atom path (no types).

    Stand-in for vacuum form factors corrected for excluded volume plus a hydration shell, the
    case where the products f_k f_j do not reduce to a few types (Section I-A, after Eq. 2): each
    atom draws its own shape a_i exp(-b_i q^2) + c_i with a_i in U[1, 8], b_i in U[0.02, 0.5] Å^2,
    c_i in U[-0.3, 0.3]; a fraction ``shell_fraction`` of the atoms (the surface, in a water
    layer) add d_i exp(-0.6 q^2) with d_i in U[-1, 1.5].  Drawn in the order a, b, c, shell mask, d.
    """
    rng = np.random.default_rng(seed)
    qq = np.asarray(q, dtype=np.float64)[:, None]
    a = rng.uniform(1.0, 8.0, size=n)
    b = rng.uniform(0.02, 0.5, size=n)
    c = rng.uniform(-0.3, 0.3, size=n)
    shell = rng.uniform(size=n) < shell_fraction
    d = np.where(shell, rng.uniform(-1.0, 1.5, size=n), 0.0)
    return np.ascontiguousarray(a * np.exp(-b * qq * qq) + c + d * np.exp(-0.6 * qq * qq))


def q_grid(lo: float, hi: float, n: int) -> np.ndarray:
    """Uniform q grid, both ends included (Å^-1)."""
    return np.linspace(lo, hi, n, dtype=np.float64)


# ----------------------------------------------------------------------------
# chains
# ----------------------------------------------------------------------------

def globule_radius(n: int) -> float:
    """Confining radius 30 (N/1000)^(1/3) Å of the random-walk globule."""
    return 30.0 * (n / 1000.0) ** (1.0 / 3.0)


def _unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def random_walk_globule(n: int, n_types: int, seed: int, bond: float = 3.8,
                        radius: float | None = None) -> Molecule:
    """Confined 3D random walk: start at the origin, steps of ``bond`` Å in a
    uniformly random direction; a step that leaves the sphere of ``radius`` is
    redrawn (at most 1000 tries, then the step points at the origin).  No
    excluded volume, so near-coincident atoms do occur.  Types are i.i.d.
    uniform over ``n_types``.
    """
    rng = np.random.default_rng(seed)
    R = globule_radius(n) if radius is None else float(radius)
    xyz = np.zeros((n, 3), dtype=np.float64)
    p = np.zeros(3)
    for i in range(1, n):
        for _ in range(1000):
            cand = p + bond * _unit(rng)
            if cand @ cand <= R * R:
                break
        else:
            nrm = np.linalg.norm(p)
            cand = p - bond * p / nrm if nrm > 0 else p + bond * _unit(rng)
        p = cand
        xyz[i] = p
    types = rng.integers(0, n_types, size=n).astype(np.int32)
    return Molecule(xyz, types, n_types, f"globule{n}")


def free_chain(n: int, n_types: int, seed: int, bond: float = 6.0) -> Molecule:
    """Unconfined ideal random walk (sparse pseudo-atom chain), ``bond`` Å steps."""
    rng = np.random.default_rng(seed)
    steps = rng.standard_normal((n - 1, 3))
    steps *= bond / np.linalg.norm(steps, axis=1, keepdims=True)
    xyz = np.zeros((n, 3), dtype=np.float64)
    np.cumsum(steps, axis=0, out=xyz[1:])
    types = rng.integers(0, n_types, size=n).astype(np.int32)
    return Molecule(xyz, types, n_types, f"chain{n}")


def double_helix_rod(seed: int, n_steps: int = 1500, rise: float = 3.4,
                     twist_deg: float = 36.0, atoms_per_strand: int = 10,
                     jitter: float = 0.3, n_types: int = 5) -> Molecule:
    """Double-helix rod: at step s the two strands sit at azimuth
    phi_s = s*twist and phi_s + 180 deg, height rise*s; each strand carries
    ``atoms_per_strand`` atoms at radii (m+1) Å with an extra azimuth of 3 deg*m;
    type = m mod n_types; Gaussian jitter ``jitter`` Å.  1500 steps x 2 strands
    x 10 atoms = 30,000 atoms, about 5,100 Å long, radius 10 Å.
    """
    rng = np.random.default_rng(seed)
    s = np.arange(n_steps, dtype=np.float64)[:, None, None]
    k = np.arange(2, dtype=np.float64)[None, :, None]
    m = np.arange(atoms_per_strand, dtype=np.float64)[None, None, :]
    phi = np.deg2rad(twist_deg * s + 180.0 * k + 3.0 * m)
    rho = (m + 1.0) * (10.0 / atoms_per_strand)
    shape = (n_steps, 2, atoms_per_strand)
    x = np.broadcast_to(rho * np.cos(phi), shape)
    y = np.broadcast_to(rho * np.sin(phi), shape)
    z = np.broadcast_to(rise * s, shape)
    xyz = np.stack([x, y, z], axis=-1).reshape(-1, 3).copy()
    xyz += rng.normal(0.0, jitter, size=xyz.shape)
    types = np.broadcast_to(np.arange(atoms_per_strand) % n_types, shape).reshape(-1).astype(np.int32)
    return Molecule(xyz, types, n_types, "helix_rod")


def cubic_lattice(n_side: int, spacing: float, n_types: int, seed: int) -> Molecule:
    """Simple cubic lattice of n_side^3 atoms, ``spacing`` Å apart, centred on the origin; types
    i.i.d. uniform.  Every squared distance is spacing^2 times an integer, so very many pairs
    share one distance exactly: a crystalline stress case for the FP32 recurrence, where the
    rounding of equal pairs can add up coherently.  With spacing 6.5 Å the (100) reflection
    2 pi / spacing = 0.967 Å^-1 falls inside a 0-1 Å^-1 grid."""
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side, dtype=np.float64) - 0.5 * (n_side - 1)) * spacing
    xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3).copy()
    types = rng.integers(0, n_types, size=xyz.shape[0]).astype(np.int32)
    return Molecule(xyz, types, n_types, f"lattice{n_side}")


def spherical_shell(n: int, radius: float, n_types: int, seed: int) -> Molecule:
    """``n`` atoms uniformly at random on one sphere of ``radius`` Å (a thin hollow shell, like
    an empty viral capsid), types i.i.d. uniform.  Its amplitude is close to sum_t n_t f_t
    sinc(q radius), so I(q) falls by about 1/n at the zeros of sinc(q radius): deep minima where
    the pair sum cancels almost completely."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    xyz = radius * v / np.linalg.norm(v, axis=1, keepdims=True)
    types = rng.integers(0, n_types, size=n).astype(np.int32)
    return Molecule(xyz, types, n_types, f"shell{n}")


def subsample(mol: Molecule, n: int, seed: int) -> Molecule:
    """Seeded uniform sample of ``n`` atoms without replacement, types kept,
    original order kept."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(mol.n, size=n, replace=False))
    return Molecule(mol.coords[idx].copy(), mol.types[idx].copy(), mol.n_types,
                    f"{mol.name}_sub{n}")


def perturbed(mol: Molecule, sigma: float, seed: int) -> Molecule:
    """Copy of ``mol`` with i.i.d. Gaussian displacements of std ``sigma`` Å."""
    rng = np.random.default_rng(seed)
    return Molecule(mol.coords + rng.normal(0.0, sigma, size=mol.coords.shape),
                    mol.types.copy(), mol.n_types, f"{mol.name}_pert")


def _rotation(rng: np.random.Generator) -> np.ndarray:
    """Haar-random rotation matrix (QR of a Gaussian matrix, sign-fixed, det +1)."""
    a = rng.standard_normal((3, 3))
    qm, r = np.linalg.qr(a)
    qm = qm * np.sign(np.diag(r))
    if np.linalg.det(qm) < 0:
        qm[:, 0] = -qm[:, 0]
    return qm


def random_rotation(seed: int) -> np.ndarray:
    return _rotation(np.random.default_rng(seed))


def pivot_conformer(base: Molecule, seed: int, radius: float, jitter: float = 0.5,
                    max_pivots: int = 4) -> Molecule:
    """Conformer of a chain made by 1..max_pivots pivot moves: rotate the chain
    tail after a random pivot atom by a Haar-random rotation about that atom,
    rejecting moves that put any atom outside ``radius``; then add Gaussian
    jitter of ``jitter`` Å."""
    rng = np.random.default_rng(seed)
    xyz = base.coords.copy()
    n_piv = int(rng.integers(1, max_pivots + 1))
    done = 0
    tries = 0
    while done < n_piv and tries < 50:
        tries += 1
        p = int(rng.integers(1, base.n - 1))
        rot = _rotation(rng)
        tail = (xyz[p + 1:] - xyz[p]) @ rot.T + xyz[p]
        if np.max(np.einsum("ij,ij->i", tail, tail)) <= radius * radius:
            xyz[p + 1:] = tail
            done += 1
    xyz += rng.normal(0.0, jitter, size=xyz.shape)
    return Molecule(xyz, base.types.copy(), base.n_types, f"{base.name}_conf")


# ----------------------------------------------------------------------------
# named workloads (the five configurations)
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    mol: Molecule
    coef: np.ndarray       # [T, 9] form-factor coefficients
    q: np.ndarray          # [Q] float64
    name: str


def c1_plain_fp64() -> Workload:
    """1,000-atom globule (R = 30 Å), 5 types, q = 0..0.5 Å^-1 with 51 points, FP64."""
    mol = random_walk_globule(1000, 5, seed_for(1, 0))
    return Workload(mol, form_factor_coefficients(5, seed_for(1, 1)), q_grid(0.0, 0.5, 51),
                    "globule 1,000 atoms x 51 q (FP64)")


def c2_globule(n: int) -> Workload:
    """Globule of ``n`` atoms (10,000 or 50,000), 5 types, q = 0..1 Å^-1 with
    201 points, float32 coordinates."""
    mol = random_walk_globule(n, 5, seed_for(2, n)).as_f32()
    return Workload(mol, form_factor_coefficients(5, seed_for(2, 1)), q_grid(0.0, 1.0, 201),
                    f"globule {n:,} atoms x 201 q (mixed)")


def c3_rod() -> Workload:
    mol = double_helix_rod(seed_for(3, 0)).as_f32()
    return Workload(mol, form_factor_coefficients(5, seed_for(3, 1)), q_grid(0.0, 0.5, 101),
                    "double-helix rod 30,000 atoms x 101 q (mixed)")


def c3_sparse(n: int = 200_000) -> Workload:
    mol = free_chain(n, 3, seed_for(3, 2)).as_f32()
    return Workload(mol, form_factor_coefficients(3, seed_for(3, 3)), q_grid(0.0, 0.5, 101),
                    f"sparse bead chain {n:,} beads x 101 q (mixed)")


def c4_refinement(n: int = 5000, batch: int = 64):
    """Base chain, target (base + N(0,1 Å^2)), and ``batch`` conformers
    (base + N(0,1 Å^2)), q = 0.01..0.5 Å^-1 with 101 points."""
    base = random_walk_globule(n, 5, seed_for(4, 0))
    target = perturbed(base, 1.0, seed_for(4, 1))
    confs = np.stack([perturbed(base, 1.0, seed_for(4, 100 + b)).coords for b in range(batch)])
    return dict(base=base, target=target, conformers=confs.astype(np.float32),
                coef=form_factor_coefficients(5, seed_for(4, 2)), q=q_grid(0.01, 0.5, 101))


def table1_globule(n: int) -> Workload:
    """The workload of the paper's Table 1: a "randomly generated protein" of ``n`` atoms (here the
    confined random walk, R = 30 (n/1000)^(1/3) Å, 5 types) and 50-point profiles on 0 < q <= 1 Å^-1,
    read as q_k = 0.02 k for k = 1..50 (Section III)."""
    mol = random_walk_globule(n, 5, seed_for(6, n)).as_f32()
    return Workload(mol, form_factor_coefficients(5, seed_for(6, 1)), q_grid(0.02, 1.0, 50),
                    f"globule {n:,} atoms x 50 q on 0.02..1.0 (Table 1's grid)")


def c5_ensemble(n_conf: int = 4096, n: int = 2000):
    """Conformer family of one ``n``-atom chain made by pivot moves; q = 0..0.5
    Å^-1 with 101 points; the screening target is a separate conformer."""
    base = random_walk_globule(n, 5, seed_for(5, 0))
    R = globule_radius(n)
    confs = np.stack([pivot_conformer(base, seed_for(5, 1000 + c), R).coords
                      for c in range(n_conf)]).astype(np.float32)
    target = pivot_conformer(base, seed_for(5, 999), R).as_f32()
    return dict(base=base, conformers=confs, target=target,
                coef=form_factor_coefficients(5, seed_for(5, 1)), q=q_grid(0.0, 0.5, 101))
