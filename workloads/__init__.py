"""Seeded synthetic multi-patch Poisson problems (input data only).

This module describes problems the way the paper states them (Sec. 2, Eq. (matching),
the geometry maps G_k: (0,1)^d -> Omega_k, the spline spaces S_{p,h}, and the
Dirichlet/Neumann sides of the model problem): patch corner vertices of multilinear
geometry maps, open uniform knot vectors at the finest level, spline degrees, one
boundary-condition tag per patch side and the number of grid levels.

It holds none of the method's arithmetic (no basis evaluation, no assembly, no dof
numbering).  Both the CPU oracle and the CUDA library read the same `Problem`, and the
random right-hand-side coefficients are drawn here as plain iid numbers once the
caller knows how many active dofs its own numbering has.

Conventions shared by both consumers (they are part of the input format, not of the
method):
  * corner c of patch k is corners[k, c] with c = sum_j c_j 2^j, where c_j in {0,1} is the
    end of the parameter direction j the corner sits at;
  * side s of a patch is direction s // 2 at end s % 2 (order -x,+x,-y,+y,-z,+z);
  * side tags: 0 = AUTO (interface when another patch has the same side, else
    Dirichlet), 1 = DIRICHLET, 2 = NEUMANN.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

SIDE_AUTO, SIDE_DIRICHLET, SIDE_NEUMANN = 0, 1, 2


@dataclass
class Problem:
    dim: int
    degree: np.ndarray          # (K, d) int
    knots: List[List[np.ndarray]]  # knots[k][j]: finest-level knot vector of patch k, dir j
    corners: np.ndarray         # (K, 2**d, d) float64, multilinear geometry control points
    side_bc: np.ndarray         # (K, 2*d) int
    num_levels: int             # L+1, level 0 is the coarsest
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def num_patches(self) -> int:
        return int(self.degree.shape[0])


def open_uniform_knot_vector(m: int, p: int) -> np.ndarray:
    """Input-format helper: the open uniform knot vector with m intervals on [0,1]
    (p+1 repeated end knots, interior knots i/m)."""
    inner = np.arange(1, m, dtype=np.float64) / m
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def _grid_problem(dim, nper, p, m, levels, vertices, bc_of_side, name, meta=None):
    """Patches are the cells of a tensor vertex grid `vertices` of shape nper+1 per axis."""
    cells = [np.array(c) for c in np.ndindex(*([nper] * dim))]
    K = len(cells)
    corners = np.zeros((K, 2 ** dim, dim))
    side_bc = np.zeros((K, 2 * dim), dtype=np.int64)
    for k, cell in enumerate(cells):
        for c in range(2 ** dim):
            off = np.array([(c >> j) & 1 for j in range(dim)])
            corners[k, c] = vertices[tuple(cell + off)]
        for s in range(2 * dim):
            j, e = divmod(s, 2)
            on_boundary = (cell[j] == 0 and e == 0) or (cell[j] == nper - 1 and e == 1)
            side_bc[k, s] = bc_of_side(j, e) if on_boundary else SIDE_AUTO
    degree = np.full((K, dim), p, dtype=np.int64)
    knots = [[open_uniform_knot_vector(m, p) for _ in range(dim)] for _ in range(K)]
    return Problem(dim, degree, knots, corners, side_bc, levels, name, meta or {})


def _vertex_lattice(dim, nper, length):
    axes = [np.linspace(0.0, length, nper + 1)] * dim
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)


def unit_square_quadrants(m: int = 8, p: int = 2, levels: int = 4) -> Problem:
    """[0,1]^2 split into 2x2 quadrants with identity (affine) maps, Dirichlet on the whole
    boundary: the manufactured-solution workload u = sin(pi x) sin(pi y) (K=4, p=2, 8
    intervals per patch direction, V-cycle down to one interval per patch)."""
    verts = _vertex_lattice(2, 2, 1.0)
    return _grid_problem(2, 2, p, m, levels, verts, lambda j, e: SIDE_DIRICHLET,
                         f"square2x2_p{p}_m{m}", {"f": "2pi^2 sin(pi x) sin(pi y)"})


def perturbed_grid_2d(nper: int = 4, p: int = 4, m: int = 256, levels: int = 9,
                      seed: int = 2, length: float = 4.0, amp: float = 0.1) -> Problem:
    """K = nper^2 bilinear patches from a (nper+1)^2 vertex grid on [0,length]^2 whose
    interior vertices move by iid U(-amp, amp) in each coordinate; Dirichlet on x=0 and
    y=0, Neumann on x=length and y=length."""
    rng = np.random.default_rng(seed)
    verts = _vertex_lattice(2, nper, length)
    inner = verts[1:-1, 1:-1]
    verts[1:-1, 1:-1] = inner + rng.uniform(-amp, amp, inner.shape)
    bc = lambda j, e: SIDE_DIRICHLET if e == 0 else SIDE_NEUMANN
    return _grid_problem(2, nper, p, m, levels, verts, bc,
                         f"grid2d_K{nper*nper}_p{p}_m{m}", {"seed": seed})


def perturbed_cube_3d(nper: int = 2, p: int = 3, m: int = 64, levels: int = 7,
                      seed: int = 3, amp: float = 0.05) -> Problem:
    """K = nper^3 trilinear patches of the unit cube; every grid vertex not on the cube
    boundary moves by U(-amp, amp) in all coordinates; vertices on a boundary face move only
    tangentially to it (corners stay fixed), so the domain stays the unit cube; Dirichlet on
    all six faces."""
    rng = np.random.default_rng(seed)
    verts = _vertex_lattice(3, nper, 1.0)
    for idx in np.ndindex(*([nper + 1] * 3)):
        on = [i == 0 or i == nper for i in idx]
        for j in range(3):
            if not on[j]:
                verts[idx + (j,)] += rng.uniform(-amp, amp)
    return _grid_problem(3, nper, p, m, levels, verts, lambda j, e: SIDE_DIRICHLET,
                         f"cube3d_K{nper**3}_p{p}_m{m}", {"seed": seed})


def fichera_corner(split: int = 1, p: int = 2, m: int = 2, levels: int = 2) -> Problem:
    """Fichera corner (0,2)^3 minus [1,2)^3 as 7 unit cubes, each split uniformly into
    split^3 patches; Dirichlet on the faces with xyz=0, Neumann elsewhere."""
    n = 2 * split
    verts = _vertex_lattice(3, n, 2.0)
    cells = []
    for cell in np.ndindex(n, n, n):
        if all(c >= split for c in cell):
            continue  # the removed octant [1,2)^3
        cells.append(np.array(cell))
    K = len(cells)
    corners = np.zeros((K, 8, 3))
    side_bc = np.zeros((K, 6), dtype=np.int64)
    cellset = {tuple(c) for c in cells}
    for k, cell in enumerate(cells):
        for c in range(8):
            off = np.array([(c >> j) & 1 for j in range(3)])
            corners[k, c] = verts[tuple(cell + off)]
        for s in range(6):
            j, e = divmod(s, 2)
            nb = cell.copy()
            nb[j] += 1 if e else -1
            if tuple(nb) in cellset:
                side_bc[k, s] = SIDE_AUTO
            else:
                plane = (cell[j] + e) / split  # coordinate of that side
                side_bc[k, s] = SIDE_DIRICHLET if plane == 0.0 else SIDE_NEUMANN
    degree = np.full((K, 3), p, dtype=np.int64)
    knots = [[open_uniform_knot_vector(m, p) for _ in range(3)] for _ in range(K)]
    return Problem(3, degree, knots, corners, side_bc, levels, f"fichera_s{split}_p{p}_m{m}")


def rhs_coefficients(num_dofs: int, seed: int) -> np.ndarray:
    """iid U(-1,1) spline coefficients of the source term, one per active dof."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, num_dofs)


def batch_problems(count: int = 512, seed: int = 4, m_choices=(16, 32, 64, 128),
                   K_choices=(4, 9, 16, 25, 36), p_range=(2, 6)) -> List[Problem]:
    """Independent 2D problems like the quadrant workload: sqrt(K) x sqrt(K) affine grid
    on [0,1]^2, all Dirichlet, with K, p and intervals per direction drawn uniformly."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        K = int(rng.choice(list(K_choices)))
        p = int(rng.integers(p_range[0], p_range[1] + 1))
        m = int(rng.choice(list(m_choices)))
        nper = int(round(K ** 0.5))
        levels = int(np.log2(m)) + 1
        verts = _vertex_lattice(2, nper, 1.0)
        out.append(_grid_problem(2, nper, p, m, levels, verts, lambda j, e: SIDE_DIRICHLET,
                                 f"batch{i}_K{K}_p{p}_m{m}"))
    return out


def serving_models():
    """Model catalog of the served workload: every 2D problem of the batched family (K in
    {4,9,16,25,36}, p in {2..6}, m in {16,32,64,128}; 100 models) and the 2x2x2 perturbed
    unit cube with p in {2,3}, m in {16,24,32,40,48} (10 models; the coarsest level keeps
    m / 2^k elements per patch direction once m is odd).  Returns (problems, is_3d)."""
    probs, is3d = [], []
    for K in (4, 9, 16, 25, 36):
        for p in range(2, 7):
            for m in (16, 32, 64, 128):
                probs.append(rect_grid_2d(int(round(K ** 0.5)), p, m))
                is3d.append(False)
    for p in (2, 3):
        for m in (16, 24, 32, 40, 48):
            levels, mm = 1, m
            while mm % 2 == 0:
                mm //= 2
                levels += 1
            probs.append(perturbed_cube_3d(2, p, m, levels, 3))
            is3d.append(True)
    return probs, is3d


def serving_requests(is3d, rate: float, count: int, seed: int = 5):
    """Poisson arrivals at `rate` per second: (arrival time s, model index, rhs seed) for
    `count` requests; 80% of the requests pick a 2D model, 20% a 3D model, uniformly."""
    rng = np.random.default_rng([seed, int(rate)])
    two = [i for i, t in enumerate(is3d) if not t]
    three = [i for i, t in enumerate(is3d) if t]
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    out = []
    for i in range(count):
        pool = three if rng.random() < 0.2 else two
        out.append((float(t[i]), int(pool[rng.integers(len(pool))]), int(rng.integers(1 << 30))))
    return out


def rect_grid_2d(nper: int = 4, p: int = 4, m: int = 64) -> Problem:
    """One member of the batched workload's family, fixed: nper x nper rectangle patches on
    [0,1]^2, all Dirichlet, degree p, m intervals per patch direction."""
    verts = _vertex_lattice(2, nper, 1.0)
    levels = int(np.log2(m)) + 1
    return _grid_problem(2, nper, p, m, levels, verts, lambda j, e: SIDE_DIRICHLET,
                         f"rect2d_K{nper*nper}_p{p}_m{m}")


CONFIGS = {
    "square2x2_p2_m8": lambda: unit_square_quadrants(8, 2, 4),
    "rect2d_K16_p4_m64": lambda: rect_grid_2d(4, 4, 64),
    "rect2d_K36_p6_m128": lambda: rect_grid_2d(6, 6, 128),
    "grid2d_K16_p4_m256": lambda: perturbed_grid_2d(4, 4, 256, 9, 2),
    "grid2d_K16_p4_m128": lambda: perturbed_grid_2d(4, 4, 128, 8, 2),
    "cube3d_K8_p3_m64": lambda: perturbed_cube_3d(2, 3, 64, 7, 3),
    "cube3d_K8_p3_m32": lambda: perturbed_cube_3d(2, 3, 32, 6, 3),
}
