"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws inputs: mesh sizes, per-element coefficients, the
substructure partition, the Dirichlet node mask and the body-force density.
It holds none of the method's arithmetic (no element matrices, no
assembly, no solver step), so the oracle and the CUDA path can both consume
its output without sharing any computation.

Indexing conventions (used by every consumer):
  element (i, j, k)  -> e = i + nx * (j + ny * k)
  node    (i, j, k)  -> n = i + (nx + 1) * (j + (ny + 1) * k)
  dof                -> n * dofs_per_node + component
  level-1 box (a, b, c) of a tensor-product partition -> a + na * (b + nb * c)

Workload shapes follow the paper's test problems (cube benchmarks with
stiff inclusions, Sec. 8.1 and 8.2; the engineering meshes of Sec. 8.3 and
8.4 are not available, so fibre/slab/random-field coefficients stand in).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Problem:
    name: str
    nx: int
    ny: int
    nz: int
    dofs_per_node: int          # 1 = scalar Poisson, 3 = linear elasticity
    coeff: np.ndarray           # (n_el,) kappa (Poisson) or Young's modulus (elasticity)
    poisson_ratio: float
    body: np.ndarray            # (n_el, dofs_per_node) body-force density
    dirichlet_node_mask: np.ndarray  # (n_nodes,) uint8, 1 = all dofs of the node fixed to 0
    cuts: List[List[np.ndarray]]     # cuts[level-1][axis] = box boundaries in element units
    elem_to_sub: np.ndarray     # (n_el,) int32 level-1 substructure of every element
    sub_to_parent: List[np.ndarray]  # levels-2 arrays: level-i substructure -> level-(i+1) one
    levels: int
    tau: float

    @property
    def h(self) -> float:
        """Edge length of the (cubic) elements; the domain is [0, nx*h] x [0, ny*h] x [0, nz*h]."""
        return 1.0 / self.nx

    @property
    def n_el(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_dofs_full(self) -> int:
        return self.n_nodes * self.dofs_per_node

    def n_subs(self, level: int = 1) -> int:
        c = self.cuts[level - 1]
        return (len(c[0]) - 1) * (len(c[1]) - 1) * (len(c[2]) - 1)


# ---------------------------------------------------------------- partitions

def _box_index(cuts_axis: np.ndarray, n: int) -> np.ndarray:
    """Box index along one axis for each element index 0..n-1."""
    return np.searchsorted(cuts_axis, np.arange(n), side="right") - 1


def tensor_partition(nx: int, ny: int, nz: int, cuts: Sequence[np.ndarray]) -> np.ndarray:
    bx = _box_index(np.asarray(cuts[0]), nx)
    by = _box_index(np.asarray(cuts[1]), ny)
    bz = _box_index(np.asarray(cuts[2]), nz)
    na, nb = len(cuts[0]) - 1, len(cuts[1]) - 1
    ii, jj, kk = np.meshgrid(bx, by, bz, indexing="ij")
    sub = ii + na * (jj + nb * kk)
    # element order is i fastest: transpose to (k, j, i) then ravel
    return np.ascontiguousarray(sub.transpose(2, 1, 0)).ravel().astype(np.int32)


def group_parents(boxes: Sequence[int], groups: Sequence[np.ndarray]) -> np.ndarray:
    """Parent of every level-i box given group boundaries (in box units) per axis."""
    na, nb, nc = boxes
    ga = _box_index(np.asarray(groups[0]), na)
    gb = _box_index(np.asarray(groups[1]), nb)
    gc = _box_index(np.asarray(groups[2]), nc)
    nga, ngb = len(groups[0]) - 1, len(groups[1]) - 1
    a, b, c = np.meshgrid(ga, gb, gc, indexing="ij")
    par = a + nga * (b + ngb * c)
    return np.ascontiguousarray(par.transpose(2, 1, 0)).ravel().astype(np.int32)


def uniform_cuts(n: int, parts: int) -> np.ndarray:
    return np.linspace(0, n, parts + 1).round().astype(np.int64)


def _dirichlet_x0(nx: int, ny: int, nz: int) -> np.ndarray:
    i = np.arange(nx + 1)
    mask = np.zeros((nz + 1, ny + 1, nx + 1), dtype=np.uint8)
    mask[:, :, i == 0] = 1
    return mask.ravel()


def _element_centres(nx: int, ny: int, nz: int):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ((i.ravel() + 0.5) / nx, (j.ravel() + 0.5) / ny, (k.ravel() + 0.5) / nz)


def _body(n_el: int, dpn: int) -> np.ndarray:
    if dpn == 1:
        return np.ones((n_el, 1))
    b = np.zeros((n_el, 3))
    b[:, 2] = -1.0
    return b


def _make(name, n, parts, dpn, coeff, levels, tau, nu=0.3, groups=None, cuts1=None):
    nx = ny = nz = n
    if cuts1 is None:
        cuts1 = [uniform_cuts(n, parts)] * 3
    cuts = [list(cuts1)]
    elem_to_sub = tensor_partition(nx, ny, nz, cuts1)
    sub_to_parent = []
    if levels >= 3:
        boxes = [len(c) - 1 for c in cuts1]
        sub_to_parent.append(group_parents(boxes, groups))
        cuts.append([np.asarray(cuts1[a])[np.asarray(groups[a])] for a in range(3)])
    return Problem(name=name, nx=nx, ny=ny, nz=nz, dofs_per_node=dpn, coeff=coeff,
                   poisson_ratio=nu, body=_body(n ** 3, dpn),
                   dirichlet_node_mask=_dirichlet_x0(nx, ny, nz), cuts=cuts,
                   elem_to_sub=elem_to_sub, sub_to_parent=sub_to_parent,
                   levels=levels, tau=tau)


# ---------------------------------------------------------------- coefficient fields

def channels(n: int, rng: np.random.Generator, value: float, frac: float) -> np.ndarray:
    """Axis-aligned lines of elements set to `value` until `frac` of the volume."""
    c = np.ones((n, n, n))   # indexed [k, j, i]
    target = int(np.ceil(frac * n ** 3))
    while int((c != 1.0).sum()) < target:
        axis = int(rng.integers(3))
        a, b = (int(x) for x in rng.integers(n, size=2))
        if axis == 0:
            c[b, a, :] = value
        elif axis == 1:
            c[b, :, a] = value
        else:
            c[:, b, a] = value
    return c.ravel()


def slabs(n: int, rng: np.random.Generator, value: float, frac: float) -> np.ndarray:
    c = np.ones((n, n, n))
    target = frac * n ** 3
    while (c != 1.0).sum() < target:
        axis = int(rng.integers(3))
        start = int(rng.integers(n))
        thick = int(rng.integers(1, 4))
        sl = slice(start, min(n, start + thick))
        if axis == 0:
            c[:, :, sl] = value
        elif axis == 1:
            c[:, sl, :] = value
        else:
            c[sl, :, :] = value
    return c.ravel()


def gaussian_random_field(n: int, rng: np.random.Generator, corr: float, sigma: float) -> np.ndarray:
    """Separable squared-exponential field on element centres, exact sampling."""
    x = np.arange(n, dtype=float)
    d = x[:, None] - x[None, :]
    k1 = np.exp(-d ** 2 / (2.0 * corr ** 2))
    w, v = np.linalg.eigh(k1)
    root = v * np.sqrt(np.clip(w, 0.0, None))
    xi = rng.standard_normal((n, n, n))
    f = np.einsum("ia,jb,kc,cba->kji", root, root, root, xi, optimize=True)
    return (sigma * f).ravel()


def fibres(n: int, rng: np.random.Generator, value: float, frac: float,
           radius_h: float = 1.5, length_h: float = 32.0) -> np.ndarray:
    h = 1.0 / n
    cx, cy, cz = _element_centres(n, n, n)
    inside = np.zeros(n ** 3, dtype=bool)
    target = frac * n ** 3
    r, L = radius_h * h, length_h * h
    pts = np.stack([cx, cy, cz], axis=1).reshape(n, n, n, 3)
    while inside.sum() < target:
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        c0 = rng.random(3)
        a, b = c0 - 0.5 * L * d, c0 + 0.5 * L * d
        lo = np.clip(np.floor((np.minimum(a, b) - r) * n).astype(int), 0, n)
        hi = np.clip(np.ceil((np.maximum(a, b) + r) * n).astype(int) + 1, 0, n)
        if np.any(hi <= lo):
            continue
        blk = pts[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        t = np.clip(((blk - a) @ d) / L, 0.0, 1.0)
        q = a + t[..., None] * (L * d)
        hit = np.linalg.norm(blk - q, axis=-1) <= r
        kk, jj, ii = np.nonzero(hit)
        inside[(ii + lo[0]) + n * ((jj + lo[1]) + n * (kk + lo[2]))] = True
    c = np.ones(n ** 3)
    c[inside] = value
    return c


def irregular_cuts(n: int, parts: int, lo: int, hi: int, rng: np.random.Generator) -> np.ndarray:
    while True:
        seg = rng.integers(lo, hi + 1, size=parts)
        if seg.sum() == n:
            return np.concatenate([[0], np.cumsum(seg)]).astype(np.int64)


# ---------------------------------------------------------------- configurations

def config(index: int) -> Problem:
    """The five benchmark workloads (1-based index), seeded with their index."""
    rng = np.random.default_rng(np.random.PCG64(index))
    if index == 1:
        coeff = channels(16, rng, 1.0e4, 0.10)
        return _make("poisson16_2x2x2_channels", 16, 2, 1, coeff, 2, 10.0)
    if index == 2:
        coeff = np.exp(1.5 * rng.standard_normal(48 ** 3))
        return _make("elasticity48_4x4x4_lognormal", 48, 4, 3, coeff, 2, 10.0)
    if index == 3:
        cuts1 = [irregular_cuts(96, 8, 6, 14, rng) for _ in range(3)]
        coeff = slabs(96, rng, 1.0e6, 0.10)
        groups = [np.array([0, 2, 4, 6, 8])] * 3
        return _make("poisson96_512irregular_slabs", 96, 8, 1, coeff, 3, 10.0,
                     groups=groups, cuts1=cuts1)
    if index == 4:
        coeff = np.exp(gaussian_random_field(64, rng, 8.0, 2.0))
        return _make("poisson64_4x4x4_grf", 64, 4, 1, coeff, 2, 10.0)
    if index == 5:
        coeff = fibres(128, rng, 1.0e6, 0.15)
        groups = [np.array([0, 4, 8, 12, 16])] * 3
        return _make("elasticity128_16x16x16_fibres", 128, 16, 3, coeff, 3, 10.0, groups=groups)
    raise ValueError(f"no config {index}")


def toy(sub_elems: int, dpn: int, seed: int, split=(2, 1, 1), sigma: float = 1.0,
        levels: int = 2, groups: Optional[Sequence[np.ndarray]] = None,
        tau: float = 10.0) -> Problem:
    """Small box meshes split into `split` substructures of sub_elems^3 elements
    with log-normal coefficients; used for brute-force checks."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    nx, ny, nz = (sub_elems * s for s in split)
    coeff = np.exp(sigma * rng.standard_normal(nx * ny * nz))
    cuts1 = [np.arange(0, (s + 1) * sub_elems, sub_elems) for s in split]
    cuts = [cuts1]
    elem_to_sub = tensor_partition(nx, ny, nz, cuts1)
    sub_to_parent = []
    if levels >= 3:
        sub_to_parent.append(group_parents(list(split), groups))
        cuts.append([np.asarray(cuts1[a])[np.asarray(groups[a])] for a in range(3)])
    return Problem(name=f"toy{split}_{sub_elems}_{dpn}_{seed}", nx=nx, ny=ny, nz=nz,
                   dofs_per_node=dpn, coeff=coeff, poisson_ratio=0.3,
                   body=_body(nx * ny * nz, dpn), dirichlet_node_mask=_dirichlet_x0(nx, ny, nz),
                   cuts=cuts, elem_to_sub=elem_to_sub, sub_to_parent=sub_to_parent,
                   levels=levels, tau=tau)


def sub_block(prob: Problem, nb: Sequence[int]) -> Problem:
    """The corner block of nb[0] x nb[1] x nb[2] level-1 boxes of a workload
    (the block at x = 0, so it keeps the Dirichlet face): same substructure
    shapes and coefficients, two levels."""
    cuts = [np.asarray(prob.cuts[0][a])[: nb[a] + 1] for a in range(3)]
    nx, ny, nz = (int(c[-1]) for c in cuts)
    coeff = prob.coeff.reshape(prob.nz, prob.ny, prob.nx)[:nz, :ny, :nx].ravel().copy()
    body = prob.body.reshape(prob.nz, prob.ny, prob.nx, -1)[:nz, :ny, :nx].reshape(nx * ny * nz, -1).copy()
    p = Problem(name=f"{prob.name}_block{nb[0]}x{nb[1]}x{nb[2]}", nx=nx, ny=ny, nz=nz,
                dofs_per_node=prob.dofs_per_node, coeff=coeff, poisson_ratio=prob.poisson_ratio, body=body,
                dirichlet_node_mask=_dirichlet_x0(nx, ny, nz), cuts=[[c - c[0] for c in cuts]],
                elem_to_sub=tensor_partition(nx, ny, nz, cuts), sub_to_parent=[], levels=2, tau=prob.tau)
    return p


def random_vector(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(np.random.PCG64(seed)).standard_normal(n)
