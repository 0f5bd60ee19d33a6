"""Seeded synthetic inputs of the weld-like travel-time workloads.

This module builds *inputs only*: stiffness matrices, densities, region maps,
region orientations, source and receiver nodes.  It holds none of the
travel-time method's arithmetic, so both the CUDA library's tests and the CPU
oracle can take their inputs from it.  Everything is numpy; nothing here
touches a GPU.

Media follow the paper's setting (Sec. 6, a weld of anisotropic grains in an
isotropic parent steel): a square weld block of Rg x Rg piecewise-constant
regions with random grain orientations, surrounded by isotropic parent steel.
The paper's EBSD weld map and its finite-element data are not available, so
these seeded media stand in for them.

Conventions
-----------
* node (i, j) is x = i*h, y = j*h; arrays are [ny, nx] (row j, column i);
* region 0 is the parent material; regions 1..Rg*Rg are the weld grains, row
  major from the weld's lower-left corner;
* orientations are radians, CCW from +x to the material's phase-angle-zero
  axis (the axis of the stiffness entry c22);
* stiffness is the 6x6 Voigt matrix in Pa.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

GPA = 1e9


def ti_voigt(c11, c33, c13, c55):
    """6x6 Voigt matrix of a transversely isotropic solid with symmetry axis 3.

    Only the YZ-plane entries (c22 = c11, c23 = c13, c33, c44 = c55) enter the
    in-plane qP speed; c12 and c66 are filled with isotropic-plane values."""
    c66 = c55
    c12 = c11 - 2.0 * c66
    C = np.zeros((6, 6))
    C[0, 0] = C[1, 1] = c11
    C[2, 2] = c33
    C[0, 1] = C[1, 0] = c12
    C[0, 2] = C[2, 0] = C[1, 2] = C[2, 1] = c13
    C[3, 3] = C[4, 4] = c55
    C[5, 5] = c66
    return C


def cubic_voigt(c11, c12, c44):
    C = np.zeros((6, 6))
    for a in range(3):
        for b in range(3):
            C[a, b] = c11 if a == b else c12
    C[3, 3] = C[4, 4] = C[5, 5] = c44
    return C


def iso_voigt(c11, c44):
    return ti_voigt(c11, c11, c11 - 2.0 * c44, c44)


# materials of the workloads
WELD_TI = (ti_voigt(234 * GPA, 216 * GPA, 145 * GPA, 129 * GPA), 8100.0)
PARENT_ISO = (ti_voigt(273 * GPA, 273 * GPA, 109 * GPA, 82 * GPA), 7850.0)
# the paper's austenitic steel (Sec. 4.5): cubic, c11 = 203.6, c12 = 133.5, c44 = 129.8 GPa
PAPER_CUBIC = (cubic_voigt(203.6 * GPA, 133.5 * GPA, 129.8 * GPA), 7850.0)


@dataclass
class Sample:
    """One medium sample: grid, region map and region orientations."""
    nx: int
    ny: int
    h: float
    region_map: np.ndarray          # uint16 [ny, nx]
    region_theta: np.ndarray        # float64 [R]
    src: np.ndarray                 # int32 [S, 2] (i, j)
    rec: np.ndarray                 # int32 [Rr, 2] (i, j)


@dataclass
class Workload:
    name: str
    materials: List[tuple]           # [(voigt 6x6, rho)]
    region_material: np.ndarray      # uint16 [R] -> index into materials
    samples: List[Sample] = field(default_factory=list)

    @property
    def nregions(self):
        return int(self.region_material.size)

    def nodes(self):
        return sum(s.nx * s.ny * len(s.src) for s in self.samples)


def weld_side(n: int, rg: int) -> int:
    """Weld block side: rg * round_half_up(0.625 * n / rg) nodes (160 for n = 256, rg = 10)."""
    return rg * int(np.floor(0.625 * n / rg + 0.5))


def weld_region_map(n: int, rg: int) -> np.ndarray:
    """Square n x n map: a centred weld block of rg x rg equal regions (ids 1..rg^2) in parent (id 0)."""
    W = weld_side(n, rg)
    o = (n - W) // 2
    cell = W // rg
    rm = np.zeros((n, n), np.uint16)
    jj, ii = np.mgrid[0:W, 0:W]
    rm[o:o + W, o:o + W] = (1 + (jj // cell) * rg + (ii // cell)).astype(np.uint16)
    return rm


def edge_nodes(n: int, k: int, j: int) -> np.ndarray:
    """k nodes on row j at i = round_half_up((m + 1/2) n / k)."""
    i = np.floor((np.arange(k) + 0.5) * n / k + 0.5).astype(np.int32)
    i = np.minimum(i, n - 1)
    return np.stack([i, np.full(k, j, np.int32)], 1)


def random_orientations(rng, rg: int) -> np.ndarray:
    """Region orientations: parent (unused, 0) + rg^2 grains uniform in [-90, 90) degrees."""
    th = np.zeros(1 + rg * rg)
    th[1:] = np.radians(rng.uniform(-90.0, 90.0, rg * rg))
    return th


def _weld_materials(rg):
    return [WELD_TI, PARENT_ISO], np.array([1] + [0] * (rg * rg), np.uint16)


def homogeneous_ti(n=64, h=1e-3, theta_deg=30.0, src=(0, 32), nrec=32) -> Workload:
    """64 x 64 homogeneous TI, orientation 30 degrees, source (0, 32), receivers at i = n-1, j = 2k+1."""
    mats = [WELD_TI]
    rec = np.stack([np.full(nrec, n - 1, np.int32), (2 * np.arange(nrec) + 1).astype(np.int32)], 1)
    s = Sample(n, n, h, np.zeros((n, n), np.uint16), np.array([np.radians(theta_deg)]),
               np.array([src], np.int32), rec)
    return Workload("homogeneous TI 64x64, h=1mm, theta=30deg, 1 source, 32 receivers", mats,
                    np.array([0], np.uint16), [s])


def weld_single(n=256, h=0.5e-3, rg=10, seed=1, nsrc=32, nrec=32) -> Workload:
    """256 x 256 weld medium, 160 x 160 weld of 10 x 10 regions, 32 bottom sources, 32 top receivers."""
    mats, rmat = _weld_materials(rg)
    rng = np.random.default_rng(seed)
    th = random_orientations(rng, rg)
    s = Sample(n, n, h, weld_region_map(n, rg), th, edge_nodes(n, nsrc, 0), edge_nodes(n, nrec, n - 1))
    return Workload(f"weld {n}x{n}, h={h*1e3:g}mm, {rg}x{rg} regions, {nsrc} src x {nrec} rec", mats, rmat, [s])


def weld_batch(nsamples=512, nsrc=32, nrec=32, sizes=tuple(range(128, 321, 32)), h=0.5e-3, rg=10,
               seed=2) -> Workload:
    """Batched media: sample k has size drawn from `sizes` (seed) and orientations from rng(seed, k)."""
    mats, rmat = _weld_materials(rg)
    size_rng = np.random.default_rng(seed)
    ns = size_rng.choice(np.asarray(sizes), size=nsamples)
    samples = []
    for k in range(nsamples):
        n = int(ns[k])
        th = random_orientations(np.random.default_rng([seed, k]), rg)
        samples.append(Sample(n, n, h, weld_region_map(n, rg), th, edge_nodes(n, nsrc, 0),
                              edge_nodes(n, nrec, n - 1)))
    return Workload(f"weld batch {nsamples} samples x {nsrc} src, n in {min(sizes)}..{max(sizes)}", mats, rmat,
                    samples)


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s own batch when several processes each solve a batch (weak scaling)."""
    return int(seed) + 7919 * int(rank)


def weld_adjoint(nsamples=256, n=200, h=0.5e-3, rg=10, nsrc=32, nrec=32, truth_seed=3, sample_seed=30):
    """Adjoint workload: truth orientations (seed 3) and nsamples candidate orientation sets (seed 30)."""
    mats, rmat = _weld_materials(rg)
    rm = weld_region_map(n, rg)
    src, rec = edge_nodes(n, nsrc, 0), edge_nodes(n, nrec, n - 1)
    truth = Sample(n, n, h, rm, random_orientations(np.random.default_rng(truth_seed), rg), src, rec)
    rng = np.random.default_rng(sample_seed)
    samples = [Sample(n, n, h, rm, random_orientations(rng, rg), src, rec) for _ in range(nsamples)]
    return (Workload(f"adjoint weld {n}x{n}, {nsamples} samples", mats, rmat, samples),
            Workload("adjoint truth", mats, rmat, [truth]))


def observation_noise(shape, sigma=10e-9, seed=33):
    return np.random.default_rng(seed).normal(0.0, sigma, size=shape)


def weld_large(n=2048, h=0.1e-3, rg=100, seed=4, nsrc=64) -> Workload:
    """2048 x 2048 weld of 100 x 100 regions, 64 bottom sources, 4096 receivers per source:
    all 2048 top-edge nodes plus the top 1024 nodes of the left and right edges."""
    mats, rmat = _weld_materials(rg)
    th = random_orientations(np.random.default_rng(seed), rg)
    top = np.stack([np.arange(n, dtype=np.int32), np.full(n, n - 1, np.int32)], 1)
    side_j = np.arange(n - 1024, n, dtype=np.int32)
    left = np.stack([np.zeros(1024, np.int32), side_j], 1)
    right = np.stack([np.full(1024, n - 1, np.int32), side_j], 1)
    rec = np.concatenate([top, left, right], 0)
    s = Sample(n, n, h, weld_region_map(n, rg), th, edge_nodes(n, nsrc, 0), rec)
    return Workload(f"weld {n}x{n}, h=0.1mm, {rg}x{rg} regions, {nsrc} src x {len(rec)} rec", mats, rmat, [s])


def velocity_gradient(nx=201, ny=211, h=1e-3, v0=3000.0, g=21.0, rho=7850.0):
    """Isotropic medium with v = v0 + g * i m/s (one isotropic material per grid column), Sec. 5.2."""
    mats = []
    for i in range(nx):
        v = v0 + g * i
        c11 = rho * v * v
        mats.append((iso_voigt(c11, c11 / 3.0), rho))
    rm = np.tile(np.arange(nx, dtype=np.uint16), (ny, 1))
    s = Sample(nx, ny, h, rm, np.zeros(nx), np.array([[1, 30]], np.int32), np.array([[199, 180]], np.int32))
    return Workload("isotropic velocity gradient v = 3000 + 21 i m/s", mats, np.arange(nx, dtype=np.uint16),
                    [s])
