"""Shared helpers of the GPU parity tests: build the library, run the oracle on the same inputs."""
import numpy as np


def oracle_medium(oracle, wl, sample, group_model=0):
    s = wl.samples[sample]
    mats = [oracle.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    return oracle.OMedium.from_regions(s.nx, s.ny, s.h, s.region_map, s.region_theta, wl.region_material, mats,
                                       group_model)


def oracle_field(oracle, wl, sample, src_index, r0=2, group_model=0, theta=None):
    s = wl.samples[sample]
    if theta is not None:
        mats = [oracle.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
        M = oracle.OMedium.from_regions(s.nx, s.ny, s.h, s.region_map, theta, wl.region_material, mats, group_model)
    else:
        M = oracle_medium(oracle, wl, sample, group_model)
    si, sj = (int(v) for v in s.src[src_index])
    fr, t0 = oracle.init_radius(M, si, sj, r0)
    tau, rec, st = oracle.fmm(M, fr, t0)
    assert st["noncausal"] == 0
    return tau, rec, fr.reshape(s.ny, s.nx), M


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    m = b > 0
    return np.abs(a - b)[m] / b[m]


def record_mismatch(gpu_rec, ora_rec, frozen):
    g = np.asarray(gpu_rec).astype(np.int64)
    o = np.asarray(ora_rec).astype(np.int64)
    o = np.where(o < 0, 255, o)
    return int(((g != o) & (frozen == 0)).sum())
