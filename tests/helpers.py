"""Small builders shared by the tests: hand-made mechanisms for closed-form
checks and conversions from the seeded workloads.  Holds none of the method's
arithmetic."""
import numpy as np
import torch

from paper_2202_02319_b300 import synth
from oracle.mech import MechT, GridT, from_synth, grid_from_synth

R = 8.314462618


def single_species(gamma=1.4, W=R, mu=0.0, mu_exp=0.0, cp_extra=None):
    """One species with constant cp/R = gamma/(gamma-1) (W = R gives R/W = 1)."""
    a = np.zeros((1, 7))
    a[0, 0] = gamma / (gamma - 1.0)
    if cp_extra is not None:
        a[0, 1:5] = cp_extra
    m = synth.Mechanism(names=["A"], W=np.array([W]), elem=np.array([[1.0]]), nasa_low=a.copy(),
                        nasa_high=a.copy(), T_mid=np.array([1000.0]), mu_ref=np.array([mu]),
                        mu_exp=np.array([mu_exp]), D_ref=np.array([[1e-5]]),
                        A=np.zeros(0), b=np.zeros(0), Theta=np.zeros(0),
                        nu_f=np.zeros((0, 1), dtype=np.int64), nu_r=np.zeros((0, 1), dtype=np.int64),
                        reversible=np.zeros(0, dtype=np.int32))
    return m


def mech_t(m):
    return from_synth(m)


def grid_t(g):
    return grid_from_synth(g)


def tensor(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64)


def random_prim(mech, shape, seed, T_lo=300.0, T_hi=2500.0, vmax=50.0, p=101325.0, smooth=False):
    """Random primitive fields (p, T, u, v, w, Y) for tests."""
    g = np.random.default_rng(seed)
    ns = mech.n_species
    if smooth:
        nz, ny, nx = shape
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

        def f(k):
            ph = g.uniform(0, 2 * np.pi, 3)
            return (np.sin(2 * np.pi * x / nx + ph[0]) * np.cos(2 * np.pi * y / ny + ph[1])
                    + np.sin(2 * np.pi * z / nz + ph[2]))
        T = 0.5 * (T_lo + T_hi) + 0.25 * (T_hi - T_lo) * f(0) / 2
        vel = [vmax * f(i) / 2 for i in range(3)]
        Yr = np.stack([1.0 + 0.5 * f(s) / 2 for s in range(ns)])
    else:
        T = g.uniform(T_lo, T_hi, shape)
        vel = [g.uniform(-vmax, vmax, shape) for _ in range(3)]
        Yr = g.dirichlet(np.ones(ns), size=shape).transpose(3, 0, 1, 2)
    Y = Yr / Yr.sum(0)
    pr = np.full(shape, p) * (1.0 + (0.05 * g.standard_normal(shape) if not smooth else 0.0))
    return np.concatenate([pr[None], T[None], *(v[None] for v in vel), Y])
