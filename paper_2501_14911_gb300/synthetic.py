"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module draws random numbers and fixes shapes; it holds none of the
method's arithmetic (no Toeplitz products, no FFTs, no covariances), so the
CUDA path and the CPU oracle can both be fed from it without sharing code.

The paper's operators come from PDE solves (Sec. 5, Phase 1) that are not
available here.  Synthetic blocks stand in for them with the structure the
method relies on (N_d << N_m, N_q << N_m, N_t >> 1, Sec. 4) and a causal decay
in k: F_k = N(0, 1) entries scaled by exp(-k / tau).

Generation is deterministic for a seed regardless of thread count: time block
k of a block array is drawn from child k of numpy SeedSequence(seed), so
blocks can be filled in parallel.
"""

from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np


def _threads():
    return max(1, min(16, os.cpu_count() or 1))


def _fill_normal(out2d, seeds, scale=None):
    """Fill out2d[k] (k = 0..len(seeds)-1) with N(0,1) from child seed k."""

    def work(k):
        g = np.random.Generator(np.random.PCG64(seeds[k]))
        if out2d.dtype == np.float64:
            g.standard_normal(out=out2d[k])
        else:
            out2d[k] = g.standard_normal(out2d[k].shape)
        if scale is not None:
            out2d[k] *= scale[k]

    n = len(seeds)
    if n == 1 or out2d[0].size < 1 << 16:
        for k in range(n):
            work(k)
    else:
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(work, range(n)))


def toeplitz_blocks(seed, Nt, R, Nm, tau, dtype=np.float64):
    """Blocks [N_t][R][N_m]: entries N(0,1) times exp(-k / tau) in block k."""
    out = np.empty((Nt, R, Nm), dtype=dtype)
    seeds = np.random.SeedSequence(seed).spawn(Nt)
    scale = np.exp(-np.arange(Nt, dtype=np.float64) / float(tau)).astype(dtype)
    _fill_normal(out.reshape(Nt, R * Nm), seeds, scale)
    return out


def gaussian(seed, shape, dtype=np.float64):
    """N(0,1) array of the given shape; the leading axis indexes child seeds."""
    shape = tuple(int(s) for s in shape)
    if len(shape) == 0:
        return np.random.Generator(np.random.PCG64(seed)).standard_normal()
    out = np.empty(shape, dtype=dtype)
    lead = shape[0]
    seeds = np.random.SeedSequence(seed).spawn(max(lead, 1))
    if lead:
        _fill_normal(out.reshape(lead, -1), seeds)
    return out


@dataclass(frozen=True)
class Problem:
    """One workload: sizes, prior and noise settings, and seeds.

    Node index on the gx x gy parameter grid is ix * gy + iy (N_m = gx * gy).
    """

    name: str
    index: int          # workload number; seeds are 1000 * index + offset
    gx: int
    gy: int
    Nd: int
    Nt: int
    Nq: int
    tau: float
    ell: float = 3.0     # SE length scale in cells
    sigma_p: float = 1.0 # SE standard deviation
    sigma2: float = 1e-4 # Gamma_noise = sigma2 * I
    n_vectors: int = 1   # m / d vectors (or observation vectors)
    col_block: int = 512
    notes: str = field(default="", compare=False)

    @property
    def Nm(self):
        return self.gx * self.gy

    @property
    def L(self):
        return 2 * self.Nt

    # seeds
    def seed(self, offset):
        return 1000 * self.index + offset

    def blocks_F(self, dtype=np.float64):
        return toeplitz_blocks(self.seed(1), self.Nt, self.Nd, self.Nm, self.tau, dtype)

    def blocks_Fq(self, dtype=np.float64):
        return toeplitz_blocks(self.seed(2), self.Nt, self.Nq, self.Nm, self.tau, dtype)

    def vectors_m(self, B=None, dtype=np.float64):
        B = self.n_vectors if B is None else B
        return gaussian(self.seed(3), (B, self.Nt, self.Nm), dtype)

    def vectors_d(self, B=None, dtype=np.float64):
        B = self.n_vectors if B is None else B
        return gaussian(self.seed(3) + 500, (B, self.Nt, self.Nd), dtype)

    def z_true(self, B=None):
        """N(0,1) draws that a prior square root maps to m_true."""
        B = self.n_vectors if B is None else B
        return gaussian(self.seed(4), (B, self.Nt, self.Nm))

    def noise(self, B=None):
        """N(0,1) draws; d_obs = F m_true + sqrt(sigma2) * noise."""
        B = self.n_vectors if B is None else B
        return gaussian(self.seed(5), (B, self.Nt, self.Nd))


TINY = Problem("tiny_inversion_Nm256_Nd8_Nt64", 1, 16, 16, 8, 64, 32, 16.0, n_vectors=1)
SWEEP = Problem("matvec_sweep_Nm65536_Nd128_Nt256", 2, 256, 256, 128, 256, 32, 64.0, n_vectors=16)
MIXED = Problem("mixed_precision_Nm16384_Nd600_Nt420", 3, 128, 128, 600, 420, 32, 105.0, n_vectors=1)
BATCHED = Problem("batched_online_Nm4096_Nd100_Nt200", 4, 64, 64, 100, 200, 32, 50.0, n_vectors=64)
DIFF = Problem("diff_qoi_Nm8192_Nd64_Nt256_Nq32", 5, 64, 128, 64, 256, 32, 64.0, n_vectors=1)

# The mixed-precision workload truncated to its first 42 time steps (K 25,200^2, which the
# oracle can still factor densely): the same workload number and decay, so its blocks are the
# first 42 blocks of MIXED; 16 observation vectors.
MIXED_NT42 = Problem("mixed_precision_Nm16384_Nd600_Nt42", 3, 128, 128, 600, 42, 32, 105.0, n_vectors=16)

WORKLOADS = {p.name: p for p in (TINY, SWEEP, MIXED, BATCHED, DIFF)}


def small(name, gx, gy, Nd, Nt, Nq=4, tau=None, index=90, **kw):
    """A reduced problem with the same recipe (for fast parity tests)."""
    return Problem(name, index, gx, gy, Nd, Nt, Nq, float(tau if tau else max(Nt / 4.0, 1.0)), **kw)
