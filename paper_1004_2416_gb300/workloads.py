"""Seeded synthetic workloads shaped like the paper's shear-flow set-ups.

This module only prepares inputs: lattice sizes, capsule placements and the
moduli and wall speeds that realise a given reduced shear rate.  It holds no
step of the method itself.  Parameter mapping (Sec. III, Eqs. Re and
shearrate; Sec. II.A): the shear rate between walls at distance H = nz moving
with +-u_wall is gdot = 2 u_wall / H, the dynamic viscosity at rest density 1 is
eta = (tau - 1/2)/3, and the reduced shear rate ("capillary number")
G = gdot eta r / k_s, so k_s = gdot eta r / G.

Workloads (lattice units, tau = 1, gdot = 1e-3 everywhere):
  config1  32^3, FP64, one capsule r = 4 (320 faces), G = 0.0125, 3-point delta,
           1000 steps
  config2  128^3, FP32, one capsule r = 16 (5120 faces), G in {0.003, 0.0125,
           0.05}, 4-point (and 2-point) delta, 20000 steps
  config3  64 independent runs, cubic side in {24, 32, 48, 64}, r = side/8,
           320 faces if r <= 4 else 1280, G log-uniform in [0.003, 0.1],
           3-point delta, 5000 steps
  config4  256 x 128 x 128, 200 capsules r = 6 (1280 faces) placed by random
           sequential addition, G = 0.02, 3-point delta, FP16 storage,
           10000 steps
  config5  64^3, FP32, one capsule r = 8 (1280 faces), G = 0.0125, 3-point
           delta, 2000 steps, checkpoints every 100 steps
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GDOT = 1e-3
TAU = 1.0


def eta(tau: float = TAU) -> float:
    return (tau - 0.5) / 3.0


def k_s_for(G: float, r: float, gdot: float = GDOT, tau: float = TAU) -> float:
    return gdot * eta(tau) * r / G


def u_wall_for(nz: int, gdot: float = GDOT) -> float:
    return gdot * nz / 2.0


@dataclasses.dataclass
class Capsule:
    center: tuple
    radius: float
    subdivisions: int
    k_s: float
    C: float = 1.0


@dataclasses.dataclass
class Case:
    name: str
    shape: tuple  # (nx, ny, nz)
    tau: float
    delta: int
    precision: str
    u_wall: float
    capsules: list
    steps: int

    @property
    def ncell(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz

    @property
    def n_nodes(self) -> int:
        return sum(10 * 4 ** c.subdivisions + 2 for c in self.capsules)


def single_capsule(name, n, r, m, G, delta, precision, steps, shape=None):
    shape = shape or (n, n, n)
    nx, ny, nz = shape
    c = Capsule(((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2), r, m, k_s_for(G, r))
    return Case(name, shape, TAU, delta, precision, u_wall_for(nz), [c], steps)


def config1() -> Case:
    return single_capsule("config1-32^3-fp64-r4-320f-phi3", 32, 4.0, 2, 0.0125, 3, "fp64", 1000)


def config2(G: float = 0.0125, delta: int = 4, precision: str = "fp32") -> Case:
    return single_capsule(f"config2-128^3-{precision}-r16-5120f-phi{delta}-G{G}", 128, 16.0, 4, G,
                          delta, precision, 20000)


def config5() -> Case:
    return single_capsule("config5-64^3-fp32-r8-1280f-phi3", 64, 8.0, 3, 0.0125, 3, "fp32", 2000)


def convergence_case(H: int, delta: int, precision: str = "fp32", Re: float = 0.02, G: float = 0.01) -> Case:
    """The coupled-convergence series of Sec. IV.C (Tab. convergence): a cubic
    box of side H with H/r = 10, N_f = 1280, 5120, 20480 faces for H = 35, 70,
    140 (mean edge / dx = 0.53), Re = gdot r^2 / nu = 0.02, G = 0.01, tau = 1,
    run to kappa t = gdot t / G = 120."""
    m = {35: 3, 70: 4, 140: 5}[H]
    r = H / 10.0
    gdot = Re * eta() / (r * r)
    steps = int(round(120.0 * G / gdot))
    c = Capsule(((H - 1) / 2, (H - 1) / 2, (H - 1) / 2), r, m, k_s_for(G, r, gdot))
    return Case(f"convergence-H{H}-{precision}-{20 * 4 ** m}f-phi{delta}", (H, H, H), TAU, delta, precision,
                u_wall_for(H, gdot), [c], steps)


def config3_specs(seed: int = 3, n_runs: int = 64):
    """Independent runs: (side, radius, subdivisions, G) per run."""
    rng = np.random.default_rng(seed)
    sides = rng.choice([24, 32, 48, 64], size=n_runs)
    Gs = np.exp(rng.uniform(math.log(0.003), math.log(0.1), size=n_runs))
    out = []
    for side, G in zip(sides.tolist(), Gs.tolist()):
        r = side / 8.0
        out.append((int(side), r, 2 if r <= 4 else 3, float(G)))
    return out


def config3_cases(seed: int = 3, n_runs: int = 64, precision: str = "fp32"):
    return [single_capsule(f"config3-run{k}-{side}^3", side, r, m, G, 3, precision, 5000)
            for k, (side, r, m, G) in enumerate(config3_specs(seed, n_runs))]


def rsa_centres(shape, n: int, r: float, seed: int, z_margin: float, gap: float = 2.0,
                max_tries: int = 200000):
    """Random sequential addition of n spheres of radius r: centres uniform in x
    and y (periodic, minimum-image distance >= 2 r + gap) and in
    z in [z_margin, nz - 1 - z_margin]."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    box = np.array([nx, ny], float)
    cs = []
    tries = 0
    while len(cs) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random sequential addition did not converge")
        c = np.array([rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(z_margin, nz - 1 - z_margin)])
        ok = True
        for d in cs:
            dxy = c[:2] - d[:2]
            dxy -= box * np.round(dxy / box)
            if dxy @ dxy + (c[2] - d[2]) ** 2 < (2 * r + gap) ** 2:
                ok = False
                break
        if ok:
            cs.append(c)
    return [tuple(map(float, c)) for c in cs]


def config4(precision: str = "fp16", n_caps: int = 200, seed: int = 4) -> Case:
    shape = (256, 128, 128)
    r, G = 6.0, 0.02
    centres = rsa_centres(shape, n_caps, r, seed, z_margin=r + 4.0)
    caps = [Capsule(c, r, 3, k_s_for(G, r)) for c in centres]
    return Case(f"config4-256x128x128-{precision}-200caps-r6-1280f-phi3", shape, TAU, 3, precision,
                u_wall_for(shape[2]), caps, 10000)


def jitter(n_nodes: int, amp: float, seed: int) -> np.ndarray:
    """Seeded node displacements [n, 3], uniform in [-amp, amp]."""
    return np.random.default_rng(seed).uniform(-amp, amp, size=(n_nodes, 3))


def population_noise(shape, amp: float, seed: int) -> np.ndarray:
    """Seeded perturbation [19, nz, ny, nx], uniform in [-amp, amp]."""
    nx, ny, nz = shape
    return np.random.default_rng(seed).uniform(-amp, amp, size=(19, nz, ny, nx))
