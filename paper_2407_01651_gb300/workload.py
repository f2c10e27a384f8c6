"""Seeded synthetic inputs shaped like the paper's coupled problem (Section 4):
dendrite seeds and gas bubbles placed in a periodic melt.

This module holds no arithmetic of the method: it only draws positions, radii
and orientations from a counter-based generator and lists the parameter sets
of the benchmark workloads.  The library and the test oracle both take their
inputs from here and nothing else is shared between them.

Generator: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), uniform doubles from the top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

_MASK = (1 << 64) - 1

# Lattice-unit parameters of the 128^2 / 4096^2 workloads, in the paper's
# symbols.  tau0 follows from D tau0 / W0^2 = 2 (the D~ = 2 of the solutal
# case A); lambda', theta_sys and M c_inf are derived by the library from
# these (thin-interface map and the isothermal closure).
BASE_PARAMS = dict(
    rho_l=1.0, rho_g=0.1, nu=0.1, sigma=1e-3, W_phi=4.0, M_phi=0.1,
    beta_phi=0.25, beta_psi=0.25, beta_inter=0.75, W0=4.0, tau0=320.0,
    eps_s=0.05, k=0.15, D=0.1, Omega=0.55, g=1e-6, grad_eps=1e-3,
    grad_eps_at=1e-2, s_e=1.0, s_eps=1.0,
    # temperature coupling off: the isothermal closure theta = theta_sys, F = 1
    thermal=0, Le=1.0, latent=1.0, theta0=-0.55, cp=10.0,
    # velocity at an inlet side (forced convection)
    vin_x=0.0, vin_y=0.0,
)
# Thermosolutal variant (Section 4 of the paper: Le = 50, c_p^s / c_p = 1,
# initial temperature -Omega); c_p is the lattice heat capacity.
THERMAL_PARAMS = dict(thermal=1, Le=50.0, latent=1.0, theta0=-0.55, cp=10.0)
SEED_RADIUS = 6.0


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


@dataclass
class Layout:
    """Seeds (x, y, theta) and bubbles (x, y, R) of one periodic domain."""
    nx: int
    ny: int
    seeds: list = field(default_factory=list)
    bubbles: list = field(default_factory=list)
    R_s: float = SEED_RADIUS
    params: dict = field(default_factory=lambda: dict(BASE_PARAMS))


def _min_image_dist(ax, ay, bx, by, nx, ny) -> float:
    dx = (ax - bx) % nx
    dy = (ay - by) % ny
    dx = min(dx, nx - dx)
    dy = min(dy, ny - dy)
    return math.hypot(dx, dy)


def single_seed_bubble(nx: int = 128, ny: int = 128, rng_seed: int = 1,
                       R_b: float = 16.0, d_max: float = 40.0) -> Layout:
    """One seed (radius 6) at the centre and one bubble (radius 16) at an
    offset drawn from splitmix64: uniform angle, distance uniform in
    [R_s + R_b + 2 W, d_max]."""
    rng = SplitMix64(rng_seed)
    W = BASE_PARAMS["W_phi"]
    cx, cy = nx / 2.0, ny / 2.0
    ang = 2.0 * math.pi * rng.uniform()
    d_min = SEED_RADIUS + R_b + 2.0 * W
    dist = d_min + (d_max - d_min) * rng.uniform()
    return Layout(nx, ny, seeds=[(cx, cy, 0.0)],
                  bubbles=[(cx + dist * math.cos(ang), cy + dist * math.sin(ang), R_b)])


def random_layout(nx: int, ny: int, n_seeds: int, n_bubbles: int, rng_seed: int,
                  R_min: float = 8.0, R_max: float = 40.0,
                  theta_max: float = math.pi / 2, max_tries: int = 100_000) -> Layout:
    """Seeds at uniform positions with uniform orientation in [0, theta_max);
    then bubbles with radius uniform in [R_min, R_max] at uniform positions,
    rejected when closer than R + R' + 2 W to another bubble or R + R_s + 2 W to
    a seed (minimum image).  Draw order: seeds (x, y, theta), then per bubble
    try (R, x, y)."""
    rng = SplitMix64(rng_seed)
    W = BASE_PARAMS["W_phi"]
    seeds = []
    for _ in range(n_seeds):
        x = nx * rng.uniform()
        y = ny * rng.uniform()
        th = theta_max * rng.uniform()
        seeds.append((x, y, th))
    bubbles = []
    tries = 0
    while len(bubbles) < n_bubbles:
        tries += 1
        if tries > max_tries:
            raise ValueError(f"could not place {n_bubbles} bubbles in {max_tries} tries")
        R = R_min + (R_max - R_min) * rng.uniform()
        x = nx * rng.uniform()
        y = ny * rng.uniform()
        ok = all(_min_image_dist(x, y, bx, by, nx, ny) >= R + bR + 2 * W
                 for bx, by, bR in bubbles)
        ok = ok and all(_min_image_dist(x, y, sx, sy, nx, ny) >= R + SEED_RADIUS + 2 * W
                        for sx, sy, _ in seeds)
        if ok:
            bubbles.append((x, y, R))
    return Layout(nx, ny, seeds=seeds, bubbles=bubbles)


def seed_bubble_128() -> Layout:
    """128 x 128, one centred seed, one R=16 bubble at a seed-drawn offset."""
    return single_seed_bubble(128, 128, rng_seed=1)


def growth_lattice(nx: int = 4096, ny: int = 4096) -> Layout:
    """4096 x 4096, 64 seeds, 128 non-overlapping bubbles, R in [8, 40]."""
    return random_layout(nx, ny, 64, 128, rng_seed=2)


def growth_512(n: int = 512, rng_seed: int = 4) -> Layout:
    """512 x 512 (or n x n), 4 seeds and 8 bubbles."""
    return random_layout(n, n, 4, 8, rng_seed=rng_seed, R_max=min(40.0, n / 8))


def ensemble_96(rng_seed: int = 5) -> list[Layout]:
    """96 uneven domains: 32 each of 256x256, 512x384, 1024x512; per-domain
    seeds, 1..6 bubbles and eps_s uniform in [0.02, 0.07]."""
    rng = SplitMix64(rng_seed)
    out = []
    for (nx, ny) in ((256, 256), (512, 384), (1024, 512)):
        for _ in range(32):
            dom_seed = rng.next_u64()
            n_b = 1 + int(6 * rng.uniform()) % 6
            n_s = 1 + int(4 * rng.uniform()) % 4
            eps = 0.02 + 0.05 * rng.uniform()
            lay = random_layout(nx, ny, n_s, n_b, rng_seed=dom_seed, R_max=32.0)
            lay.params = dict(BASE_PARAMS, eps_s=eps)
            out.append(lay)
    return out


def growth_3d(n: int = 256, n_seeds: int = 64, rng_seed: int = 4, R_s: float = 8.0):
    """A periodic n^3 melt with n_seeds spherical seeds (radius R_s) at
    uniform positions, for the 3-D dendrite step; returns (seeds, R_s)."""
    rng = SplitMix64(rng_seed)
    seeds = [(n * rng.uniform(), n * rng.uniform(), n * rng.uniform()) for _ in range(n_seeds)]
    return seeds, R_s


def flow_3d(n: int = 256, n_seeds: int = 32, n_bub: int = 64, rng_seed: int = 5,
            R_s: float = 8.0, R_b=(6.0, 14.0)):
    """A periodic n^3 melt with n_seeds spherical seeds (radius R_s) and n_bub
    spherical bubbles (radius uniform in R_b) at uniform positions, for the 3-D
    two-phase step; returns (seeds, R_s, bubbles)."""
    rng = SplitMix64(rng_seed)
    seeds = [(n * rng.uniform(), n * rng.uniform(), n * rng.uniform()) for _ in range(n_seeds)]
    bubbles = [(n * rng.uniform(), n * rng.uniform(), n * rng.uniform(),
                R_b[0] + (R_b[1] - R_b[0]) * rng.uniform()) for _ in range(n_bub)]
    return seeds, R_s, bubbles
