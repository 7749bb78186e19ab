"""Named workloads: problem + architecture specifications with their seeds.

Every input of the method is synthetic by construction: the Brownian paths are
the method's own draws (Philox, keyed by the seed) and Theta_0 is a seeded
Xavier initialisation.  The shapes follow Section 4 (Black--Scholes--Barenblatt
with d = 100, r = 0.05, sigma = 0.4; HJB with d = 100, T = 1, x0 = 0) at the
sizes used for measurement.  This module holds specifications only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

from .solver import ArchSpec, ProblemSpec


def bsb_x0(D: int):
    """x0 = (1, 0.5, 1, 0.5, ...); with D = 100 the closed form gives
    u(0, x0) = 62.5 exp(0.21) ~ 77.1, the value the paper's figure marks."""
    return [1.0 if i % 2 == 0 else 0.5 for i in range(D)]


@dataclass(frozen=True)
class Workload:
    name: str
    problem: ProblemSpec
    arch: ArchSpec
    seed: int = 0
    adam_steps: int = 0
    lr: float = 1e-3

    def with_prec(self, prec: str) -> "Workload":
        return replace(self, arch=replace(self.arch, prec=prec))


WORKLOADS = {
    # 10-D BSB, N = 8 steps, M = 64 paths, FC 4 x 64 sin: the small case
    "bsb_d10_n8_m64_fc4x64_sin": Workload(
        "bsb_d10_n8_m64_fc4x64_sin",
        ProblemSpec(kind="bsb", D=10, N=8, M=64, x0=bsb_x0(10)),
        ArchSpec(kind="fc", width=64, depth=4, act="sin"), seed=0, adam_steps=200),
    # 100-D BSB, N = 64, M = 4096, ResNet 5 blocks x 256 tanh: the measured workload
    "bsb_d100_n64_m4096_resnet5x256_tanh": Workload(
        "bsb_d100_n64_m4096_resnet5x256_tanh",
        ProblemSpec(kind="bsb", D=100, N=64, M=4096, x0=bsb_x0(100)),
        ArchSpec(kind="resnet", width=256, depth=5, act="tanh"), seed=0, adam_steps=5000),
    # 100-D HJB, N = 64, M = 8192, x0 = 0, NAIS 6 blocks x 256 tanh
    "hjb_d100_n64_m8192_nais6x256_tanh": Workload(
        "hjb_d100_n64_m8192_nais6x256_tanh",
        ProblemSpec(kind="hjb", D=100, N=64, M=8192, x0=[0.0] * 100),
        ArchSpec(kind="nais", width=256, depth=6, act="tanh"), seed=0, adam_steps=5000),
    # 100-D BSB, N = 64, M = 16384, NAIS 6 blocks x 512 tanh: the wide network
    # of the multilevel study (Section 3.2); width 512 runs on the layered path
    "bsb_d100_n64_m16384_nais6x512_tanh": Workload(
        "bsb_d100_n64_m16384_nais6x512_tanh",
        ProblemSpec(kind="bsb", D=100, N=64, M=16384, x0=bsb_x0(100)),
        ArchSpec(kind="nais", width=512, depth=6, act="tanh"), seed=0, adam_steps=5000),
}

# Closed-form anchors (Section 4): BSB u(0, x0) and HJB u(0, 0) (Cole-Hopf,
# chi-square quadrature), used for the accuracy of a trained Y_0.
BSB_Y0_D100 = 62.5 * math.exp(0.21)  # ||x0||^2 = 62.5, (r + sigma^2) T = 0.21
BSB_Y0_D10 = 6.25 * math.exp(0.21)
HJB_U00_D100 = 4.590162


def bsb_y0(x0, r: float = 0.05, sigma: float = 0.4, T: float = 1.0) -> float:
    """Closed form of the BSB problem (Section 4.1) at t = 0:
    u(0, x) = exp((r + sigma^2) T) ||x||^2."""
    return math.exp((r + sigma * sigma) * T) * sum(float(v) * float(v) for v in x0)


# Multilevel schedule of the measured workload (Section 3.2): grids of 4, 8,
# 16 and 32 Euler steps for a fixed number of Adam steps each, then the
# target grid of 64 steps.
MULTILEVEL_LEVELS = (4, 8, 16, 32, 64)
MULTILEVEL_COARSE_STEPS = 100


def batched_instances(seed: int = 0, n: int = 32, budget_gb: float = 140.0):
    """Uneven independent instances (half BSB, half HJB): D from
    {10, 20, 50, 100, 200}, N from {16, 32, 64, 128}, M from {1024, 4096,
    16384}, ResNet 4 x w tanh with w from {128, 256, 512}, all seeded.  The
    largest instances' M is halved until the estimated device memory of all
    workspaces fits `budget_gb`.  Returns a list of Workloads."""
    import random
    rng = random.Random(seed)
    specs = []
    for i in range(n):
        kind = "bsb" if i % 2 == 0 else "hjb"
        D = rng.choice([10, 20, 50, 100, 200])
        N = rng.choice([16, 32, 64, 128])
        M = rng.choice([1024, 4096, 16384])
        w = rng.choice([128, 256, 512])
        specs.append([kind, D, N, M, w])

    def est_bytes(D, N, M, w, L=4):
        P = M * (N + 1)
        Dp = (D + 63) // 64 * 64
        per_point = 4 * (L + 1) * 2 * w + 2 * 2 * Dp + 4 * 4 * D + 64
        if w <= 256:  # fused kernels: g_l and per-CTA scratch
            return P * (per_point + L * 2 * w) + 152 * (2 * L + 2) * 128 * w * 2
        return P * (per_point + 6 * (L + 1) * 4 * w)  # layered: FP32 per-layer tensors

    while sum(est_bytes(D, N, M, w) for _, D, N, M, w in specs) > budget_gb * 1e9:
        big = max(range(n), key=lambda i: est_bytes(*specs[i][1:]))
        specs[big][3] //= 2
    out = []
    for i, (kind, D, N, M, w) in enumerate(specs):
        x0 = bsb_x0(D) if kind == "bsb" else [0.0] * D
        out.append(Workload(f"inst{i}_{kind}_d{D}_n{N}_m{M}_resnet4x{w}",
                            ProblemSpec(kind=kind, D=D, N=N, M=M, x0=x0),
                            ArchSpec(kind="resnet", width=w, depth=4, act="tanh", prec="bf16"), seed=seed + i))
    return out

