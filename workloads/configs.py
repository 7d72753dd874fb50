"""The seeded workloads the solver is measured and checked on.

Each entry mirrors one of the paper-shaped problems: 2-D/3-D SIPG Poisson with a
coefficient jump across a ball of radius 0.3 centred in the unit square/cube (the paper's
Poisson benchmark, Sec. 5.1, uses a jump of 1000 across a spherical interface).
"""
from __future__ import annotations

import dataclasses

from .sipg import make_problem


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    d: int
    p: int
    n: tuple
    nlevels: int
    length: tuple | None = None
    nu_kind: str = "jump"
    nu_inside: float = 1000.0
    nrhs: int = 1
    precision: str = "fp64"     # fp64 | mixed | mixed_bf16
    description: str = ""

    @property
    def np_(self):
        from math import comb
        return comb(self.p + self.d, self.d)

    @property
    def ndof(self):
        c = 1
        for v in self.n:
            c *= v
        return c * self.np_

    def make(self, seed: int = 0):
        return make_problem(self.d, self.p, self.n, self.nlevels, length=self.length,
                            nu_kind=self.nu_kind, nu_inside=self.nu_inside, seed=seed,
                            nrhs=self.nrhs)


WORKLOADS = {w.name: w for w in [
    Workload("sipg2d_p1_16x16", 2, 1, (16, 16), 3,
             description="2-D SIPG p=1, 16x16 cells (768 DOFs), nu 1000 inside r=0.3, 3 levels"),
    Workload("sipg3d_p2_64cube", 3, 2, (64, 64, 64), 5,
             description="3-D SIPG p=2, 64^3 cells (2,621,440 DOFs), nu 1:1000, 5 levels, FP64"),
    Workload("sipg3d_p3_48cube_zstretch", 3, 3, (48, 48, 48), 5, length=(1.0, 1.0, 10.0),
             nu_inside=1.0e4, precision="mixed",
             description="3-D SIPG p=3, 48^3 cells stretched 1:10 in z (2,211,840 DOFs), "
                         "nu 1:1e4, FP32 inner / FP64 refinement"),
    Workload("sipg3d_p2_64cube_rhs32", 3, 2, (64, 64, 64), 5, nrhs=32, precision="mixed",
             description="3-D SIPG p=2, 64^3 cells, 32 right-hand sides in one solve"),
    Workload("sipg3d_p2_32cube_rhs32", 3, 2, (32, 32, 32), 4, nrhs=32, precision="mixed_bf16",
             description="3-D SIPG p=2, 32^3 cells (327,680 DOFs), nu 1:1000, 32 right-hand "
                         "sides in one solve (the 32-column batch at a size whose slowest "
                         "column converges within a minute)"),
    Workload("sipg3d_p2_48cube_rhs32", 3, 2, (48, 48, 48), 4, nrhs=32, precision="mixed_bf16",
             description="3-D SIPG p=2, 48^3 cells, 32 right-hand sides (profiling case of the "
                         "batched kernels: vectors larger than L2, a few GB on the device)"),
    Workload("sipg3d_p2_32cube_lognormal", 3, 2, (32, 32, 32), 4, nu_kind="lognormal",
             description="3-D SIPG p=2, 32^3 cells (327,680 DOFs), log nu ~ N(0,1) + ln 1000 "
                         "inside the ball; adjoint gradient workload"),
    # small cases for parity tests: several tiles and ragged tails
    Workload("sipg3d_p2_8cube", 3, 2, (8, 8, 8), 3, description="3-D p=2, 8^3, 3 levels"),
    Workload("sipg3d_p1_8x4x4", 3, 1, (8, 4, 4), 3, description="3-D p=1, 8x4x4, 3 levels"),
    Workload("sipg3d_p3_8cube_zstretch", 3, 3, (8, 8, 8), 3, length=(1.0, 1.0, 10.0),
             nu_inside=1.0e4, description="3-D p=3, 8^3 stretched 1:10 in z, nu 1:1e4"),
    Workload("sipg2d_p2_32x16", 2, 2, (32, 16), 4, description="2-D p=2, 32x16, 4 levels"),
]}


def workload(name: str) -> Workload:
    return WORKLOADS[name]
