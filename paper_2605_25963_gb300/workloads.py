"""Synthetic workloads: detector parameter sets, sources, energies, history counts.

Pure data -- no transport, geometry or cross-section arithmetic lives here, so
the same definitions can feed the CUDA path and the CPU oracle.

Units: mm, keV, g/cm^3.  Geometry parameters follow Table 2 of the paper
(external group d1..d10, internal group D1..D7); the coaxial layout is the
one documented with ``detmesh_params`` in ``include/gadep.h``.

Workloads (shapes of the paper's Sec. 3.2 / Table 4 experiments, with
closed-form synthetic cross sections instead of evaluated data):
  bare_cylinder     Ge cylinder R 30, L 60, 48 segments, point source 100 mm
                    above the top face, 662 keV, photoabsorption + Compton.
  coax_p            p-type coaxial HPGe in an Al endcap with Cu holder,
                    128 segments, point source 25 mm above the endcap,
                    59.5 / 122 / 662 / 1332 keV, pair production on.
  batched           bare-cylinder detector, 40 log-spaced energies 40-2000 keV
                    x 3 sources (point 25 mm, disk 60 mm dia at 10 mm, water
                    prism 70 dia x 40 on the top face) with log-uniform
                    history counts 1e6-5e7.
  gradient          coax_p + water prism 70 dia x 40 on the endcap; four density
                    groups (dead layer, endcap, active Ge, source matrix).
  stress            gradient geometry at 1024 segments (~1e6 triangles) with a
                    back-face contact groove and a bolted Cu flange; 8 energies
                    59.5-1836 keV, 1.25e8 histories each.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

DET_BARE_CYLINDER = 0
DET_COAX = 1
SRC_POINT, SRC_DISK, SRC_PRISM, SRC_PENCIL = 0, 1, 2, 3
MAT_VACUUM, MAT_GE, MAT_AL, MAT_CU, MAT_WATER = 0, 1, 2, 3, 4
MATERIAL_CODES = (MAT_VACUUM, MAT_GE, MAT_AL, MAT_CU, MAT_WATER)

# density groups of the detector builders
GROUP_DEAD_LAYER, GROUP_ENDCAP, GROUP_ACTIVE, GROUP_SOURCE = 0, 1, 2, 3


@dataclass
class Detector:
    kind: int = DET_BARE_CYLINDER
    d: tuple = (0.0,) * 10
    D: tuple = (0.0,) * 7
    n_theta: int = 48
    n_phi: int = 10
    z_slices: int = 1
    cup_rim_drop: float = 10.0
    sep_delta: float = 1e-4
    has_source_solid: int = 0
    src_r: float = 0.0
    src_h: float = 0.0
    src_z0: float = 0.0
    src_n_sides: int = 48
    # stress features of the coax (0 = absent)
    groove_r: float = 0.0
    groove_w: float = 0.0
    groove_d: float = 0.0
    flange_r_in: float = 0.0
    flange_r_out: float = 0.0
    flange_h: float = 0.0
    flange_z_top: float = 0.0
    n_bolt_holes: int = 0
    bolt_n_sides: int = 0
    bolt_r: float = 0.0
    bolt_rc: float = 0.0

    def as_dict(self):
        return dict(self.__dict__)


@dataclass
class Source:
    kind: int = SRC_POINT
    pos: tuple = (0.0, 0.0, 0.0)
    dir: tuple = (0.0, 0.0, -1.0)
    radius: float = 0.0
    height: float = 0.0
    n_sides: int = 48
    solid: int = -1            # source solid index for SRC_PRISM


# ---------------- bare Ge cylinder ----------------
BARE_CYLINDER = Detector(kind=DET_BARE_CYLINDER, D=(60.0, 30.0, 0.0, 0.0, 0.0, 0.0, 0.0),
                         n_theta=48, n_phi=10)
BARE_POINT_100 = Source(kind=SRC_POINT, pos=(0.0, 0.0, 100.0))

# ---------------- p-type coaxial HPGe ----------------
COAX_D_EXT = (38.0, 1.0, 1.0, 0.8, 5.0, 0.5, 120.0, 80.0, 1.0, 0.8)
COAX_D_INT = (62.0, 30.5, 3.0, 0.7, 48.0, 5.0, 0.0003)
COAX_P = Detector(kind=DET_COAX, d=COAX_D_EXT, D=COAX_D_INT, n_theta=128, n_phi=10,
                  cup_rim_drop=10.0, sep_delta=1e-4)
COAX_POINT_25 = Source(kind=SRC_POINT, pos=(0.0, 0.0, 25.0))
COAX_ENERGIES = (59.5, 122.0, 662.0, 1332.0)
COAX_HISTORIES = 100_000_000

# n-type variant (Table 1 #1 style dead layers: thin outer, thick inner)
COAX_N = Detector(kind=DET_COAX, d=COAX_D_EXT, D=(62.0, 30.5, 3.0, 0.0003, 48.0, 5.0, 0.7),
                  n_theta=128, n_phi=10, cup_rim_drop=10.0, sep_delta=1e-4)

# ---------------- batched ----------------
BATCH_DET = Detector(kind=DET_BARE_CYLINDER, D=(60.0, 30.0, 0.0, 0.0, 0.0, 0.0, 0.0),
                     n_theta=48, n_phi=10, has_source_solid=1, src_r=35.0, src_h=40.0,
                     src_z0=1.0, src_n_sides=48)
BATCH_SOURCES = (
    Source(kind=SRC_POINT, pos=(0.0, 0.0, 25.0)),
    Source(kind=SRC_DISK, pos=(0.0, 0.0, 10.0), radius=30.0),
    Source(kind=SRC_PRISM, pos=(0.0, 0.0, 1.0), radius=35.0, height=40.0, n_sides=48, solid=1),
)
BATCH_ENERGIES = tuple(40.0 * 50.0 ** (j / 39.0) for j in range(40))


def batch_instances(seed: int = 1, lo: float = 1e6, hi: float = 5e7):
    """(energy, source index, n_hist, source-matrix density scale) per instance.

    Instance id = 3 * energy index + source index.  History counts are drawn
    log-uniform in [lo, hi] from numpy's seeded generator.  The water prism is
    part of the mesh; instances with the point and disk sources give its
    density group scale 0 (no matrix present), the volume source scale 1.
    """
    rng = np.random.default_rng(seed)
    u = rng.random(len(BATCH_ENERGIES) * len(BATCH_SOURCES))
    out = []
    for j, E in enumerate(BATCH_ENERGIES):
        for s in range(len(BATCH_SOURCES)):
            i = 3 * j + s
            n = int(round(math.exp(math.log(lo) + u[i] * math.log(hi / lo))))
            out.append((E, s, n, 1.0 if s == 2 else 0.0))
    return out


# ---------------- gradient ----------------
GRAD_DET = Detector(kind=DET_COAX, d=COAX_D_EXT, D=COAX_D_INT, n_theta=128, n_phi=10,
                    cup_rim_drop=10.0, sep_delta=1e-4, has_source_solid=1, src_r=35.0,
                    src_h=40.0, src_z0=0.01, src_n_sides=128)
GRAD_SOURCE = Source(kind=SRC_PRISM, pos=(0.0, 0.0, 0.01), radius=35.0, height=40.0,
                     n_sides=128, solid=7)
GRAD_ENERGIES = (59.5, 122.0, 662.0, 1332.0)
GRAD_HISTORIES = 50_000_000
GRAD_N_GROUP = 4

# ---------------- Table 4 shape ----------------
# Detector #2 of Table 1 (p-type, crystal 68.1 dia x 63.3, hole 10.1 dia x 50.2,
# dead layers 0.7 mm / 0.3 um) in the coax_p housing, N_theta 32 and N_phi 10 (the
# paper's defaults); front-edge rounding 3 mm (Table 1 gives none).  Point source
# on the axis 250 mm above the endcap window; the 13 energies of Table 3.
DET2 = Detector(kind=DET_COAX, d=COAX_D_EXT, D=(63.3, 34.05, 3.0, 0.7, 50.2, 5.05, 0.0003), n_theta=32, n_phi=10,
                cup_rim_drop=10.0, sep_delta=1e-4)
TABLE4_SOURCE = Source(kind=SRC_POINT, pos=(0.0, 0.0, 250.0))
TABLE4_ENERGIES = (59.54, 81.00, 121.78, 244.70, 344.28, 356.02, 411.13, 443.97, 778.90, 964.06, 1112.09,
                   1332.49, 1408.02)

# ---------------- stress ----------------
# The gradient workload's detector and volume source at 1024 segments per circle,
# with a 2 x 1 mm contact groove on the crystal back face (centred at r = 8 mm)
# and a 3 mm Cu flange ring around the holder carrying 16 bolt holes (r 1.5 mm,
# 64-gon walls); z_slices brings the mesh to about 1e6 triangles.  The flange is
# solid 8 (after the source, solid 7).
STRESS_FEATURES = dict(groove_r=8.0, groove_w=2.0, groove_d=1.0, flange_r_in=32.0, flange_r_out=36.5,
                       flange_h=3.0, flange_z_top=-21.0, n_bolt_holes=16, bolt_n_sides=64, bolt_r=1.5,
                       bolt_rc=34.25)
STRESS_DET = Detector(kind=DET_COAX, d=COAX_D_EXT, D=COAX_D_INT, n_theta=1024, n_phi=10, z_slices=214,
                      cup_rim_drop=10.0, sep_delta=1e-4, has_source_solid=1, src_r=35.0, src_h=40.0,
                      src_z0=0.01, src_n_sides=128, **STRESS_FEATURES)
# the same features at 64 segments per circle (fast host checks and oracle parity)
STRESS_SMALL = Detector(kind=DET_COAX, d=COAX_D_EXT, D=COAX_D_INT, n_theta=64, n_phi=10, z_slices=4,
                        cup_rim_drop=10.0, sep_delta=1e-4, has_source_solid=1, src_r=35.0, src_h=40.0,
                        src_z0=0.01, src_n_sides=128, **dict(STRESS_FEATURES, bolt_n_sides=16))
STRESS_SOURCE = GRAD_SOURCE
STRESS_ENERGIES = tuple(59.5 * (1836.0 / 59.5) ** (j / 7.0) for j in range(8))
STRESS_HISTORIES = 125_000_000
STRESS_FLANGE_SOLID = 8

# ---------------- slabs (analytic checks) ----------------


def box_mesh(boxes):
    """Closed box solids: boxes = [(xmin, ymin, zmin, xmax, ymax, zmax), ...].

    Returns (xyz, tri, tri_solid) with counter-clockwise faces seen from outside.
    """
    xyz, tri, ts = [], [], []
    quads = ((0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5))
    for s, (x0, y0, z0, x1, y1, z1) in enumerate(boxes):
        base = len(xyz)
        for k in range(8):
            xyz.append((x1 if k & 1 else x0, y1 if k & 2 else y0, z1 if k & 4 else z0))
        for a, b, c, d in quads:
            tri.append((base + a, base + b, base + c))
            tri.append((base + a, base + c, base + d))
            ts += [s, s]
    return np.array(xyz, dtype=np.float64), np.array(tri, dtype=np.int32), np.array(ts, dtype=np.int32)


TABLE_N_GRID = 1000
TABLE_E_MIN = 10.0
TABLE_E_MAX = 3000.0
# charged-particle (e_model 1) range tables: kinetic energies from 1 keV (below it a
# particle deposits where it is) to TABLE_E_MAX
ERANGE_T_MIN = 1.0
ERANGE_N = 2048
N_BINS = 4096
E_MAX = 3000.0
E_CUT = 10.0
FEP_DELTA = 0.01
