"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this module.  It loads ``oracle/liboracle.so`` (built from
the C sources beside it by :func:`build`) and never touches the product
library or the GPU.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SOURCES = ["orc_rng.c", "orc_xs.c", "orc_mesh.c", "orc_transport.c"]

MAT_VACUUM, MAT_GE, MAT_AL, MAT_CU, MAT_WATER = 0, 1, 2, 3, 4
DET_BARE_CYLINDER, DET_COAX = 0, 1
SRC_POINT, SRC_DISK, SRC_PRISM, SRC_PENCIL = 0, 1, 2, 3
MEC2 = 510.99895


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C99, -O2, no fast-math)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    if not force and os.path.exists(LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(HERE, "oracle.h")])
        if os.path.getmtime(LIB_PATH) >= newest:
            return LIB_PATH
    tmp = LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-D_POSIX_C_SOURCE=200809L",
           "-o", tmp] + srcs + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class DetParams(C.Structure):
    _fields_ = [("kind", C.c_int), ("d", C.c_double * 10), ("D", C.c_double * 7),
                ("n_theta", C.c_int), ("n_phi", C.c_int), ("z_slices", C.c_int),
                ("cup_rim_drop", C.c_double), ("sep_delta", C.c_double),
                ("has_source_solid", C.c_int), ("src_r", C.c_double), ("src_h", C.c_double),
                ("src_z0", C.c_double), ("src_n_sides", C.c_int),
                ("groove_r", C.c_double), ("groove_w", C.c_double), ("groove_d", C.c_double),
                ("flange_r_in", C.c_double), ("flange_r_out", C.c_double), ("flange_h", C.c_double),
                ("flange_z_top", C.c_double), ("n_bolt_holes", C.c_int), ("bolt_n_sides", C.c_int),
                ("bolt_r", C.c_double), ("bolt_rc", C.c_double)]


class MeshC(C.Structure):
    _fields_ = [("n_vert", C.c_int), ("n_tri", C.c_int), ("n_solid", C.c_int),
                ("xyz", C.POINTER(C.c_double)), ("tri", C.POINTER(C.c_int)),
                ("tri_solid", C.POINTER(C.c_int)), ("solid_material", C.POINTER(C.c_int)),
                ("solid_active", C.POINTER(C.c_int)), ("solid_group", C.POINTER(C.c_int)),
                ("solid_parent", C.POINTER(C.c_int))]


class TablesC(C.Structure):
    _fields_ = [("n_mat", C.c_int), ("n_grid", C.c_int), ("lnE_min", C.c_double),
                ("lnE_max", C.c_double), ("mu", C.POINTER(C.c_float)), ("e_n", C.c_int),
                ("lnT_min", C.c_double), ("lnT_max", C.c_double), ("e_range", C.POINTER(C.c_double))]


class SourceC(C.Structure):
    _fields_ = [("kind", C.c_int), ("pos", C.c_double * 3), ("dir", C.c_double * 3),
                ("radius", C.c_double), ("height", C.c_double), ("n_sides", C.c_int)]


class OptsC(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("history_offset", C.c_uint64), ("instance", C.c_uint32),
                ("energy_keV", C.c_double), ("e_cut_keV", C.c_double),
                ("fep_delta_keV", C.c_double), ("e_max_keV", C.c_double), ("n_bins", C.c_int),
                ("step_cap", C.c_int), ("n_group", C.c_int), ("group_scale", C.c_double * 8),
                ("e_model", C.c_int)]


class TallyC(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "n_hist", "n_fep", "n_zero", "n_over", "n_err", "n_parity_mismatch", "n_dup_hits",
        "n_segments", "n_interactions", "n_crossings", "n_flights", "n_first_pe",
        "n_first_compton", "n_first_pair", "n_first_none")] + [
        (n, C.c_double) for n in ("sum_dep_active", "sum_dep_all", "sum_esc",
                                  "max_rel_energy_err")] + [
        ("fep_score", C.c_double * 8), ("fep_score_sq", C.c_double * 8)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                        C.POINTER(C.c_uint32)]
        L.orc_u01.restype = C.c_double
        L.orc_u01.argtypes = [C.c_uint32]
        L.orc_stream_words.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_int,
                                       C.POINTER(C.c_uint32)]
        for f in ("orc_sigma_kn",):
            getattr(L, f).restype = C.c_double
            getattr(L, f).argtypes = [C.c_double]
        L.orc_dsigma_kn_dcos.restype = C.c_double
        L.orc_dsigma_kn_dcos.argtypes = [C.c_double, C.c_double]
        L.orc_sigma_pe.restype = C.c_double
        L.orc_sigma_pe.argtypes = [C.c_int, C.c_double]
        L.orc_sigma_pair.restype = C.c_double
        L.orc_sigma_pair.argtypes = [C.c_int, C.c_double]
        L.orc_mu.argtypes = [C.c_int, C.c_double, C.POINTER(C.c_double)]
        L.orc_tables_build.restype = C.POINTER(TablesC)
        L.orc_tables_build.argtypes = [C.POINTER(C.c_int), C.c_int, C.c_int, C.c_double, C.c_double]
        L.orc_tables_from_array.restype = C.POINTER(TablesC)
        L.orc_tables_from_array.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double,
                                            C.POINTER(C.c_float)]
        L.orc_tables_free.argtypes = [C.POINTER(TablesC)]
        L.orc_tables_eval.argtypes = [C.POINTER(TablesC), C.c_int, C.c_double,
                                      C.POINTER(C.c_double)]
        L.orc_e_stopping.argtypes = [C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_e_range.restype = C.c_double
        L.orc_e_range.argtypes = [C.POINTER(TablesC), C.c_int, C.c_double]
        L.orc_e_energy_after.restype = C.c_double
        L.orc_e_energy_after.argtypes = [C.POINTER(TablesC), C.c_int, C.c_double, C.c_double]
        L.orc_e_track.argtypes = [C.POINTER(MeshC), C.POINTER(TablesC), C.POINTER(OptsC), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.c_double, C.c_double, C.c_int, C.POINTER(C.c_double)]
        L.orc_mesh_build.argtypes = [C.POINTER(DetParams), C.POINTER(C.POINTER(MeshC))]
        L.orc_mesh_from_arrays.restype = C.POINTER(MeshC)
        L.orc_mesh_from_arrays.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int,
                                           C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int,
                                           C.POINTER(C.c_int), C.POINTER(C.c_int),
                                           C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_mesh_free.argtypes = [C.POINTER(MeshC)]
        for f in ("orc_mesh_volume", "orc_mesh_area"):
            getattr(L, f).restype = C.c_double
            getattr(L, f).argtypes = [C.POINTER(MeshC), C.c_int]
        for f in ("orc_mesh_euler", "orc_mesh_open_edges"):
            getattr(L, f).argtypes = [C.POINTER(MeshC), C.c_int]
        L.orc_locate.argtypes = [C.POINTER(MeshC), C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_nearest_hit.argtypes = [C.POINTER(MeshC), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
        L.orc_sample_birth.argtypes = [C.POINTER(SourceC), C.c_uint64, C.c_uint64, C.c_uint32,
                                       C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_kahn_samples.argtypes = [C.c_double, C.c_uint64, C.c_int, C.POINTER(C.c_double)]
        L.orc_transport.argtypes = [C.POINTER(MeshC), C.POINTER(TablesC), C.POINTER(SourceC),
                                    C.POINTER(OptsC), C.c_uint64, C.c_int, C.POINTER(TallyC),
                                    C.POINTER(C.c_uint32), C.POINTER(C.c_double)]
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


# ---------------- RNG ----------------

def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def stream_words(seed, hid, inst, n):
    out = np.zeros(n, dtype=np.uint32)
    lib().orc_stream_words(seed, hid, inst, n, _ptr(out, C.c_uint32))
    return out


def u01(x):
    return lib().orc_u01(int(x))


# ---------------- cross sections ----------------

def sigma_kn(k):
    return lib().orc_sigma_kn(k)


def dsigma_kn_dcos(k, c):
    return lib().orc_dsigma_kn_dcos(k, c)


def sigma_pe(Z, E):
    return lib().orc_sigma_pe(Z, E)


def sigma_pair(Z, E):
    return lib().orc_sigma_pair(Z, E)


def mu(code, E):
    out = (C.c_double * 3)()
    if lib().orc_mu(code, E, out) != 0:
        raise ValueError("unknown material code %r" % code)
    return tuple(out)


class Tables:
    """Log-energy tables (binary32 values, mm^-1), layout [n_mat][3][n_grid]."""

    def __init__(self, ptr):
        self._p = ptr
        t = ptr.contents
        self.n_mat, self.n_grid = t.n_mat, t.n_grid
        self.lnE_min, self.lnE_max = t.lnE_min, t.lnE_max

    def e_range(self, m, T_keV):
        """CSDA range (mm, unit density scale) of table material m at T."""
        return lib().orc_e_range(self._p, m, T_keV)

    def e_energy_after(self, m, T_keV, L_mm):
        """Kinetic energy left after L mm in table material m."""
        return lib().orc_e_energy_after(self._p, m, T_keV, L_mm)

    def e_range_array(self):
        """[n_mat][e_n] CSDA ranges (mm) and the kinetic energies of the grid (keV)."""
        t = self._p.contents
        a = np.ctypeslib.as_array(t.e_range, shape=(t.n_mat * t.e_n,)).reshape(t.n_mat, t.e_n).copy()
        return a, np.exp(np.linspace(t.lnT_min, t.lnT_max, t.e_n))

    @classmethod
    def build(cls, codes, n_grid=1000, E_min=10.0, E_max=3000.0):
        c = (C.c_int * len(codes))(*codes)
        p = lib().orc_tables_build(c, len(codes), n_grid, E_min, E_max)
        if not p:
            raise ValueError("table build failed")
        return cls(p)

    @classmethod
    def from_array(cls, mu, E_min=10.0, E_max=3000.0):
        a = np.ascontiguousarray(mu, dtype=np.float32)
        n_mat, three, n_grid = a.shape
        assert three == 3
        p = lib().orc_tables_from_array(n_mat, n_grid, E_min, E_max, _ptr(a, C.c_float))
        if not p:
            raise ValueError("bad table")
        return cls(p)

    def array(self):
        n = self.n_mat * 3 * self.n_grid
        return np.ctypeslib.as_array(self._p.contents.mu, shape=(n,)).reshape(
            self.n_mat, 3, self.n_grid).copy()

    def set_mu(self, mu):
        """Replace the photon table in place (same [n_mat][3][n_grid] shape), keeping
        the charged-particle ranges of tables built from material codes."""
        a = np.ascontiguousarray(mu, dtype=np.float32)
        assert a.shape == (self.n_mat, 3, self.n_grid)
        C.memmove(self._p.contents.mu, a.ctypes.data, a.nbytes)

    def eval(self, m, E):
        out = (C.c_double * 3)()
        lib().orc_tables_eval(self._p, m, E, out)
        return tuple(out)

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.orc_tables_free(self._p)
            self._p = None


# ---------------- meshes ----------------

@dataclass
class Det:
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

    def c(self):
        p = DetParams()
        p.kind = self.kind
        for i in range(10):
            p.d[i] = self.d[i]
        for i in range(7):
            p.D[i] = self.D[i]
        p.n_theta, p.n_phi, p.z_slices = self.n_theta, self.n_phi, self.z_slices
        p.cup_rim_drop, p.sep_delta = self.cup_rim_drop, self.sep_delta
        p.has_source_solid = self.has_source_solid
        p.src_r, p.src_h, p.src_z0, p.src_n_sides = self.src_r, self.src_h, self.src_z0, self.src_n_sides
        p.groove_r, p.groove_w, p.groove_d = self.groove_r, self.groove_w, self.groove_d
        p.flange_r_in, p.flange_r_out, p.flange_h, p.flange_z_top = (self.flange_r_in, self.flange_r_out,
                                                                    self.flange_h, self.flange_z_top)
        p.n_bolt_holes, p.bolt_n_sides, p.bolt_r, p.bolt_rc = (self.n_bolt_holes, self.bolt_n_sides, self.bolt_r,
                                                               self.bolt_rc)
        return p


class Mesh:
    def __init__(self, ptr):
        self._p = ptr
        m = ptr.contents
        self.n_vert, self.n_tri, self.n_solid = m.n_vert, m.n_tri, m.n_solid

    @classmethod
    def build(cls, det: Det):
        out = C.POINTER(MeshC)()
        p = det.c()
        rc = lib().orc_mesh_build(C.byref(p), C.byref(out))
        if rc != 0:
            raise ValueError("oracle mesh build failed: %d" % rc)
        return cls(out)

    @classmethod
    def from_arrays(cls, xyz, tri, tri_solid, material, active, group, parent):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        ts = np.ascontiguousarray(tri_solid, dtype=np.int32)
        mats = [np.ascontiguousarray(a, dtype=np.int32) for a in (material, active, group, parent)]
        p = lib().orc_mesh_from_arrays(len(xyz), _ptr(xyz, C.c_double), len(tri), _ptr(tri, C.c_int),
                                       _ptr(ts, C.c_int), len(mats[0]),
                                       *[_ptr(a, C.c_int) for a in mats])
        return cls(p)

    def arrays(self):
        m = self._p.contents
        xyz = np.ctypeslib.as_array(m.xyz, shape=(self.n_vert * 3,)).reshape(-1, 3).copy()
        tri = np.ctypeslib.as_array(m.tri, shape=(self.n_tri * 3,)).reshape(-1, 3).copy()
        ts = np.ctypeslib.as_array(m.tri_solid, shape=(self.n_tri,)).copy()
        solids = {k: np.ctypeslib.as_array(getattr(m, "solid_" + k), shape=(self.n_solid,)).copy()
                  for k in ("material", "active", "group", "parent")}
        return xyz, tri, ts, solids

    def volume(self, s):
        return lib().orc_mesh_volume(self._p, s)

    def area(self, s):
        return lib().orc_mesh_area(self._p, s)

    def euler(self, s):
        return lib().orc_mesh_euler(self._p, s)

    def open_edges(self, s):
        return lib().orc_mesh_open_edges(self._p, s)

    def locate(self, p, d):
        a = (C.c_double * 3)(*p)
        b = (C.c_double * 3)(*d)
        return lib().orc_locate(self._p, a, b)

    def nearest_hit(self, o, d, t_min=0.0, exclude=-1):
        a = (C.c_double * 3)(*o)
        b = (C.c_double * 3)(*d)
        t = C.c_double()
        e = C.c_int()
        k = lib().orc_nearest_hit(self._p, a, b, t_min, exclude, C.byref(t), C.byref(e))
        return k, t.value, e.value

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.orc_mesh_free(self._p)
            self._p = None


# ---------------- sources and transport ----------------

@dataclass
class Source:
    kind: int = SRC_POINT
    pos: tuple = (0.0, 0.0, 0.0)
    dir: tuple = (0.0, 0.0, -1.0)
    radius: float = 0.0
    height: float = 0.0
    n_sides: int = 48

    def c(self):
        s = SourceC()
        s.kind = self.kind
        for i in range(3):
            s.pos[i] = self.pos[i]
            s.dir[i] = self.dir[i]
        s.radius, s.height, s.n_sides = self.radius, self.height, self.n_sides
        return s


def sample_birth(src: Source, seed, hid, inst=0):
    p = (C.c_double * 3)()
    d = (C.c_double * 3)()
    s = src.c()
    lib().orc_sample_birth(C.byref(s), seed, hid, inst, p, d)
    return np.array(p), np.array(d)


def kahn_samples(k, n, seed=1):
    out = np.zeros(n, dtype=np.float64)
    if lib().orc_kahn_samples(k, seed, n, _ptr(out, C.c_double)) != 0:
        raise RuntimeError("Kahn sampler exceeded its trial bound")
    return out


@dataclass
class Result:
    tally: dict
    spectrum: np.ndarray
    edep: np.ndarray | None
    n_bins: int
    e_max: float

    @property
    def fepe(self):
        return self.tally["n_fep"] / self.tally["n_hist"]

    @property
    def sigma(self):
        p, n = self.fepe, self.tally["n_hist"]
        return (p * (1 - p) / n) ** 0.5

    def dfepe(self, g):
        return self.tally["fep_score"][g] / self.tally["n_hist"]

    def dfepe_sigma(self, g):
        n = self.tally["n_hist"]
        m = self.tally["fep_score"][g] / n
        m2 = self.tally["fep_score_sq"][g] / n
        return max(m2 - m * m, 0.0) ** 0.5 / n ** 0.5


E_TMIN = 1.0   # keV: charged particles below this deposit where they are


def e_stopping(code, T_keV):
    """(collision, total) mass stopping power of material `code` for an electron
    of kinetic energy T, MeV cm^2/g."""
    c, t = C.c_double(), C.c_double()
    if lib().orc_e_stopping(code, T_keV, C.byref(c), C.byref(t)) != 0:
        raise ValueError("unknown material code %r" % code)
    return c.value, t.value


def e_track(mesh: Mesh, tables: Tables, p, u, T_keV, region, weight=1.0, group_scale=()):
    """One charged-particle line (e_model 1): returns (active deposit, all deposits,
    escaped) in keV; raises on a geometry error."""
    o = OptsC()
    o.e_model = 1
    o.n_group = len(group_scale)
    for i, s in enumerate(group_scale):
        o.group_scale[i] = s
    pp = (C.c_double * 3)(*p)
    uu = (C.c_double * 3)(*u)
    out = (C.c_double * 3)()
    rc = lib().orc_e_track(mesh._p, tables._p, C.byref(o), pp, uu, T_keV, weight, region, out)
    if rc != 0:
        raise ValueError("oracle e_track failed: %d" % rc)
    return tuple(out)


def transport(mesh: Mesh, tables: Tables, src: Source, energy, n_hist, seed=1, history_offset=0,
              instance=0, e_cut=10.0, fep_delta=0.01, n_bins=4096, e_max=3000.0, step_cap=10000,
              group_scale=(), n_threads=None, want_edep=False, e_model=0) -> Result:
    o = OptsC()
    o.e_model = e_model
    o.seed, o.history_offset, o.instance = seed, history_offset, instance
    o.energy_keV, o.e_cut_keV, o.fep_delta_keV, o.e_max_keV = energy, e_cut, fep_delta, e_max
    o.n_bins, o.step_cap = n_bins, step_cap
    o.n_group = len(group_scale)
    for i, s in enumerate(group_scale):
        o.group_scale[i] = s
    T = TallyC()
    spec = np.zeros(n_bins, dtype=np.uint32)
    edep = np.zeros(n_hist, dtype=np.float64) if want_edep else None
    if n_threads is None:
        n_threads = max(1, min(os.cpu_count() or 1, 64))
    s = src.c()
    rc = lib().orc_transport(mesh._p, tables._p, C.byref(s), C.byref(o), n_hist, n_threads,
                             C.byref(T), _ptr(spec, C.c_uint32),
                             _ptr(edep, C.c_double) if edep is not None else None)
    if rc != 0:
        raise ValueError("oracle transport rejected its arguments: %d" % rc)
    tally = {}
    for name, _ in TallyC._fields_:
        v = getattr(T, name)
        tally[name] = list(v) if name.startswith("fep_score") else v
    return Result(tally, spec, edep, n_bins, e_max)
