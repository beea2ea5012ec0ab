"""Python face of libgadep, with the C ABI's names.

Only argument marshalling happens here: every step of mesh generation, BVH
construction, transport and tallying runs in the compiled library (host C++ for
DetMesh and the BVH, CUDA kernels for transport).  PyTorch provides device
buffers and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi
from .capi import check
from . import workloads as W


def _torch():
    import torch
    return torch


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(int(stream))
    torch = _torch()
    if torch.cuda.is_available():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(0)


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


# ---------------- DetMesh ----------------

class _Handle:
    """Owner of one library handle, released by close(), at the end of a
    with-block, or when the object is collected.  The destroy function is bound
    at construction, so release needs no module globals (interpreter exit)."""
    _destroy_name = ""

    def __init__(self, handle):
        self._destroy = getattr(capi.load(), self._destroy_name)
        self._h = handle

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._destroy(h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        self.close()

    @property
    def handle(self):
        return self._h


class Mesh(_Handle):
    """Triangulated detector surfaces (library-owned handle)."""
    _destroy_name = "detmesh_destroy"

    def arrays(self):
        L = capi.load()
        xyz = C.POINTER(C.c_float)()
        tri = C.POINTER(C.c_int32)()
        ts = C.POINTER(C.c_int32)()
        sol = C.POINTER(capi.gadep_solid)()
        nv, nt, ns = C.c_int32(), C.c_int32(), C.c_int32()
        check(L.detmesh_get(self._h, C.byref(xyz), C.byref(nv), C.byref(tri), C.byref(ts), C.byref(nt),
                            C.byref(sol), C.byref(ns)))
        X = np.ctypeslib.as_array(xyz, shape=(nv.value * 3,)).reshape(-1, 3).copy()
        T = np.ctypeslib.as_array(tri, shape=(nt.value * 3,)).reshape(-1, 3).copy()
        S = np.ctypeslib.as_array(ts, shape=(nt.value,)).copy()
        solids = [dict(material=sol[i].material, active=sol[i].active, group=sol[i].group,
                       parent=sol[i].parent) for i in range(ns.value)]
        return X, T, S, solids

    def solid_stats(self, s):
        v, e = C.c_double(), C.c_int32()
        check(capi.load().detmesh_solid_stats(self._h, s, C.byref(v), C.byref(e)))
        return v.value, e.value

    def locate(self, p):
        a = (C.c_double * 3)(*p)
        out = C.c_int32()
        check(capi.load().detmesh_locate(self._h, a, C.byref(out)))
        return out.value


def detmesh_build(det: W.Detector) -> Mesh:
    p = capi.detmesh_params()
    p.kind = det.kind
    for i in range(10):
        p.d[i] = det.d[i]
    for i in range(7):
        p.D[i] = det.D[i]
    p.n_theta, p.n_phi, p.z_slices = det.n_theta, det.n_phi, det.z_slices
    p.cup_rim_drop, p.sep_delta = det.cup_rim_drop, det.sep_delta
    p.has_source_solid = det.has_source_solid
    p.src_r, p.src_h, p.src_z0, p.src_n_sides = det.src_r, det.src_h, det.src_z0, det.src_n_sides
    p.groove_r, p.groove_w, p.groove_d = det.groove_r, det.groove_w, det.groove_d
    p.flange_r_in, p.flange_r_out, p.flange_h, p.flange_z_top = (det.flange_r_in, det.flange_r_out,
                                                                det.flange_h, det.flange_z_top)
    p.n_bolt_holes, p.bolt_n_sides, p.bolt_r, p.bolt_rc = det.n_bolt_holes, det.bolt_n_sides, det.bolt_r, det.bolt_rc
    h = C.c_void_p()
    check(capi.load().detmesh_build(C.byref(p), C.byref(h)))
    return Mesh(h)


def detmesh_from_arrays(xyz, tri, tri_solid, material, active, group) -> Mesh:
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    ts = np.ascontiguousarray(tri_solid, dtype=np.int32)
    mats = [np.ascontiguousarray(a, dtype=np.int32) for a in (material, active, group)]
    h = C.c_void_p()
    check(capi.load().detmesh_from_arrays(_ptr(xyz, C.c_float), len(xyz), _ptr(tri, C.c_int32),
                                          _ptr(ts, C.c_int32), len(tri), *[_ptr(a, C.c_int32) for a in mats],
                                          len(mats[0]), C.byref(h)))
    return Mesh(h)


# ---------------- cross sections ----------------

def gadep_xs_build(codes=W.MATERIAL_CODES, n_grid=W.TABLE_N_GRID, E_min=W.TABLE_E_MIN, E_max=W.TABLE_E_MAX):
    c = np.ascontiguousarray(codes, dtype=np.int32)
    mu = np.zeros((len(c), 3, n_grid), dtype=np.float32)
    check(capi.load().gadep_xs_build(_ptr(c, C.c_int32), len(c), n_grid, E_min, E_max, _ptr(mu, C.c_float)))
    return mu


def gadep_erange_build(codes=W.MATERIAL_CODES, e_n=W.ERANGE_N, T_min=W.ERANGE_T_MIN, T_max=W.TABLE_E_MAX):
    """CSDA ranges [n_mat][e_n] (mm, unit density) of electrons for e_model 1."""
    c = np.ascontiguousarray(codes, dtype=np.int32)
    r = np.zeros((len(c), e_n), dtype=np.float32)
    check(capi.load().gadep_erange_build(_ptr(c, C.c_int32), len(c), e_n, T_min, T_max, _ptr(r, C.c_float)))
    return r


class Materials:
    """Attenuation tables mu[n_mat][3][n_grid] (host, float32) on a log grid, and
    optionally the charged-particle ranges e_range[n_mat][e_n] on [T_min, T_max]."""

    def __init__(self, mu, E_min=W.TABLE_E_MIN, E_max=W.TABLE_E_MAX, e_range=None, T_min=W.ERANGE_T_MIN,
                 T_max=W.TABLE_E_MAX):
        self.mu = np.ascontiguousarray(mu, dtype=np.float32)
        self.E_min, self.E_max = E_min, E_max
        self.e_range = None if e_range is None else np.ascontiguousarray(e_range, dtype=np.float32)
        self.T_min, self.T_max = T_min, T_max
        self.c = capi.gadep_materials(self.mu.shape[0], self.mu.shape[2], E_min, E_max,
                                      _ptr(self.mu, C.c_float))
        if self.e_range is not None:
            assert self.e_range.shape[0] == self.mu.shape[0]
            self.c.e_n, self.c.T_min, self.c.T_max = self.e_range.shape[1], T_min, T_max
            self.c.e_range = _ptr(self.e_range, C.c_float)

    @classmethod
    def default(cls):
        return cls(gadep_xs_build(), e_range=gadep_erange_build())


# ---------------- BVH ----------------

class Bvh(_Handle):
    """BVH of a mesh on one device (library-owned handle)."""
    _destroy_name = "gadep_bvh_destroy"

    def stats(self):
        s = capi.gadep_bvh_stats()
        check(capi.load().gadep_bvh_get_stats(self._h, C.byref(s)))
        d = {k: getattr(s, k) for k, _ in capi.gadep_bvh_stats._fields_}
        d["opts"] = {k: getattr(s.opts, k) for k, _ in capi.gadep_bvh_opts._fields_}
        return d

    def validate(self):
        check(capi.load().gadep_bvh_validate(self._h))


def bvh_opts(**kw) -> "capi.gadep_bvh_opts":
    """gadep_bvh_opts with the library defaults, then the given fields
    (max_leaf, c_trav, c_tri, split_alpha, max_dup, clip_ratio, clip_pieces)."""
    o = capi.gadep_bvh_opts()
    capi.load().gadep_bvh_opts_default(C.byref(o))
    for k, v in kw.items():
        if k not in dict(capi.gadep_bvh_opts._fields_):
            raise TypeError("unknown BVH option %r" % k)
        setattr(o, k, v)
    return o


def gadep_bvh_build(mesh: Mesh, device: int = 0, **opts) -> Bvh:
    """BVH of the mesh on `device` (-1: host copy only); keyword options as in
    bvh_opts (defaults: the library's)."""
    h = C.c_void_p()
    if opts:
        check(capi.load().gadep_bvh_build_opts(mesh.handle, C.byref(bvh_opts(**opts)), device, C.byref(h)))
    else:
        check(capi.load().gadep_bvh_build(mesh.handle, device, C.byref(h)))
    return Bvh(h)


def gadep_nearest_hit(bvh: Bvh, rays, regions=None, stream=None):
    """rays: CUDA float32 tensor [n, 8] = (o, t_min, d, exclude as float bits);
    regions: optional CUDA int32 tensor [n] (0 = world, s + 1 = solid s)."""
    torch = _torch()
    assert rays.is_cuda and rays.dtype == torch.float32 and rays.shape[1] == 8 and rays.is_contiguous()
    n = rays.shape[0]
    if regions is not None:
        assert regions.is_cuda and regions.dtype == torch.int32 and regions.numel() == n
    t = torch.empty(n, dtype=torch.float32, device=rays.device)
    tri = torch.empty(n, dtype=torch.int32, device=rays.device)
    ent = torch.empty(n, dtype=torch.int32, device=rays.device)
    check(capi.load().gadep_nearest_hit(bvh.handle, rays.data_ptr(),
                                        regions.data_ptr() if regions is not None else None, n,
                                        t.data_ptr(), tri.data_ptr(), ent.data_ptr(), _stream(stream)))
    return t, tri, ent


def gadep_philox_words(seed, hid, inst, n_words, device="cuda", stream=None):
    torch = _torch()
    out = torch.empty(n_words, dtype=torch.int32, device=device)
    check(capi.load().gadep_philox_words(seed, hid, inst, n_words, out.data_ptr(), _stream(stream)))
    return out


# ---------------- transport ----------------

def make_opts(**kw) -> capi.gadep_opts:
    o = capi.gadep_opts()
    capi.load().gadep_opts_default(C.byref(o))
    scales = kw.pop("group_scale", None)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError("unknown option %r" % k)
        setattr(o, k, v)
    if scales is not None:
        for i, s in enumerate(scales):
            o.group_scale[i] = s
    return o


def make_source(src: W.Source) -> capi.gadep_source:
    s = capi.gadep_source()
    s.kind = src.kind
    for i in range(3):
        s.pos[i] = src.pos[i]
        s.dir[i] = src.dir[i]
    s.radius, s.height, s.n_sides, s.solid = src.radius, src.height, src.n_sides, src.solid
    return s


def make_instances(items):
    """items: iterable of (energy, W.Source, n_hist, instance id, group scales)."""
    items = list(items)
    arr = (capi.gadep_instance * len(items))()
    for i, (E, src, n, inst, scales) in enumerate(items):
        arr[i].energy_keV = E
        arr[i].src = make_source(src)
        arr[i].n_hist = n
        arr[i].instance = inst
        sc = list(scales) + [1.0] * (capi.MAX_GROUPS - len(scales))
        for g in range(capi.MAX_GROUPS):
            arr[i].group_scale[g] = sc[g]
    return arr


def measure_peaks(device=0):
    """(FP32 TFLOP/s, L2 read GB/s) of the device from the library's microbenchmarks."""
    f, l2 = C.c_double(), C.c_double()
    check(capi.load().gadep_measure_peaks(device, C.byref(f), C.byref(l2)))
    return f.value, l2.value


def result_dict(r: capi.gadep_result):
    return {k: getattr(r, k) for k, _ in capi.gadep_result._fields_}


def gadep_run(bvh: Bvh, mat: Materials, src: W.Source, energy, n_hist, instance=0, opts=None,
              spectrum=None, edep_trace=None, stream=None):
    """One instance.  spectrum: None (host numpy returned) or a CUDA uint32/int32 tensor.
    edep_trace: optional CUDA float32 tensor receiving the first len() deposits."""
    o = opts if opts is not None else make_opts()
    s = make_source(src)
    r = capi.gadep_result()
    if spectrum is None:
        spec = np.zeros(o.n_bins, dtype=np.uint32)
        sp = spec.ctypes.data
    else:
        spec = spectrum
        sp = spectrum.data_ptr()
    tp, nt = (edep_trace.data_ptr(), edep_trace.numel()) if edep_trace is not None else (None, 0)
    check(capi.load().gadep_run(bvh.handle, C.byref(mat.c), C.byref(s), energy, n_hist, instance, C.byref(o),
                                sp, tp, nt, C.byref(r), _stream(stream)))
    return result_dict(r), spec


def gadep_run_noalloc(bvh: Bvh, mat: Materials, src: W.Source, energy, n_hist, spectrum, instance=0, opts=None,
                      stream=None):
    """gadep_run for callers that cannot have the library allocate device memory
    (an application-owned allocator holds the device memory, or a loop cannot take
    cudaFree's device synchronisation): scratch lives in a fixed device array inside
    the library.  Runs the megakernel form (a wavefront variant is refused).
    spectrum: the caller's CUDA uint32/int32 tensor of n_bins counts.  The call
    synchronises its stream.  Calls that overlap on the GPU race on that array;
    the first call on a device should precede any stream capture."""
    o = opts if opts is not None else make_opts()
    s = make_source(src)
    r = capi.gadep_result()
    check(capi.load().gadep_run_noalloc(bvh.handle, C.byref(mat.c), C.byref(s), energy, n_hist, instance,
                                        C.byref(o), spectrum.data_ptr(), C.byref(r), _stream(stream)))
    return result_dict(r)


def gadep_run_batch(bvh: Bvh, mat: Materials, instances, opts=None, spectra=None, stream=None):
    o = opts if opts is not None else make_opts()
    n = len(instances)
    res = (capi.gadep_result * n)()
    if spectra is None:
        spec = np.zeros((n, o.n_bins), dtype=np.uint32)
        sp = spec.ctypes.data
    else:
        spec, sp = spectra, spectra.data_ptr()
    check(capi.load().gadep_run_batch(bvh.handle, C.byref(mat.c), n, instances, C.byref(o), sp, res,
                                      _stream(stream)))
    return [result_dict(r) for r in res], spec


def gadep_grad(bvh: Bvh, mat: Materials, instances, opts, spectra=None, stream=None):
    n = len(instances)
    ng = opts.n_group
    res = (capi.gadep_result * n)()
    d = np.zeros((n, ng), dtype=np.float64)
    ds = np.zeros((n, ng), dtype=np.float64)
    if spectra is None:
        spec = np.zeros((n, opts.n_bins), dtype=np.uint32)
        sp = spec.ctypes.data
    else:
        spec, sp = spectra, spectra.data_ptr()
    check(capi.load().gadep_grad(bvh.handle, C.byref(mat.c), n, instances, C.byref(opts), sp, res,
                                 _ptr(d, C.c_double), _ptr(ds, C.c_double), _stream(stream)))
    return [result_dict(r) for r in res], spec, d, ds


def gadep_count_work(bvh: Bvh, mat: Materials, instances, opts=None, stream=None):
    """Traversal work of a batch: (results, 4-wide nodes visited, triangles tested,
    relocated queries, child boxes tested)."""
    o = opts if opts is not None else make_opts()
    n = len(instances)
    res = (capi.gadep_result * n)()
    nodes, tris, reloc, boxes = C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_uint64()
    st = capi.load().gadep_count_work(bvh.handle, C.byref(mat.c), n, instances, C.byref(o), res,
                                      C.byref(nodes), C.byref(tris), C.byref(reloc), C.byref(boxes),
                                      _stream(stream))
    if st != capi.GADEP_E_DEVICE:
        check(st)
    return [result_dict(r) for r in res], nodes.value, tris.value, reloc.value, boxes.value


class Plan(_Handle):
    """Device-resident batched run: create once, launch repeatedly (graph-capturable)."""
    _destroy_name = "gadep_plan_destroy"

    def __init__(self, bvh: Bvh, mat: Materials, instances, opts=None, grad=False):
        super().__init__(None)
        self._keep = (bvh, mat, instances)
        self.opts = opts if opts is not None else make_opts()
        self.n_inst = len(instances)
        self.grad = grad
        h = C.c_void_p()
        check(capi.load().gadep_plan_create(bvh.handle, C.byref(mat.c), self.n_inst, instances,
                                            C.byref(self.opts), 1 if grad else 0, C.byref(h)))
        self._h = h

    def shape(self):
        g, b, s = C.c_int32(), C.c_int32(), C.c_int32()
        check(capi.load().gadep_plan_shape(self._h, C.byref(g), C.byref(b), C.byref(s)))
        return g.value, b.value, s.value

    def launch(self, spectra=None, stream=None):
        check(capi.load().gadep_plan_launch(self._h, spectra.data_ptr() if spectra is not None else None,
                                            _stream(stream)))

    def set_timing(self, on=True):
        """Record a CUDA event pair around every kernel of later launches."""
        check(capi.load().gadep_plan_set_timing(self._h, 1 if on else 0))

    def kernel_stats(self, reset=False):
        """{kind: (launches, ms)} since the last reset; ms is 0 unless timing was on."""
        ks = capi.gadep_kernel_stats()
        check(capi.load().gadep_plan_kernel_stats(self._h, C.byref(ks), 1 if reset else 0))
        return {k: (int(ks.launches[i]), float(ks.ms[i])) for i, k in enumerate(capi.KERNEL_KINDS)}

    def queue_sizes(self, max_entries=8192, stream=None):
        """Trace queue size of each wavefront iteration of the last launch (empty
        for a megakernel plan)."""
        buf = (C.c_uint32 * max_entries)()
        n = C.c_int32()
        check(capi.load().gadep_plan_queue_sizes(self._h, buf, max_entries, C.byref(n), _stream(stream)))
        return [int(buf[i]) for i in range(n.value)]

    def results(self, want_spectra=True, stream=None, raise_device_errors=True):
        """Tallies of the last launch.  With raise_device_errors=False a set device
        error word is reported through each result's n_err / dev_err instead."""
        res = (capi.gadep_result * self.n_inst)()
        spec = np.zeros((self.n_inst, self.opts.n_bins), dtype=np.uint32) if want_spectra else None
        ng = max(self.opts.n_group, 1)
        d = np.zeros((self.n_inst, ng), dtype=np.float64)
        ds = np.zeros((self.n_inst, ng), dtype=np.float64)
        st = capi.load().gadep_plan_results(self._h, spec.ctypes.data if spec is not None else None, res,
                                            _ptr(d, C.c_double), _ptr(ds, C.c_double), _stream(stream))
        if not (st == capi.GADEP_E_DEVICE and not raise_device_errors):
            check(st)
        return [result_dict(r) for r in res], spec, d, ds
