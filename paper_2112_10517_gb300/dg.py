"""ctypes binding of libdg.so (include/dg.h): argument marshalling only; every step of the RHS runs in the
library's CUDA kernels. PyTorch provides device memory and streams.

The module-level functions mirror the C entry points one to one (dg_init, dg_rhs, dg_step, dg_entropy_rate,
dg_check_status, dg_free, ...) and take raw pointers; the class ``DG`` wraps one context for torch tensors.
Importing this module loads libdg.so and raises if it has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libdg.so not found at %s: build it with `python -m paper_2112_10517_gb300.build` "
                      "(needs nvcc); there is no CPU fallback" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

# ---- status codes and enums (include/dg.h) ----
DG_OK, DG_ERR_ARG, DG_ERR_CUDA, DG_ERR_OOM, DG_ERR_UNSUPPORTED, DG_ERR_NONPHYSICAL, DG_ERR_TIMEOUT = range(7)
DG_MAP_AFFINE, DG_MAP_SINE, DG_MAP_NODES = 0, 1, 2
DG_SURF_EC, DG_SURF_EC_LLF = 0, 1
DG_FP64, DG_FP32 = 0, 1
DG_VOL_RANOCHA, DG_VOL_SHIMA = 0, 1
FLUXES = {"ranocha": DG_VOL_RANOCHA, "shima": DG_VOL_SHIMA}
DG_LOGMEAN_SHARED_RCP, DG_LOGMEAN_ALG, DG_LOGMEAN_ALG_POLY = 0, 1, 2
LOGMEANS = {"rcp": DG_LOGMEAN_SHARED_RCP, "alg": DG_LOGMEAN_ALG, "alg_poly": DG_LOGMEAN_ALG_POLY}
DG_NODES_LGL, DG_NODES_GAUSS = 0, 1
NODES = {"lgl": DG_NODES_LGL, "gauss": DG_NODES_GAUSS}
DG_STAGING_AUTO, DG_STAGING_DIRECT, DG_STAGING_PIPELINED = 0, 1, 2
DG_LAUNCH_OVERLAP, DG_LAUNCH_SERIAL = 0, 1
STAGINGS = {"auto": DG_STAGING_AUTO, "direct": DG_STAGING_DIRECT, "pipelined": DG_STAGING_PIPELINED}
LAUNCHES = {"overlap": DG_LAUNCH_OVERLAP, "serial": DG_LAUNCH_SERIAL}
DG_RK4_CLASSIC, DG_LSRK45_CK = 0, 1
DG_REGION_INTERIOR, DG_REGION_BOUNDARY = 0, 1
KERNEL_VOLUME, KERNEL_INTERFACE, KERNEL_PROJECT = 0, 1, 2

EXPORTED = ["dg_init", "dg_rhs", "dg_step", "dg_entropy_rate", "dg_check_status", "dg_get_info",
            "dg_get_node_coords", "dg_get_metrics", "dg_profile_enable", "dg_profile_read", "dg_launch_count",
            "dg_free", "dg_status_string", "dg_rhs_noalloc", "dg_batch_create", "dg_batch_rhs",
            "dg_batch_autotune", "dg_batch_set_tuning", "dg_batch_free", "dg_vjp", "dg_selftest_wait_timeout",
            "dg_profile_enable_kernels", "dg_profile_enable_sampled", "dg_step_host", "dg_rhs_host",
            "dg_init_part", "dg_part_get_info", "dg_part_pack", "dg_part_unpack", "dg_step_stage", "dg_stage_input",
            "dg_conserved_totals", "dg_stage_interface", "dg_stage_volume"]


class DgMesh(ctypes.Structure):
    _fields_ = [("ndims", ctypes.c_int), ("nelem", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("mapping", ctypes.c_int), ("map_amp", ctypes.c_double),
                ("node_xyz_host", ctypes.POINTER(ctypes.c_double))]


class DgMetrics(ctypes.Structure):
    _fields_ = [("Ja_host", ctypes.POINTER(ctypes.c_double)), ("J_host", ctypes.POINTER(ctypes.c_double))]


class DgOpts(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("volume_flux", ctypes.c_int), ("surface_flux", ctypes.c_int),
                ("precision", ctypes.c_int), ("precompute_logs", ctypes.c_int), ("logmean", ctypes.c_int),
                ("nodes", ctypes.c_int), ("staging", ctypes.c_int), ("launch", ctypes.c_int),
                ("p_ref", ctypes.c_double)]


class DgPart(ctypes.Structure):
    _fields_ = [("begin", ctypes.c_int), ("end", ctypes.c_int)]


class DgPartInfo(ctypes.Structure):
    _fields_ = [("layer", ctypes.c_longlong), ("own_elems", ctypes.c_longlong), ("ghost_elems", ctypes.c_longlong),
                ("halo_len", ctypes.c_longlong), ("begin", ctypes.c_int), ("end", ctypes.c_int)]


class DgInfo(ctypes.Structure):
    _fields_ = [("ndims", ctypes.c_int), ("polydeg", ctypes.c_int), ("nvar", ctypes.c_int),
                ("nodes_per_elem", ctypes.c_int), ("nelem_total", ctypes.c_longlong), ("ndofs", ctypes.c_longlong),
                ("state_len", ctypes.c_longlong), ("precision", ctypes.c_int), ("surface_flux", ctypes.c_int)]


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_sig = {
    "dg_init": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(DgMesh), ctypes.c_int, ctypes.POINTER(DgMetrics),
                               ctypes.POINTER(DgOpts)]),
    "dg_rhs": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, _vp]),
    "dg_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp]),
    "dg_entropy_rate": (ctypes.c_int, [_vp, _vp, _vp, _dp, _dp, _vp]),
    "dg_check_status": (ctypes.c_int, [_vp]),
    "dg_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(DgInfo)]),
    "dg_get_node_coords": (ctypes.c_int, [_vp, _dp]),
    "dg_get_metrics": (ctypes.c_int, [_vp, _dp, _dp]),
    "dg_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "dg_profile_enable_kernels": (ctypes.c_int, [_vp, ctypes.c_uint]),
    "dg_profile_enable_sampled": (ctypes.c_int, [_vp, ctypes.c_uint, ctypes.c_int]),
    "dg_step_host": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp]),
    "dg_rhs_host": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, _vp]),
    "dg_profile_read": (ctypes.c_int, [_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "dg_launch_count": (ctypes.c_longlong, [_vp]),
    "dg_free": (None, [_vp]),
    "dg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "dg_rhs_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, _vp]),
    "dg_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp),
                                       ctypes.POINTER(_vp)]),
    "dg_batch_rhs": (ctypes.c_int, [_vp, _vp]),
    "dg_batch_autotune": (ctypes.c_int, [_vp, ctypes.c_char_p, _vp, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]),
    "dg_batch_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "dg_batch_free": (None, [_vp]),
    "dg_vjp": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "dg_init_part": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(DgMesh), ctypes.c_int, ctypes.POINTER(DgOpts),
                                    ctypes.POINTER(DgPart)]),
    "dg_part_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(DgPartInfo)]),
    "dg_part_pack": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "dg_part_unpack": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "dg_step_stage": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                     _vp]),
    "dg_stage_input": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "dg_stage_interface": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
    "dg_stage_volume": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                       _vp]),
    "dg_conserved_totals": (ctypes.c_int, [_vp, _vp, _dp, _vp]),
    "dg_selftest_wait_timeout": (ctypes.c_int, [_vp, _vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class DGError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, dg_status_string(status).decode(), status))


def check(status: int, what: str):
    if status != DG_OK:
        raise DGError(status, what)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class DG:
    """One context of the flux-differencing LGL-DGSEM RHS on the current CUDA device.

    mapping: "affine", "sine" (x = xi + amp prod sin) or "nodes" (node_xyz [E, d, Nd] given).
    surface: "ec" or "llf"; precision: "fp64" or "fp32"; flux: "ranocha" (Ranocha's EC/KEP/PEP flux) or
    "shima" (the KEEP/PEP flux of Shima et al.), used in the volume and as the surface flux's central part.
    An affine mesh without node or metric overrides runs the Cartesian specialisation (constant Ja, 1/J).
    logmean ("rcp", "alg", "alg_poly") and precompute_logs select how the volume terms evaluate the logarithmic
    means of Ranocha's flux (Sec. 3.1, 7.2; see dg_opts in include/dg.h); the defaults are the fastest.
    nodes: "lgl" (flux-differencing LGL-DGSEM) or "gauss" (Legendre-Gauss collocation with entropy projection,
    Sec. 6; affine meshes, FP64, Ranocha's flux).
    staging: "pipelined" (the volume kernel copies tiles with asynchronous copies that overlap computation),
    "direct" (one CTA per tile, loads by its threads) or "auto" (pipelined on meshes with enough tiles per CTA,
    except FP32 at p = 2); the same terms, added in another order (the surface term starts the pipelined kernel's
    line sums and follows the direct kernel's), so the two agree to rounding.
    launch: "overlap" (each interface and pipelined volume kernel is scheduled ahead and starts as the kernel
    before it ends, waiting for its writes before reading them) or "serial" (ordinary launches); the same values.
    p_ref: FP32 mode only, a reference pressure (0: none) on which the momentum equations' pressure terms are
    evaluated as p - p_ref (the same scheme up to rounding; for low-Mach flows, the flow's mean pressure).
    part: (begin, end) makes the context of the slab of element layers [begin, end) of the mesh along its last
    direction (dg_init_part): state tensors then hold a ghost layer in front of the slab's elements, filled by
    unpack() from the neighbouring slabs' pack() buffers before each RHS or Runge-Kutta stage.
    """

    def __init__(self, ndims: int, nelem, polydeg: int, lo=None, hi=None, mapping: str = "affine", amp: float = 0.0,
                 node_xyz=None, Ja=None, J=None, gamma: float = 1.4, surface: str = "llf",
                 precision: str = "fp64", flux: str = "ranocha", logmean: str = "rcp",
                 precompute_logs: bool = False, nodes: str = "lgl", staging: str = "auto",
                 launch: str = "overlap", p_ref: float = 0.0, part=None):
        mesh = DgMesh()
        mesh.ndims = ndims
        ne = list(nelem) + [1] * (3 - len(nelem))
        lo = list(lo) if lo is not None else [-1.0] * ndims
        hi = list(hi) if hi is not None else [1.0] * ndims
        for i in range(3):
            mesh.nelem[i] = int(ne[i])
            mesh.lo[i] = float(lo[i]) if i < len(lo) else 0.0
            mesh.hi[i] = float(hi[i]) if i < len(hi) else 1.0
        mesh.mapping = {"affine": DG_MAP_AFFINE, "sine": DG_MAP_SINE, "nodes": DG_MAP_NODES}[mapping]
        mesh.map_amp = float(amp)
        self._keep = []
        if node_xyz is not None:
            xyz = np.ascontiguousarray(node_xyz, dtype=np.float64)
            self._keep.append(xyz)
            mesh.node_xyz_host = _dptr(xyz)
        met = None
        if Ja is not None:
            Ja = np.ascontiguousarray(Ja, dtype=np.float64)
            J = np.ascontiguousarray(J, dtype=np.float64)
            self._keep += [Ja, J]
            met = DgMetrics(_dptr(Ja), _dptr(J))
        opts = DgOpts()
        opts.gamma = gamma
        opts.volume_flux = FLUXES[flux]
        opts.logmean = LOGMEANS[logmean]
        opts.precompute_logs = 1 if precompute_logs else 0
        opts.nodes = NODES[nodes]
        opts.staging = STAGINGS[staging]
        opts.launch = LAUNCHES[launch]
        opts.p_ref = float(p_ref)
        opts.surface_flux = {"ec": DG_SURF_EC, "llf": DG_SURF_EC_LLF}[surface]
        opts.precision = {"fp64": DG_FP64, "fp32": DG_FP32}[precision]
        ctx = ctypes.c_void_p()
        if part is None:
            check(dg_init(ctypes.byref(ctx), ctypes.byref(mesh), int(polydeg),
                          ctypes.byref(met) if met is not None else None, ctypes.byref(opts)), "dg_init")
        else:
            if met is not None:
                raise ValueError("a partitioned context computes its own metric terms")
            dp = DgPart(int(part[0]), int(part[1]))
            check(dg_init_part(ctypes.byref(ctx), ctypes.byref(mesh), int(polydeg), ctypes.byref(opts),
                               ctypes.byref(dp)), "dg_init_part")
        self.ctx = ctx
        info = DgInfo()
        check(dg_get_info(ctx, ctypes.byref(info)), "dg_get_info")
        self.ndims, self.polydeg, self.nvar = info.ndims, info.polydeg, info.nvar
        self.nodes_per_elem, self.nelem_total = info.nodes_per_elem, info.nelem_total
        self.ndofs, self.state_len = info.ndofs, info.state_len
        self.shape = (self.nelem_total, self.nvar, self.nodes_per_elem)
        self.precision = precision
        self.part = None
        if part is not None:
            pi = DgPartInfo()
            check(dg_part_get_info(ctx, ctypes.byref(pi)), "dg_part_get_info")
            self.part = pi
            self.ghost_elems, self.halo_len = pi.ghost_elems, pi.halo_len
        import torch
        self.device = torch.device("cuda", torch.cuda.current_device())

    # ---- lifetime ----
    def close(self):
        if getattr(self, "ctx", None):
            dg_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- argument checks ----
    def _state(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
            raise TypeError("%s must be a CUDA float64 tensor" % name)
        if tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError("%s must be contiguous with shape %s, got %s" % (name, self.shape, tuple(t.shape)))
        return ctypes.c_void_p(t.data_ptr())

    # ---- entry points ----
    def rhs(self, u, du=None, stream=None):
        import torch
        if du is None:
            du = torch.empty_like(u)
        check(dg_rhs(self.ctx, self._state(u, "u"), self._state(du, "du"), 0.0, _stream_handle(stream)), "dg_rhs")
        return du

    def step(self, u, dt: float, scheme: int = DG_RK4_CLASSIC, scratch=None, stream=None):
        import torch
        nreg = 2 if scheme == DG_RK4_CLASSIC else 1
        if scratch is None:
            scratch = torch.empty((nreg,) + self.shape, dtype=torch.float64, device=u.device)
        if scratch.numel() < nreg * self.state_len or scratch.dtype != torch.float64 or not scratch.is_contiguous():
            raise ValueError("scratch must be contiguous float64 with %d elements" % (nreg * self.state_len))
        check(dg_step(self.ctx, self._state(u, "u"), ctypes.c_void_p(scratch.data_ptr()), 0.0, float(dt), int(scheme),
                      _stream_handle(stream)), "dg_step")
        return u

    def step_stage(self, u, scratch, dt: float, scheme: int, stage: int, stream=None):
        """Stage `stage` of dg_step's scheme (dg_step_stage); it reads u or scratch[0] (stage_input)."""
        nreg = 2 if scheme == DG_RK4_CLASSIC else 1
        if scratch.numel() < nreg * self.state_len or scratch.dtype != __import__("torch").float64 or \
                not scratch.is_contiguous():
            raise ValueError("scratch must be contiguous float64 with %d elements" % (nreg * self.state_len))
        check(dg_step_stage(self.ctx, self._state(u, "u"), ctypes.c_void_p(scratch.data_ptr()), 0.0, float(dt),
                            int(scheme), int(stage), _stream_handle(stream)), "dg_step_stage")
        return u

    def _scratch(self, scratch, scheme):
        nreg = 2 if scheme == DG_RK4_CLASSIC else 1
        if scratch.numel() < nreg * self.state_len or scratch.dtype != __import__("torch").float64 or \
                not scratch.is_contiguous():
            raise ValueError("scratch must be contiguous float64 with %d elements" % (nreg * self.state_len))
        return ctypes.c_void_p(scratch.data_ptr())

    def stage_interface(self, u, scratch, scheme: int, stage: int, region: int, stream=None):
        """The interface fluxes of stage `stage`'s input for DG_REGION_INTERIOR (faces that read no ghost-layer data)
        or DG_REGION_BOUNDARY (the rest) of a slab (dg_stage_interface)."""
        check(dg_stage_interface(self.ctx, self._state(u, "u"), self._scratch(scratch, scheme), int(scheme),
                                 int(stage), int(region), _stream_handle(stream)), "dg_stage_interface")

    def stage_volume(self, u, scratch, dt: float, scheme: int, stage: int, stream=None):
        """The volume kernel and update of stage `stage` after both regions' interface fluxes (dg_stage_volume)."""
        check(dg_stage_volume(self.ctx, self._state(u, "u"), self._scratch(scratch, scheme), 0.0, float(dt),
                              int(scheme), int(stage), _stream_handle(stream)), "dg_stage_volume")
        return u

    @staticmethod
    def stage_input(scheme: int, stage: int) -> int:
        """0: the stage reads u; 1: it reads scratch[0]."""
        return int(dg_stage_input(int(scheme), int(stage)))

    def halo_buffers(self):
        """Four float64 device tensors of halo_len values: send_lo, send_hi, recv_lo, recv_hi."""
        import torch
        return [torch.empty(self.halo_len, dtype=torch.float64, device=self.device) for _ in range(4)]

    def pack(self, state, send_lo, send_hi, stream=None):
        check(dg_part_pack(self.ctx, self._state(state, "state"), ctypes.c_void_p(send_lo.data_ptr()),
                           ctypes.c_void_p(send_hi.data_ptr()), _stream_handle(stream)), "dg_part_pack")

    def unpack(self, state, recv_lo, recv_hi, stream=None):
        check(dg_part_unpack(self.ctx, self._state(state, "state"), ctypes.c_void_p(recv_lo.data_ptr()),
                             ctypes.c_void_p(recv_hi.data_ptr()), _stream_handle(stream)), "dg_part_unpack")

    def conserved_totals(self, q, stream=None) -> np.ndarray:
        out = np.zeros(self.nvar)
        check(dg_conserved_totals(self.ctx, self._state(q, "q"), _dptr(out), _stream_handle(stream)),
              "dg_conserved_totals")
        return out

    def vjp(self, u, gbar, ubar=None, stream=None):
        """ubar = (d RHS/du)^T gbar (dg_vjp)."""
        import torch
        if ubar is None:
            ubar = torch.empty_like(u)
        check(dg_vjp(self.ctx, self._state(u, "u"), self._state(gbar, "gbar"), self._state(ubar, "ubar"),
                     _stream_handle(stream)), "dg_vjp")
        return ubar

    def entropy_rate(self, u, du, stream=None):
        out = ctypes.c_double()
        ab = ctypes.c_double()
        check(dg_entropy_rate(self.ctx, self._state(u, "u"), self._state(du, "du"), ctypes.byref(out),
                              ctypes.byref(ab), _stream_handle(stream)), "dg_entropy_rate")
        return out.value, ab.value

    # ---- host-resident state: the library copies in and out (asynchronous for pinned tensors) ----
    def _host_state(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.is_cuda:
            raise TypeError("%s must be a CPU float64 tensor" % name)
        if tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError("%s must be contiguous with shape %s, got %s" % (name, self.shape, tuple(t.shape)))
        return ctypes.c_void_p(t.data_ptr())

    def step_host(self, u_host, dt: float, scheme: int = DG_RK4_CLASSIC, stream=None):
        """One time step of the host state u_host (dg_step_host); synchronize the stream before reading it."""
        check(dg_step_host(self.ctx, self._host_state(u_host, "u_host"), 0.0, float(dt), int(scheme),
                           _stream_handle(stream)), "dg_step_host")
        return u_host

    def rhs_host(self, u_host, du_host, stream=None):
        """du_host = RHS(u_host) through device copies (dg_rhs_host); synchronize the stream before reading."""
        check(dg_rhs_host(self.ctx, self._host_state(u_host, "u_host"), self._host_state(du_host, "du_host"), 0.0,
                          _stream_handle(stream)), "dg_rhs_host")
        return du_host

    def check_status(self) -> int:
        return dg_check_status(self.ctx)

    def node_coords(self) -> np.ndarray:
        xyz = np.zeros((self.nelem_total, self.ndims, self.nodes_per_elem))
        check(dg_get_node_coords(self.ctx, _dptr(xyz)), "dg_get_node_coords")
        return xyz

    def metrics(self):
        Ja = np.zeros((self.nelem_total, self.ndims, self.ndims, self.nodes_per_elem))
        J = np.zeros((self.nelem_total, self.nodes_per_elem))
        check(dg_get_metrics(self.ctx, _dptr(Ja), _dptr(J)), "dg_get_metrics")
        return Ja, J

    def profile(self, on: bool, kernels=None, every: int = 1):
        """Time every kernel (kernels=None) or only the given kernel ids (KERNEL_*) while on; every: time each
        every-th launch of them."""
        if not on:
            check(dg_profile_enable(self.ctx, 0), "dg_profile_enable")
            return
        mask = 0xFFFFFFFF
        if kernels is not None:
            mask = 0
            for k in kernels:
                mask |= 1 << int(k)
        check(dg_profile_enable_sampled(self.ctx, mask, int(every)), "dg_profile_enable_sampled")

    def profile_read(self, kernel: int = KERNEL_VOLUME):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        check(dg_profile_read(self.ctx, int(kernel), ctypes.byref(ms), ctypes.byref(n)), "dg_profile_read")
        return ms.value, n.value

    def launch_count(self) -> int:
        return int(dg_launch_count(self.ctx))


class DGBatch:
    """A batch plan (dg_batch_create): contexts `ctxs` (DG objects) bound to state tensors u[i], du[i]."""

    def __init__(self, ctxs, us, dus):
        if not (len(ctxs) == len(us) == len(dus)) or not ctxs:
            raise ValueError("need one u and one du per context")
        for c, u, du in zip(ctxs, us, dus):
            c._state(u, "u")
            c._state(du, "du")
        n = len(ctxs)
        self.ctxs, self.us, self.dus = list(ctxs), list(us), list(dus)  # keep alive
        carr = (_vp * n)(*[c.ctx.value for c in ctxs])
        uarr = (_vp * n)(*[u.data_ptr() for u in us])
        darr = (_vp * n)(*[d.data_ptr() for d in dus])
        b = ctypes.c_void_p()
        check(dg_batch_create(ctypes.byref(b), carr, n, uarr, darr), "dg_batch_create")
        self.b = b
        self.ndofs = sum(c.ndofs for c in ctxs)

    def rhs(self, stream=None):
        check(dg_batch_rhs(self.b, _stream_handle(stream)), "dg_batch_rhs")

    def autotune(self, cache_path=None, stream=None):
        th = ctypes.c_int()
        cps = ctypes.c_int()
        check(dg_batch_autotune(self.b, cache_path.encode() if cache_path else None, _stream_handle(stream),
                                ctypes.byref(th), ctypes.byref(cps)), "dg_batch_autotune")
        return th.value, cps.value

    def set_tuning(self, threads: int, ctas_per_sm: int = 0):
        check(dg_batch_set_tuning(self.b, int(threads), int(ctas_per_sm)), "dg_batch_set_tuning")

    def close(self):
        if getattr(self, "b", None):
            dg_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rhs_function():
    """torch.autograd.Function: forward = dg_rhs, backward = dg_vjp. Usage: DGRhs.apply(ctx, u)."""
    import torch

    class DGRhs(torch.autograd.Function):
        @staticmethod
        def forward(fctx, ctx, u):
            fctx.dg = ctx
            fctx.save_for_backward(u)
            return ctx.rhs(u.contiguous())

        @staticmethod
        def backward(fctx, grad):
            (u,) = fctx.saved_tensors
            return None, fctx.dg.vjp(u.contiguous(), grad.contiguous())

    return DGRhs
