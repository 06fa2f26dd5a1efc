"""ctypes binding of the C ABI in include/pmg.h (argument marshalling only).

Device vectors are torch CUDA tensors (float64 unless a call says float32); every call
runs on torch's current CUDA stream.  Errors raise PmgError with the library's message.
"""
import ctypes
import os

import torch

from . import build as _build

PMG_OK, PMG_ERR_INVALID, PMG_ERR_OOM, PMG_ERR_CUDA = 0, 1, 2, 3
PMG_ERR_NOT_CONVERGED, PMG_ERR_NONFINITE, PMG_ERR_TIMEOUT = 4, 5, 6
PMG_FP64, PMG_MIXED_FP32, PMG_MIXED_BF16 = 0, 1, 2
PMG_PCG, PMG_FCG, PMG_PDC, PMG_IR, PMG_GMRES = 0, 1, 2, 3, 4
PMG_ASM_FDM = 0
PMG_ASM_DENSE = 1
PMG_ACTUAL = 0
PMG_FLAT_LINEARISED = 1

KERNEL_CLASSES = ["curved64", "curved32", "level64", "level32", "smooth64", "smooth32", "transfer",
                  "coarse", "vector", "setup", "vcycle_fused"]

STATUS_NAMES = {0: "PMG_OK", 1: "PMG_ERR_INVALID", 2: "PMG_ERR_OOM", 3: "PMG_ERR_CUDA",
                4: "PMG_ERR_NOT_CONVERGED", 5: "PMG_ERR_NONFINITE", 6: "PMG_ERR_TIMEOUT"}


class PmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class MeshDesc(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("x1", ctypes.c_double), ("h", ctypes.c_double),
                ("cells_x", ctypes.c_int), ("cells_z", ctypes.c_int), ("order", ctypes.c_int),
                ("periodic_x", ctypes.c_int), ("order_z", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("outer", ctypes.c_int), ("smoother", ctypes.c_int),
                ("precond_geom", ctypes.c_int), ("overlap", ctypes.c_int), ("nu", ctypes.c_int),
                ("omega", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("inner_max", ctypes.c_int), ("inner_tol", ctypes.c_double), ("nlevels", ctypes.c_int),
                ("level_orders", ctypes.c_int * 8), ("fuse_residual", ctypes.c_int), ("flat_kernel", ctypes.c_int),
                ("df64_outer", ctypes.c_int), ("gmres_restart", ctypes.c_int), ("sweep_kernel", ctypes.c_int),
                ("fuse_coarse", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("inner_iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_SIGNATURES = {
    "pmg_default_opts": (None, [ctypes.POINTER(Opts)]),
    "pmg_create": (_I, [ctypes.POINTER(MeshDesc), ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "pmg_destroy": (_I, [_P]),
    "pmg_num_nodes": (_I, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "pmg_level_info": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "pmg_level_kernels": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "pmg_fused_vcycle_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                   ctypes.POINTER(_I), _P]),
    "pmg_set_fused_vcycle": (_I, [_P, _I]),
    "pmg_level_sequence": (_I, [ctypes.POINTER(MeshDesc), ctypes.POINTER(Opts), ctypes.POINTER(_I),
                               ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "pmg_basis_tables": (_I, [_I, _I, _P, _P, _P, _P]),
    "pmg_schwarz_class": (_I, [_I, _I, _I, _I, _P, _P, ctypes.POINTER(_I)]),
    "pmg_node_coords": (_I, [_P, _P, _P]),
    "pmg_set_geometry": (_I, [_P, _P, _P]),
    "pmg_set_geometry_mixed": (_I, [_P, _P, _P, _P]),
    "pmg_set_bathymetry": (_I, [_P, _P, _P]),
    "pmg_assemble_rhs": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "pmg_assemble_rhs_div": (_I, [_P, _P, _P, _D, _P, _P]),
    "pmg_solve": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(SolveInfo), _P]),
    "pmg_solve_host": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(SolveInfo), _P]),
    "pmg_residual_norm": (_I, [_P, _P, _P, _P, ctypes.POINTER(_D), _P]),
    "pmg_apply": (_I, [_P, _P, _P, _P]),
    "pmg_apply_f32": (_I, [_P, _P, _P, _P]),
    "pmg_apply_bf16": (_I, [_P, _P, _P, _I, _P]),
    "pmg_level_apply": (_I, [_P, _I, _P, _P, _I, _P]),
    "pmg_level_smooth": (_I, [_P, _I, _P, _P, _I, _I, _P]),
    "pmg_level_sweep": (_I, [_P, _I, _P, _P, _I, _I, _P]),
    "pmg_restrict": (_I, [_P, _I, _P, _P, _I, _P]),
    "pmg_prolong": (_I, [_P, _I, _P, _P, _I, _P]),
    "pmg_coarse_solve": (_I, [_P, _P, _P, _P]),
    "pmg_vcycle": (_I, [_P, _P, _P, _I, _P]),
    "pmg_apply_noalloc": (_I, [ctypes.POINTER(MeshDesc), _P, _P, _P, _P]),
    "pmg_gradient": (_I, [_P, _P, _P, _P, _P]),
    "pmg_surface_slope": (_I, [_P, _P, _P]),
    "pmg_set_filter": (_I, [_P, _I, _D, _D]),
    "pmg_filter": (_I, [_P, _P, _P, _I, _P]),
    "pmg_forcing": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _D, _P, _P, _P]),
    "pmg_stage_rates": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _D, _P, _P, _P, _P]),
    "pmg_axpy": (_I, [_P, ctypes.c_int64, _D, _P, _P, _P, _P]),
    "pmg_batch_create": (_I, [_I, ctypes.POINTER(MeshDesc), ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "pmg_batch_destroy": (_I, [_P]),
    "pmg_batch_handle": (_I, [_P, _I, ctypes.POINTER(_P)]),
    "pmg_batch_solve": (_I, [_P, _P, _P, _P, ctypes.POINTER(SolveInfo), _P]),
    "pmg_batch_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "pmg_batch_set_path": (_I, [_P, _I]),
    "pmg_autotune": (_I, [_P]),
    "pmg_set_wait_limit": (_I, [_P, ctypes.c_int64]),
    "pmg_profile_reset": (_I, [_P, _I]),
    "pmg_profile_read": (_I, [_P, _P, _P, _P, _P]),
    "pmg_ws_create": (_I, [_I, _I, _I, _I, _I, _I, ctypes.c_uint64, _D, _D, _D, _D, ctypes.POINTER(_P)]),
    "pmg_ws_destroy": (_I, [_P]),
    "pmg_ws_num_params": (_I, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "pmg_ws_set_roughness": (_I, [_P, _D]),
    "pmg_ws_get_params": (_I, [_P, _P]),
    "pmg_ws_set_params": (_I, [_P, _P]),
    "pmg_ws_pack": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "pmg_ws_target": (_I, [_P, _P, _P, _P, _P]),
    "pmg_ws_forward": (_I, [_P, _P, _I, _P, _P]),
    "pmg_ws_predict": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "pmg_ws_gradients": (_I, [_P, _P, _P, _I, _P, ctypes.POINTER(_D), _P]),
    "pmg_ws_train_step": (_I, [_P, _P, _P, _I, ctypes.c_float, ctypes.POINTER(_D), _P]),
    "pmg_ws_save": (_I, [_P, ctypes.c_char_p]),
    "pmg_ws_load": (_I, [_P, ctypes.c_char_p]),
    "pmg_last_error": (ctypes.c_char_p, []),
}

_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load libpmg.so (raises if absent: the product path has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"native library {path} is missing: run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st):
    if st != PMG_OK:
        raise PmgError(st, _lib.pmg_last_error().decode())


def _ptr(t, dtype=torch.float64):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def default_opts(**kw):
    lib = load()
    o = Opts()
    lib.pmg_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "level_orders":
            o.nlevels = len(v)
            for i, p in enumerate(v):
                o.level_orders[i] = p
        else:
            setattr(o, k, v)
    return o


def apply_noalloc(mesh, eta, x, out):
    """pmg_apply_noalloc: the actual-geometry operator without a handle and without device
    allocation (static library scratch).  mesh: MeshDesc or dict of its fields."""
    if isinstance(mesh, dict):
        mesh = MeshDesc(mesh.get("x0", 0.0), mesh.get("x1", 1.0), mesh.get("h", 1.0), mesh["cells_x"],
                        mesh["cells_z"], mesh["order"], int(bool(mesh.get("periodic", False))))
    _check(load().pmg_apply_noalloc(ctypes.byref(mesh), _ptr(eta), _ptr(x), _ptr(out), _stream()))
    return out


def level_sequence(cells_x, cells_z, order, x0=0.0, x1=1.0, h=1.0, periodic=False, order_z=None, **opts):
    """pmg_level_sequence: the (order along x, order along sigma) of every level pmg_create
    would build for this mesh and these options, finest first (host-only, no GPU)."""
    mesh = MeshDesc(x0, x1, h, cells_x, cells_z, order, int(bool(periodic)), int(order_z or 0))
    o = default_opts(**opts)
    nl = ctypes.c_int()
    ox, oz = (ctypes.c_int * 16)(), (ctypes.c_int * 16)()
    _check(load().pmg_level_sequence(ctypes.byref(mesh), ctypes.byref(o), ctypes.byref(nl), ox, oz))
    return [(ox[i], oz[i]) for i in range(nl.value)]


def basis_tables(p, pc=0):
    """pmg_basis_tables: LGL nodes and weights of order p, the derivative matrix D
    ((p+1) x (p+1)) and, for pc >= 1, the order-pc -> order-p interpolation J ((p+1) x (pc+1)),
    as float64 CPU tensors (host-only, no GPU)."""
    n = p + 1
    x, w = torch.empty(n, dtype=torch.float64), torch.empty(n, dtype=torch.float64)
    D = torch.empty(n, n, dtype=torch.float64)
    J = torch.empty(n, max(pc, 0) + 1, dtype=torch.float64)
    _check(load().pmg_basis_tables(p, pc, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                   ctypes.c_void_p(D.data_ptr()),
                                   ctypes.c_void_p(J.data_ptr()) if pc >= 1 else None))
    return {"nodes": x, "weights": w, "D": D, "J": J if pc >= 1 else None}


def schwarz_class(p, overlap, direction, cls):
    """pmg_schwarz_class: (V, lam, k) of one Schwarz element class of a level of order p,
    direction 0 (x) or 1 (sigma), class 0 interior / 1 first / 2 last / 3 single element
    (host-only, no GPU)."""
    nb = p + 1 + 2 * overlap
    V = torch.zeros(nb, nb, dtype=torch.float64)
    lam = torch.zeros(nb, dtype=torch.float64)
    k = ctypes.c_int()
    _check(load().pmg_schwarz_class(p, overlap, direction, cls, ctypes.c_void_p(V.data_ptr()),
                                    ctypes.c_void_p(lam.data_ptr()), ctypes.byref(k)))
    return V, lam, k.value


class Solver:
    """One mesh + multigrid hierarchy on the current CUDA device (pmg_create)."""

    def __init__(self, cells_x, cells_z, order, x0=0.0, x1=1.0, h=1.0, periodic=False, order_z=None, **opts):
        lib = load()
        self.mesh = MeshDesc(x0, x1, h, cells_x, cells_z, order, int(bool(periodic)), int(order_z or 0))
        self.opts = default_opts(**opts)
        hh = ctypes.c_void_p()
        _check(lib.pmg_create(ctypes.byref(self.mesh), ctypes.byref(self.opts), ctypes.byref(hh)))
        self._h = hh
        n, nf = ctypes.c_int64(), ctypes.c_int64()
        nx, nz, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.pmg_num_nodes(self._h, ctypes.byref(n), ctypes.byref(nf), ctypes.byref(nx),
                                 ctypes.byref(nz), ctypes.byref(nl)))
        self.n, self.n_free, self.NX, self.NZ, self.nlevels = n.value, nf.value, nx.value, nz.value, nl.value

    def close(self):
        if getattr(self, "_h", None):
            load().pmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- sizes and coordinates
    def level_info(self, level):
        p, nx, nz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().pmg_level_info(self._h, level, ctypes.byref(p), ctypes.byref(nx), ctypes.byref(nz)))
        return p.value, nx.value, nz.value

    def level_kernels(self, level):
        """Launch configuration of level `level`'s FP32 kernels (after autotune, the tuned
        one): {"flat32": slab CTA size > 0, node-parallel CTA size < 0 or tiled shape
        code >= 10000, "fdm32": sweep CTA size, "xfer": transfer CTA size}."""
        f, d, x = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().pmg_level_kernels(self._h, level, ctypes.byref(f), ctypes.byref(d), ctypes.byref(x)))
        return {"flat32": f.value, "fdm32": d.value, "xfer": x.value}

    def fused_vcycle_info(self):
        """{"first_level", "on", "threads", "ctas_per_sm", "us_off", "us_on"} of the fused
        coarse V-cycle (first_level -1: the levels do not qualify)."""
        fl, on, thr, per = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        us = (ctypes.c_float * 2)()
        _check(load().pmg_fused_vcycle_info(self._h, ctypes.byref(fl), ctypes.byref(on), ctypes.byref(thr),
                                            ctypes.byref(per), ctypes.cast(us, ctypes.c_void_p)))
        return {"first_level": fl.value, "on": on.value, "threads": thr.value, "ctas_per_sm": per.value,
                "us_off": us[0], "us_on": us[1]}

    def set_fused_vcycle(self, on):
        _check(load().pmg_set_fused_vcycle(self._h, int(bool(on))))

    def node_coords(self):
        xc = torch.empty(self.NX, dtype=torch.float64)
        sr = torch.empty(self.NZ, dtype=torch.float64)
        _check(load().pmg_node_coords(self._h, ctypes.c_void_p(xc.data_ptr()), ctypes.c_void_p(sr.data_ptr())))
        return xc.numpy(), sr.numpy()

    # ---- per-stage inputs
    def set_geometry_mixed(self, eta, eta_prev):
        """Mixed-stage operator: test gradients on `eta` (stage k), trial gradients on
        `eta_prev` (stage k-1); solve with outer PMG_PDC or PMG_GMRES."""
        _check(load().pmg_set_geometry_mixed(self._h, _ptr(eta), _ptr(eta_prev), _stream()))

    def set_geometry(self, eta):
        _check(load().pmg_set_geometry(self._h, _ptr(eta), _stream()))

    def set_bathymetry(self, depth):
        """Varying still-water depth h(x) at the node columns (NX doubles on the device)."""
        _check(load().pmg_set_bathymetry(self._h, _ptr(depth), _stream()))

    def assemble_rhs(self, f, g_bottom=None, g_left=None, g_right=None, out=None):
        out = torch.empty(self.n, dtype=torch.float64, device=f.device) if out is None else out
        _check(load().pmg_assemble_rhs(self._h, _ptr(f), _ptr(g_bottom), _ptr(g_left), _ptr(g_right),
                                       _ptr(out), _stream()))
        return out

    def assemble_rhs_div(self, u, w, scale=1.0, out=None):
        out = torch.empty(self.n, dtype=torch.float64, device=u.device) if out is None else out
        _check(load().pmg_assemble_rhs_div(self._h, _ptr(u), _ptr(w), float(scale), _ptr(out), _stream()))
        return out

    # ---- solve
    def solve(self, b, p_dirichlet, x0=None, out=None, raise_on_error=True):
        out = torch.empty(self.n, dtype=torch.float64, device=b.device) if out is None else out
        info = SolveInfo()
        st = load().pmg_solve(self._h, _ptr(b), _ptr(p_dirichlet), _ptr(x0), _ptr(out), ctypes.byref(info),
                              _stream())
        if raise_on_error and st not in (PMG_OK,):
            _check(st)
        return out, info.as_dict()

    def solve_host(self, b, p_dirichlet, x0=None, out=None, raise_on_error=True):
        """Host (CPU float64) buffers in and out; copies are part of the call."""
        def hp(t):
            if t is None:
                return None
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError("expected contiguous CPU float64 tensors")
            return ctypes.c_void_p(t.data_ptr())
        out = torch.empty(self.n, dtype=torch.float64, pin_memory=True) if out is None else out
        info = SolveInfo()
        st = load().pmg_solve_host(self._h, hp(b), hp(p_dirichlet), hp(x0), hp(out), ctypes.byref(info),
                                   _stream())
        if raise_on_error and st != PMG_OK:
            _check(st)
        return out, info.as_dict()

    # ---- time-stepper support
    def residual_norm(self, b, p_dirichlet, x):
        """||b~ - A x~|| with the surface row of x replaced by p_dirichlet (synchronises)."""
        r = ctypes.c_double()
        _check(load().pmg_residual_norm(self._h, _ptr(b), _ptr(p_dirichlet), _ptr(x), ctypes.byref(r), _stream()))
        return r.value

    def gradient(self, f, fx=None, fz=None):
        fx = torch.empty_like(f) if fx is None else fx
        fz = torch.empty_like(f) if fz is None else fz
        _check(load().pmg_gradient(self._h, _ptr(f), _ptr(fx), _ptr(fz), _stream()))
        return fx, fz

    def set_filter(self, cutoff, alpha, beta):
        """Exponential cut-off filter of the element modes above `cutoff`."""
        _check(load().pmg_set_filter(self._h, int(cutoff), float(alpha), float(beta)))

    def filter(self, f, out=None, surface=False):
        out = torch.empty_like(f) if out is None else out
        _check(load().pmg_filter(self._h, _ptr(f), _ptr(out), int(bool(surface)), _stream()))
        return out

    def surface_slope(self, out=None):
        out = torch.empty(self.NX, dtype=torch.float64, device="cuda") if out is None else out
        _check(load().pmg_surface_slope(self._h, _ptr(out), _stream()))
        return out

    def forcing(self, u, w, ux, uz, wx, wz, etax, g, Fu, Fw):
        _check(load().pmg_forcing(self._h, _ptr(u), _ptr(w), _ptr(ux), _ptr(uz), _ptr(wx), _ptr(wz), _ptr(etax),
                                  float(g), _ptr(Fu), _ptr(Fw), _stream()))

    def stage_rates(self, u, w, uz, wz, Fu, Fw, px, pz, etax, rho, du, dw, deta):
        _check(load().pmg_stage_rates(self._h, _ptr(u), _ptr(w), _ptr(uz), _ptr(wz), _ptr(Fu), _ptr(Fw), _ptr(px),
                                      _ptr(pz), _ptr(etax), float(rho), _ptr(du), _ptr(dw), _ptr(deta), _stream()))

    def axpy(self, a, x, y, out):
        _check(load().pmg_axpy(self._h, x.numel(), float(a), _ptr(x), _ptr(y), _ptr(out), _stream()))
        return out

    def set_wait_limit(self, cycles):
        """pmg_set_wait_limit: bound (SM clock cycles) of the handle's device-side waits;
        negative restores the default, 0 gives up at once."""
        _check(load().pmg_set_wait_limit(self._h, int(cycles)))

    def autotune(self):
        """pmg_autotune: pick the CTA sizes of this handle's kernels by timing."""
        _check(load().pmg_autotune(self._h))

    # ---- profiling
    def profile_reset(self, timing=False):
        _check(load().pmg_profile_reset(self._h, int(bool(timing))))

    def profile_read(self, full=False):
        """{class: (launches, device ms)} since the last reset (synchronises); with
        full=True: {class: (launches, ms, algorithmic bytes, flops)}."""
        k = len(KERNEL_CLASSES)
        cnt = (ctypes.c_int64 * k)()
        ms, by, fl = (ctypes.c_double * k)(), (ctypes.c_double * k)(), (ctypes.c_double * k)()
        v = lambda a: ctypes.cast(a, ctypes.c_void_p)
        _check(load().pmg_profile_read(self._h, v(cnt), v(ms), v(by), v(fl)))
        if full:
            return {name: (cnt[i], ms[i], by[i], fl[i]) for i, name in enumerate(KERNEL_CLASSES)}
        return {name: (cnt[i], ms[i]) for i, name in enumerate(KERNEL_CLASSES)}

    # ---- components
    def apply(self, x, out=None):
        out = torch.empty_like(x) if out is None else out
        _check(load().pmg_apply(self._h, _ptr(x), _ptr(out), _stream()))
        return out

    def apply_f32(self, x, out=None):
        out = torch.empty_like(x) if out is None else out
        _check(load().pmg_apply_f32(self._h, _ptr(x, torch.float32), _ptr(out, torch.float32), _stream()))
        return out

    def apply_bf16(self, x, out=None, split=True):
        """A x on the BF16 tensor cores (FP32 vectors); split: hi/lo BF16 parts."""
        out = torch.empty_like(x) if out is None else out
        _check(load().pmg_apply_bf16(self._h, _ptr(x, torch.float32), _ptr(out, torch.float32), int(bool(split)),
                                     _stream()))
        return out

    @staticmethod
    def _f32(t):
        return 1 if t.dtype == torch.float32 else 0

    def level_apply(self, level, x, out=None):
        out = torch.empty_like(x) if out is None else out
        _check(load().pmg_level_apply(self._h, level, _ptr(x, x.dtype), _ptr(out, x.dtype), self._f32(x), _stream()))
        return out

    def level_sweep(self, level, r, x, post=False):
        """One Schwarz sweep x += B_l r (a single kernel launch)."""
        dt = r.dtype
        _check(load().pmg_level_sweep(self._h, level, _ptr(r, dt), _ptr(x, dt), int(post), self._f32(r), _stream()))
        return x

    def level_smooth(self, level, b, x, post=False):
        _check(load().pmg_level_smooth(self._h, level, _ptr(b, b.dtype), _ptr(x, b.dtype), int(post),
                                       self._f32(b), _stream()))
        return x

    def restrict(self, level, rf, out):
        _check(load().pmg_restrict(self._h, level, _ptr(rf, rf.dtype), _ptr(out, rf.dtype), self._f32(rf),
                                   _stream()))
        return out

    def prolong(self, level, xc, xf):
        _check(load().pmg_prolong(self._h, level, _ptr(xc, xc.dtype), _ptr(xf, xc.dtype), self._f32(xc),
                                  _stream()))
        return xf

    def coarse_solve(self, b, out=None):
        out = torch.empty_like(b) if out is None else out
        _check(load().pmg_coarse_solve(self._h, _ptr(b), _ptr(out), _stream()))
        return out

    def vcycle(self, r, out=None):
        out = torch.empty_like(r) if out is None else out
        _check(load().pmg_vcycle(self._h, _ptr(r, r.dtype), _ptr(out, r.dtype), self._f32(r), _stream()))
        return out


class _BatchMember(Solver):
    """A handle owned by a Batch (not destroyed on its own)."""

    def __init__(self, handle, mesh, opts):
        lib = load()
        self._h = handle
        self.mesh, self.opts = mesh, opts
        n, nf = ctypes.c_int64(), ctypes.c_int64()
        nx, nz, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.pmg_num_nodes(self._h, ctypes.byref(n), ctypes.byref(nf), ctypes.byref(nx), ctypes.byref(nz),
                                 ctypes.byref(nl)))
        self.n, self.n_free, self.NX, self.NZ, self.nlevels = n.value, nf.value, nx.value, nz.value, nl.value

    def close(self):
        self._h = None


class Batch:
    """pmg_batch_*: independent problems solved together (one handle each): one graph of
    batched launches over all problems, or concurrent per-problem loops (see info())."""

    def __init__(self, meshes, **opts):
        lib = load()
        self.opts = default_opts(**opts)
        arr = (MeshDesc * len(meshes))()
        for i, m in enumerate(meshes):
            arr[i] = MeshDesc(m.get("x0", 0.0), m.get("x1", 1.0), m.get("h", 1.0), m["cells_x"], m["cells_z"],
                              m["order"], int(bool(m.get("periodic", False))), int(m.get("order_z") or 0))
        hb = ctypes.c_void_p()
        _check(lib.pmg_batch_create(len(meshes), arr, ctypes.byref(self.opts), ctypes.byref(hb)))
        self._b = hb
        self.members = []
        for i in range(len(meshes)):
            hh = ctypes.c_void_p()
            _check(lib.pmg_batch_handle(self._b, i, ctypes.byref(hh)))
            self.members.append(_BatchMember(hh, arr[i], self.opts))

    def close(self):
        if getattr(self, "_b", None):
            load().pmg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, bs, pds, outs=None, raise_on_error=True):
        n = len(self.members)
        outs = [torch.empty_like(b) for b in bs] if outs is None else outs
        vp = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
        for t in list(bs) + list(pds) + list(outs):
            _ptr(t)
        infos = (SolveInfo * n)()
        st = load().pmg_batch_solve(self._b, ctypes.cast(vp(bs), ctypes.c_void_p), ctypes.cast(vp(pds), ctypes.c_void_p),
                                    ctypes.cast(vp(outs), ctypes.c_void_p), infos, _stream())
        if raise_on_error and st != PMG_OK:
            _check(st)
        return outs, [infos[i].as_dict() for i in range(n)]

    def set_path(self, path):
        """pmg_batch_set_path: 0 one graph of batched launches, 1 the same launches from a
        host loop (profiling), 2 concurrent per-problem loops."""
        _check(load().pmg_batch_set_path(self._b, int(path)))

    def info(self):
        """pmg_batch_info: {"batched": 1 for the single graph of batched launches, 0 for
        concurrent per-problem loops; "launches": kernel launches per batched iteration}."""
        b, l = ctypes.c_int(), ctypes.c_int()
        _check(load().pmg_batch_info(self._b, ctypes.byref(b), ctypes.byref(l)))
        return {"batched": b.value, "launches": l.value}
