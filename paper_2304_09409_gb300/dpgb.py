"""Thin Python binding of libdpgb (include/dpgb.h): argument marshalling only.

Every step of the energy / force / virial path runs in the library's CUDA kernels.
Arrays may be numpy arrays (host; the library copies them) or torch CUDA tensors
(device; the library reads and writes them in place).  There is no CPU fallback:
loading fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdpgb.so")

DP_OK = 0
DP_E_ARG = 1
DP_E_CUDA = 2
DP_E_OOM = 3
DP_E_SEL_OVERFLOW = 4
DP_E_TIMEOUT = 5
DP_E_RANGE = 6
DP_E_CAPACITY = 7
DP_E_UNSUPPORTED = 8

PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}

EXPORTED = [
    "dp_model_create", "dp_init_model", "dp_free_model", "dp_model_n_params", "dp_build_nlist",
    "dp_nlist_export", "dp_free_nlist", "dp_compute", "dp_model_export_table", "dp_last_error",
    "dp_build_nlist_noalloc", "dp_compute_batch", "dp_param_grad", "dp_model_set_params", "dp_wait_selftest",
    "dp_profile_work", "dp_model_deviation",
]


class DPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dpgb error {code}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    """dp_model_config of include/dpgb.h."""
    _fields_ = [
        ("ntypes", ctypes.c_int),
        ("sel", ctypes.c_int * 8),
        ("rcut", ctypes.c_double),
        ("rcut_smth", ctypes.c_double),
        ("n_embed", ctypes.c_int),
        ("embed", ctypes.c_int * 8),
        ("axis", ctypes.c_int),
        ("n_fit", ctypes.c_int),
        ("fit", ctypes.c_int * 8),
        ("type_one_side", ctypes.c_int),
        ("descriptor", ctypes.c_int),
        ("rcut_2", ctypes.c_double),
        ("rcut_smth_2", ctypes.c_double),
        ("sel_2", ctypes.c_int * 8),
        ("n_embed_2", ctypes.c_int),
        ("embed_2", ctypes.c_int * 8),
    ]

    @classmethod
    def from_model(cls, cfg) -> "Config":
        c = cls()
        c.ntypes = int(cfg.ntypes)
        for t, v in enumerate(cfg.sel):
            c.sel[t] = int(v)
        c.rcut = float(cfg.rcut)
        c.rcut_smth = float(cfg.rcut_smth)
        c.n_embed = len(cfg.embed)
        for k, v in enumerate(cfg.embed):
            c.embed[k] = int(v)
        c.axis = int(cfg.axis)
        c.n_fit = len(cfg.fit)
        for k, v in enumerate(cfg.fit):
            c.fit[k] = int(v)
        c.type_one_side = int(getattr(cfg, "type_one_side", 0))
        c.descriptor = int(getattr(cfg, "descriptor", 0))
        if c.descriptor in (2, 4):  # hybrid: the second part (defaults: the first part's list)
            c.rcut_2 = float(getattr(cfg, "rcut_2", 0.0) or cfg.rcut)
            c.rcut_smth_2 = float(getattr(cfg, "rcut_smth_2", 0.0) or cfg.rcut_smth)
            for t, v in enumerate(tuple(getattr(cfg, "sel_2", ()) or cfg.sel)):
                c.sel_2[t] = int(v)
            embed_2 = tuple(getattr(cfg, "embed_2", ()))
            c.n_embed_2 = len(embed_2)
            for k, v in enumerate(embed_2):
                c.embed_2[k] = int(v)
        return c


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdpgb is not built ({LIB_PATH} missing): run paper_2304_09409_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        ip = ctypes.c_int
        L.dp_model_create.argtypes = [ctypes.POINTER(Config), vp, ctypes.c_long, ip, ip, ip, ctypes.POINTER(vp)]
        L.dp_init_model.argtypes = [ctypes.c_char_p, ip, ip, ip, ctypes.POINTER(vp)]
        L.dp_free_model.argtypes = [vp]
        L.dp_model_n_params.argtypes = [ctypes.POINTER(Config)]
        L.dp_model_n_params.restype = ctypes.c_long
        L.dp_build_nlist.argtypes = [vp, ip, vp, vp, vp, ctypes.POINTER(vp), ctypes.POINTER(ip), vp]
        L.dp_nlist_export.argtypes = [vp, vp, vp]
        L.dp_free_nlist.argtypes = [vp]
        L.dp_compute.argtypes = [vp, vp, ip, vp, vp, vp, vp, vp, vp, vp, vp]
        L.dp_model_export_table.argtypes = [vp, vp, ctypes.POINTER(ip)]
        L.dp_last_error.argtypes = [ctypes.c_char_p, ip]
        L.dp_last_error.restype = ip
        L.dp_wait_selftest.argtypes = [ctypes.c_long, vp]
        L.dp_profile_enable.argtypes = [vp, ip]
        L.dp_profile_reset.argtypes = [vp]
        L.dp_profile_count.argtypes = [vp]
        L.dp_profile_read.argtypes = [vp, ip, ctypes.c_char_p, ip, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_long)]
        L.dp_launch_count.argtypes = [vp]
        L.dp_launch_count.restype = ctypes.c_long
        _lib = L
    return _lib


def last_error() -> str:
    L = lib()
    n = L.dp_last_error(None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    L.dp_last_error(buf, n + 1)
    return buf.value.decode(errors="replace")


def wait_selftest(spin_limit: int = 0, stream=None) -> int:
    """dp_wait_selftest: a bounded mbarrier wait that nothing releases; DP_E_TIMEOUT expected."""
    return int(lib().dp_wait_selftest(int(spin_limit), _stream_handle(stream)))


def _check(code: int, allow=()):
    if code != DP_OK and code not in allow:
        raise DPError(code, last_error())
    return code


def _ptr(x):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


class NList:
    def __init__(self, handle, natoms: int, nc: int, n_overflow: int):
        self.handle = handle
        self.natoms = natoms
        self.nc = nc
        self.n_overflow = n_overflow

    def export(self):
        nl_j = np.zeros((self.natoms, self.nc), dtype=np.int32)
        nl_s = np.zeros((self.natoms, self.nc, 3), dtype=np.int32)
        _check(lib().dp_nlist_export(self.handle, nl_j.ctypes.data, nl_s.ctypes.data))
        return nl_j, nl_s

    def free(self):
        if self.handle:
            lib().dp_free_nlist(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Model:
    """A Deep Potential model (se_e2_a, se_e2_r, se_e3 or hybrid descriptor) resident on one GPU."""

    def __init__(self, cfg, params: np.ndarray, device: int = 0, precision: str = "fp64", compressed: bool = False):
        self.cfg = cfg
        self.c = Config.from_model(cfg)
        p = np.ascontiguousarray(params, dtype=np.float64)
        h = ctypes.c_void_p()
        _check(lib().dp_model_create(ctypes.byref(self.c), p.ctypes.data, p.size, device, PREC[precision],
                                     1 if compressed else 0, ctypes.byref(h)))
        self.handle = h
        self.device = device
        self.nc = int(cfg.nc)

    @classmethod
    def from_file(cls, path: str, cfg, device: int = 0, precision: str = "fp64", compressed: bool = False):
        """A model created by dp_init_model from a weight file (see write_weight_file); cfg is
        the configuration the file holds (kept on the Python side for array shapes)."""
        self = cls.__new__(cls)
        self.cfg = cfg
        self.c = Config.from_model(cfg)
        self.handle = load_model_file(path, device, precision, compressed)
        self.device = device
        self.nc = int(cfg.nc)
        return self

    def free(self):
        if getattr(self, "handle", None):
            lib().dp_free_model(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # ---- tracing ----
    def profile(self, on: bool = True):
        _check(lib().dp_profile_enable(self.handle, 1 if on else 0))

    def profile_reset(self):
        _check(lib().dp_profile_reset(self.handle))

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} accumulated while profiling was on."""
        out = {}
        buf = ctypes.create_string_buffer(64)
        for k in range(lib().dp_profile_count(self.handle)):
            ms = ctypes.c_double()
            n = ctypes.c_long()
            _check(lib().dp_profile_read(self.handle, k, buf, 64, ctypes.byref(ms), ctypes.byref(n)))
            out[buf.value.decode()] = (ms.value, n.value)
        return out

    def profile_work(self) -> dict:
        """{kernel name: tensor-core FLOPs issued} for the scopes that count their issued work."""
        L = lib()
        L.dp_profile_work.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        out = {}
        buf = ctypes.create_string_buffer(64)
        for k in range(L.dp_profile_count(self.handle)):
            w = ctypes.c_double()
            _check(L.dp_profile_read(self.handle, k, buf, 64, None, None))
            _check(L.dp_profile_work(self.handle, k, ctypes.byref(w)))
            if w.value > 0:
                out[buf.value.decode()] = w.value
        return out

    def launch_count(self) -> int:
        return int(lib().dp_launch_count(self.handle))

    def set_params(self, params, stream=None):
        """dp_model_set_params: replace the parameters (numpy or torch CUDA FP64, n_params)."""
        L = lib()
        L.dp_model_set_params.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p]
        if not (_is_torch(params) and params.is_cuda):
            params = np.ascontiguousarray(params, dtype=np.float64)
        else:
            params = params.detach().contiguous()
        n = int(params.numel() if _is_torch(params) else params.size)
        _check(L.dp_model_set_params(self.handle, _ptr(params), n, _stream_handle(stream)))

    def build_nlist(self, coord, atype, box, stream=None) -> NList:
        N = int(coord.shape[0])
        h = ctypes.c_void_p()
        ov = ctypes.c_int(0)
        boxp = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
        _check(lib().dp_build_nlist(self.handle, N, _ptr(coord), _ptr(atype), _ptr(boxp), ctypes.byref(h),
                                    ctypes.byref(ov), _stream_handle(stream)), allow=(DP_E_SEL_OVERFLOW,))
        return NList(h, N, self.nc, ov.value)

    def export_table(self) -> np.ndarray:
        nets = int(self.cfg.n_embed_nets)
        M = int(self.cfg.embed[-1])
        lc = ctypes.c_int(0)
        smax = 1.0 / float(self.cfg.rcut_smth)
        n1 = int(np.floor(0.9 * smax / 0.01 + 0.5))
        n2 = max(1, int(np.ceil((smax - n1 * 0.01) / 0.1 - 1e-9)))
        out = np.zeros(nets * (n1 + n2) * M * 6)
        _check(lib().dp_model_export_table(self.handle, out.ctypes.data, ctypes.byref(lc)))
        return out[: nets * lc.value * M * 6].reshape(nets, lc.value, M, 6)

    def compute(self, coord, atype, box, nlist: Optional[NList] = None, atom_energy: bool = False, stream=None,
                out=None, allow=(DP_E_SEL_OVERFLOW,)):
        """Energy, forces [N,3] and virial [3,3] (and per-atom energies).

        Host (numpy) inputs give numpy outputs; torch CUDA inputs give torch CUDA outputs
        written in place by the kernels (pass `out=(e, f, v, ae)` to reuse buffers)."""
        N = int(coord.shape[0])
        boxp = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
        if _is_torch(coord) and coord.is_cuda:
            import torch
            if out is None:
                e = torch.empty(1, dtype=torch.float64, device=coord.device)
                f = torch.empty((N, 3), dtype=torch.float64, device=coord.device)
                v = torch.empty((3, 3), dtype=torch.float64, device=coord.device)
                ae = torch.empty(N, dtype=torch.float64, device=coord.device) if atom_energy else None
            else:
                e, f, v, ae = out
        else:
            coord = np.ascontiguousarray(coord, dtype=np.float64)
            atype = np.ascontiguousarray(atype, dtype=np.int32)
            if out is None:
                e = np.zeros(1)
                f = np.zeros((N, 3))
                v = np.zeros((3, 3))
                ae = np.zeros(N) if atom_energy else None
            else:
                e, f, v, ae = out
        code = lib().dp_compute(self.handle, nlist.handle if nlist is not None else None, N, _ptr(coord), _ptr(atype),
                                _ptr(boxp), _ptr(e), _ptr(f), _ptr(v), _ptr(ae), _stream_handle(stream))
        _check(code, allow=allow)
        self.last_status = code
        return e, f, v, ae


def _batch_argtypes():
    L = lib()
    vp = ctypes.c_void_p
    L.dp_compute_batch.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    return L


def compute_batch(model, natoms, coord, atype, boxes, atom_energy: bool = False, stream=None, out=None,
                  allow=(DP_E_SEL_OVERFLOW,), frame_model=None):
    """dp_compute_batch: several frames, of one model or of several, in one call.

    model: a Model, or a list of Models with frame_model [F] (the index of each frame's model);
    natoms: int32 array [F]; coord [sum(natoms), 3], atype [sum(natoms)] (numpy or torch CUDA);
    boxes [F, 3, 3] numpy.  Returns (energy [F], force [sum, 3], virial [F, 3, 3], atom_energy)."""
    L = _batch_argtypes()
    models = list(model) if isinstance(model, (list, tuple)) else [model]
    handles = (ctypes.c_void_p * len(models))(*[m.handle for m in models])
    nat = np.ascontiguousarray(natoms, dtype=np.int32)
    F = int(nat.size)
    N = int(nat.sum())
    fm = None if frame_model is None else np.ascontiguousarray(frame_model, dtype=np.int32)
    if len(models) > 1 and fm is None:
        raise ValueError("several models need frame_model")
    bx = np.ascontiguousarray(boxes, dtype=np.float64).reshape(F, 9)
    if _is_torch(coord) and coord.is_cuda:
        import torch
        if out is None:
            e = torch.empty(F, dtype=torch.float64, device=coord.device)
            f = torch.empty((N, 3), dtype=torch.float64, device=coord.device)
            v = torch.empty((F, 3, 3), dtype=torch.float64, device=coord.device)
            ae = torch.empty(N, dtype=torch.float64, device=coord.device) if atom_energy else None
        else:
            e, f, v, ae = out
    else:
        coord = np.ascontiguousarray(coord, dtype=np.float64)
        atype = np.ascontiguousarray(atype, dtype=np.int32)
        if out is None:
            e, f, v = np.zeros(F), np.zeros((N, 3)), np.zeros((F, 3, 3))
            ae = np.zeros(N) if atom_energy else None
        else:
            e, f, v, ae = out
    code = L.dp_compute_batch(handles, len(models), F, nat.ctypes.data, None if fm is None else fm.ctypes.data,
                              _ptr(coord), _ptr(atype), bx.ctypes.data, _ptr(e), _ptr(f), _ptr(v), _ptr(ae),
                              _stream_handle(stream))
    _check(code, allow=allow)
    return e, f, v, ae


def model_deviation(models, coord, atype, box, nu: float = 0.0, stream=None):
    """dp_model_deviation: (devi_f [N], devi_v [3, 3], stats [6], force_mean [N, 3]) of an ensemble on
    one frame; stats = (eps_F max, mean, min, eps_Xi max, mean, min).  Arrays come back as
    torch CUDA tensors when coord is one, else numpy."""
    L = lib()
    vp = ctypes.c_void_p
    L.dp_model_deviation.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.c_double, vp, vp, vp, vp, vp]
    handles = (ctypes.c_void_p * len(models))(*[m.handle for m in models])
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64).reshape(9)
    if _is_torch(coord) and coord.is_cuda:
        import torch
        N = int(coord.shape[0])
        mk = lambda *s: torch.empty(s, dtype=torch.float64, device=coord.device)  # noqa: E731
        df, dv, st, fm = mk(N), mk(3, 3), mk(6), mk(N, 3)
    else:
        coord = np.ascontiguousarray(coord, dtype=np.float64)
        atype = np.ascontiguousarray(atype, dtype=np.int32)
        N = int(coord.shape[0])
        df, dv, st, fm = np.zeros(N), np.zeros((3, 3)), np.zeros(6), np.zeros((N, 3))
    _check(L.dp_model_deviation(handles, len(models), N, _ptr(coord), _ptr(atype), None if bx is None else bx.ctypes.data,
                                float(nu), _ptr(df), _ptr(dv), _ptr(st), _ptr(fm), _stream_handle(stream)),
           allow=(DP_E_SEL_OVERFLOW,))
    return df, dv, st, fm


def param_grad(model: "Model", natoms, coord, atype, boxes, g_energy, g_force, stream=None, out=None,
               g_virial=None):
    """dp_param_grad: d/dtheta [sum_f g_energy[f] E_f + sum_i g_force[i] . F_i + sum_f g_virial[f] : Xi_f]
    for the model's current parameters.  natoms int32 [F]; coord [N, 3] and atype [N] (numpy or
    torch CUDA); boxes [F, 3, 3] numpy, or None for one open-boundary frame; g_energy [F],
    g_force [N, 3], g_virial [F, 3, 3] or None.  Returns [n_params] FP64 (a torch CUDA tensor
    when coord is one, else numpy)."""
    L = lib()
    vp = ctypes.c_void_p
    L.dp_param_grad.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    nat = np.ascontiguousarray(natoms, dtype=np.int32)
    F = int(nat.size)
    bx = None if boxes is None else np.ascontiguousarray(boxes, dtype=np.float64).reshape(F, 9)
    npar = n_params(model.cfg)
    if _is_torch(coord) and coord.is_cuda:
        import torch
        g_energy = torch.as_tensor(g_energy, dtype=torch.float64, device=coord.device).contiguous()
        g_force = torch.as_tensor(g_force, dtype=torch.float64, device=coord.device).contiguous()
        if g_virial is not None:
            g_virial = torch.as_tensor(g_virial, dtype=torch.float64, device=coord.device).reshape(F, 9).contiguous()
        grad = out if out is not None else torch.empty(npar, dtype=torch.float64, device=coord.device)
    else:
        coord = np.ascontiguousarray(coord, dtype=np.float64)
        atype = np.ascontiguousarray(atype, dtype=np.int32)
        g_energy = np.ascontiguousarray(g_energy, dtype=np.float64)
        g_force = np.ascontiguousarray(g_force, dtype=np.float64)
        if g_virial is not None:
            g_virial = np.ascontiguousarray(g_virial, dtype=np.float64).reshape(F, 9)
        grad = out if out is not None else np.zeros(npar)
    _check(L.dp_param_grad(model.handle, F, nat.ctypes.data, _ptr(coord), _ptr(atype), _ptr(bx), _ptr(g_energy),
                           _ptr(g_force), _ptr(g_virial), _ptr(grad), _stream_handle(stream)))
    return grad


def n_params(cfg) -> int:
    c = Config.from_model(cfg)
    return int(lib().dp_model_n_params(ctypes.byref(c)))


def write_weight_file(path: str, cfg, params: np.ndarray) -> None:
    """Weight file read by dp_init_model: magic, dp_model_config, int64 n, n FP64."""
    c = Config.from_model(cfg)
    p = np.ascontiguousarray(params, dtype=np.float64)
    with open(path, "wb") as fh:
        fh.write(b"DPGBW002")
        fh.write(bytes(c))
        fh.write(np.int64(p.size).tobytes())
        fh.write(p.tobytes())


def load_model_file(path: str, device: int = 0, precision: str = "fp64", compressed: bool = False):
    h = ctypes.c_void_p()
    _check(lib().dp_init_model(path.encode(), device, PREC[precision], 1 if compressed else 0, ctypes.byref(h)))
    return h


def build_nlist_noalloc(cfg, coord, atype, box, nl_j=None, nl_shift=None, stream=None):
    """dp_build_nlist_noalloc: neighbour list of a frame whose coordinates and types are
    torch CUDA tensors, written into caller-owned device buffers (allocated here with torch
    when not given).  The library call itself allocates nothing."""
    import torch
    c = Config.from_model(cfg)
    N = int(coord.shape[0])
    nc = int(cfg.nc)
    if nl_j is None:
        nl_j = torch.empty((N, nc), dtype=torch.int32, device=coord.device)
    if nl_shift is None:
        nl_shift = torch.empty((N, nc, 3), dtype=torch.int32, device=coord.device)
    boxp = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    ov = ctypes.c_int(0)
    L = lib()
    L.dp_build_nlist_noalloc.argtypes = [ctypes.POINTER(Config), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                         ctypes.c_void_p]
    _check(L.dp_build_nlist_noalloc(ctypes.byref(c), N, _ptr(coord), _ptr(atype), _ptr(boxp), _ptr(nl_j),
                                    _ptr(nl_shift), ctypes.byref(ov), _stream_handle(stream)),
           allow=(DP_E_SEL_OVERFLOW,))
    return nl_j, nl_shift, ov.value
