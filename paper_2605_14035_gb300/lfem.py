"""Python binding of liblfem.so (ctypes; argument marshalling only).

Every computation runs in the CUDA library; torch supplies device memory and
streams.  If the library cannot be loaded the import of this module raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblfem.so")

MASS, STIFF, CMASS = 1, 2, 4
FP64, MIXED = 0, 1
STATUS = {0: "LFEM_OK", 1: "LFEM_E_ARG", 2: "LFEM_E_INDEX", 3: "LFEM_E_UNSUPPORTED", 4: "LFEM_E_TOO_LARGE",
          5: "LFEM_E_NOMEM", 6: "LFEM_E_CUDA", 7: "LFEM_E_DEGENERATE", 8: "LFEM_E_TIMEOUT"}

# Every entry point declared in include/lfem.h.
EXPORTS = (
    "lfem_pattern", "lfem_pattern_csr", "lfem_pattern_copy_csr", "lfem_pattern_info", "lfem_pattern_retile",
    "lfem_pattern_destroy", "lfem_assemble", "lfem_set_launch", "lfem_set_mixed_kappa", "lfem_assemble_load",
    "lfem_assemble_mcf_nonlinear", "lfem_mcf_step", "lfem_lift_order", "lfem_assemble_adjoint", "lfem_assemble_adjoint_mixed",
    "lfem_eval_points",
    "lfem_geometry", "lfem_local", "lfem_sync_status", "lfem_mixed_fallback_count", "lfem_last_error",
    "lfem_status_string", "lfem_pattern_csr_noalloc", "lfem_debug_starve_wait", "lfem_debug_alloc_count", "lfem_debug_wide_entries", "lfem_autotune",
    "lfem_batch_create", "lfem_batch_assemble", "lfem_batch_graph_launch", "lfem_batch_sync_status",
    "lfem_batch_info", "lfem_batch_destroy", "lfem_batch_autotune",
)


class LfemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Quad(ctypes.Structure):
    _fields_ = [("n_pts", ctypes.c_int), ("xi", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("pattern", ctypes.c_void_p), ("coords", ctypes.c_void_p), ("ambient", ctypes.c_int),
                ("quad", ctypes.c_void_p), ("coef", ctypes.c_void_p), ("M", ctypes.c_void_p),
                ("A", ctypes.c_void_p), ("MC", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built; run __graft_entry__.build() (the CUDA library is required)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, L, U = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint
    sig = {
        "lfem_pattern": [P, L, ctypes.c_int32, I, I, P, P],
        "lfem_pattern_csr": [P, P, P, P, P],
        "lfem_pattern_copy_csr": [P, P, P, P],
        "lfem_pattern_info": [P, P, P, P, P],
        "lfem_pattern_retile": [P, ctypes.c_int32, P],
        "lfem_assemble": [P, P, I, P, P, I, U, I, P, P, P, P],
        "lfem_set_launch": [P, ctypes.c_int32, ctypes.c_int32],
        "lfem_set_mixed_kappa": [P, ctypes.c_double],
        "lfem_assemble_load": [P, P, I, P, P, P, P],
        "lfem_assemble_mcf_nonlinear": [P, P, P, P, P, P],
        "lfem_mcf_step": [P, P, I, P, ctypes.c_double, ctypes.c_double, I, P, P, P],
        "lfem_lift_order": [P, P, I, I, P, P, P, P],
        "lfem_assemble_adjoint": [P, P, I, P, P, P, P, P, P, P, P],
        "lfem_assemble_adjoint_mixed": [P, P, I, P, P, P, P, P, P, P, P],
        "lfem_eval_points": [P, L, I, I, P, I, P, P, P],
        "lfem_geometry": [P, L, I, I, P, I, P, P, P, P, P],
        "lfem_local": [P, L, I, I, P, I, P, P, P, P, P, P],
        "lfem_sync_status": [P, P],
        "lfem_mixed_fallback_count": [P, P, P],
        "lfem_pattern_csr_noalloc": [P, L, ctypes.c_int32, I, I, P, P, L, P, P],
        "lfem_debug_starve_wait": [P, I],
        "lfem_debug_wide_entries": [P, I, P],
        "lfem_autotune": [P, P, I, P, P, I, U, I, P, P, P, ctypes.c_char_p, P, P],
        "lfem_batch_create": [P, I, U, I, P, P],
        "lfem_batch_assemble": [P, P],
        "lfem_batch_graph_launch": [P, P],
        "lfem_batch_sync_status": [P, P],
        "lfem_batch_info": [P, P, P, P],
        "lfem_batch_autotune": [P, I, U, I, ctypes.c_char_p, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.lfem_pattern_destroy.argtypes = [P]
    lib.lfem_pattern_destroy.restype = None
    lib.lfem_batch_destroy.argtypes = [P]
    lib.lfem_batch_destroy.restype = None
    lib.lfem_last_error.restype = ctypes.c_char_p
    lib.lfem_status_string.restype = ctypes.c_char_p
    lib.lfem_status_string.argtypes = [I]
    lib.lfem_debug_alloc_count.argtypes = []
    lib.lfem_debug_alloc_count.restype = ctypes.c_longlong
    return lib


_lib = _load()


def lib():
    return _lib


def _check(code):
    if code != 0:
        raise LfemError(code, _lib.lfem_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class QuadRule:
    """Host copy of a rule in the layout the C ABI takes (keeps the arrays alive)."""

    xi: np.ndarray
    w: np.ndarray

    def __post_init__(self):
        self.xi = np.ascontiguousarray(self.xi, dtype=np.float64)
        self.w = np.ascontiguousarray(self.w, dtype=np.float64)
        self._c = _Quad(int(self.w.shape[0]), self.xi.ctypes.data, self.w.ctypes.data)

    @property
    def n_pts(self):
        return int(self.w.shape[0])

    @property
    def ref(self):
        return ctypes.byref(self._c)


class _ExactP1:
    """No rule: order-1 elements get their exact reference matrices (NULL rule in the C ABI)."""

    ref = None
    n_pts = 0
    _c = None


EXACT_P1 = _ExactP1()


def as_rule(rule) -> QuadRule:
    if rule is None or isinstance(rule, _ExactP1):
        return EXACT_P1
    if isinstance(rule, QuadRule):
        return rule
    return QuadRule(np.asarray(rule.xi), np.asarray(rule.w))


def _dev_i32(t):
    if not (t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()):
        raise TypeError("conn must be a contiguous int32 CUDA tensor")
    return t


def _dev_f64(t, name):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return t


class Pattern:
    """CSR pattern + assembly maps of one topology (lfem_pattern)."""

    def __init__(self, conn: torch.Tensor, n_nodes: int, dim: int, order: int, stream=None):
        conn = _dev_i32(conn)
        self.dim, self.order, self.n_nodes = int(dim), int(order), int(n_nodes)
        self.n_elem = int(conn.shape[0])
        self.ref = int(conn.shape[1]) if conn.dim() == 2 else 0
        h = ctypes.c_void_p()
        _check(_lib.lfem_pattern(_ptr(conn), self.n_elem, self.n_nodes, self.dim, self.order, _stream(stream),
                                 ctypes.byref(h)))
        self._h = h
        nr, nnz = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.lfem_pattern_csr(self._h, ctypes.byref(nr), ctypes.byref(nnz), None, None))
        self.nnz = int(nnz.value)

    @property
    def handle(self):
        return self._h

    def csr(self, stream=None):
        dev = torch.cuda.current_device()
        rp = torch.empty(self.n_nodes + 1, dtype=torch.int64, device=dev)
        ci = torch.empty(max(self.nnz, 1), dtype=torch.int32, device=dev)
        _check(_lib.lfem_pattern_copy_csr(self._h, _ptr(rp), _ptr(ci), _stream(stream)))
        return rp, ci[: self.nnz]

    def info(self):
        nt, rc, mr, ts = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.lfem_pattern_info(self._h, ctypes.byref(nt), ctypes.byref(rc), ctypes.byref(mr),
                                      ctypes.byref(ts)))
        return {"tiles": nt.value, "recompute": rc.value / 1000.0, "max_row": mr.value, "tile_slots": ts.value}

    def retile(self, tile_slots: int, stream=None):
        _check(_lib.lfem_pattern_retile(self._h, int(tile_slots), _stream(stream)))

    def set_launch(self, elems_per_chunk: int = 0, threads: int = 0):
        _check(_lib.lfem_set_launch(self._h, int(elems_per_chunk), int(threads)))

    def set_mixed_kappa(self, kappa_max: float):
        """LFEM_MIXED redoes in double the elements whose metric may have cond(G) > kappa_max."""
        _check(_lib.lfem_set_mixed_kappa(self._h, float(kappa_max)))

    def debug_wide_entries(self, wide: bool, stream=None):
        """Test knob: 32-bit slot entries in the tile blocks (rebuilds the tiles)."""
        _check(_lib.lfem_debug_wide_entries(self._h, int(bool(wide)), _stream(stream)))

    def debug_starve_wait(self, starve: bool):
        _check(_lib.lfem_debug_starve_wait(self._h, int(bool(starve))))

    def sync_status(self, stream=None):
        _check(_lib.lfem_sync_status(self._h, _stream(stream)))

    def fallback_count(self, stream=None) -> int:
        n = ctypes.c_int64()
        _check(_lib.lfem_mixed_fallback_count(self._h, _stream(stream), ctypes.byref(n)))
        return int(n.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.lfem_pattern_destroy(h)
            self._h = ctypes.c_void_p()


def assemble(pat: Pattern, coords: torch.Tensor, rule, coef: Optional[torch.Tensor] = None,
             which: int = MASS | STIFF, precision: int = FP64, out=None, stream=None):
    """lfem_assemble: returns a dict {'M', 'A', 'MC'} of CSR value tensors."""
    coords = _dev_f64(coords, "coords")
    rule = as_rule(rule)
    dt = torch.float64 if precision == FP64 else torch.float32
    out = dict(out or {})
    for key, bit in (("M", MASS), ("A", STIFF), ("MC", CMASS)):
        if which & bit and key not in out:
            out[key] = torch.empty(max(pat.nnz, 1), dtype=dt, device=coords.device)
    coef_f32 = 0
    if coef is not None:
        if not (coef.is_cuda and coef.is_contiguous() and coef.dtype in (torch.float32, torch.float64)):
            raise TypeError("coef must be a contiguous float32/float64 CUDA tensor")
        coef_f32 = int(coef.dtype == torch.float32)
    _check(_lib.lfem_assemble(pat.handle, _ptr(coords), int(coords.shape[1]), rule.ref, _ptr(coef), coef_f32,
                              int(which), int(precision), _ptr(out.get("M")), _ptr(out.get("A")),
                              _ptr(out.get("MC")), _stream(stream)))
    return {k: v[: pat.nnz] for k, v in out.items()}


def autotune(pat: Pattern, coords: torch.Tensor, rule, coef=None, which: int = MASS | STIFF,
             precision: int = FP64, cache_path: Optional[str] = None, stream=None) -> int:
    """lfem_autotune: pick and apply the fastest tile capacity; returns it."""
    coords = _dev_f64(coords, "coords")
    rule = as_rule(rule)
    dt = torch.float64 if precision == FP64 else torch.float32
    bufs = {k: (torch.empty(max(pat.nnz, 1), dtype=dt, device=coords.device) if which & bit else None)
            for k, bit in (("M", MASS), ("A", STIFF), ("MC", CMASS))}
    best = ctypes.c_int32()
    coef_f32 = int(coef is not None and coef.dtype == torch.float32)
    _check(_lib.lfem_autotune(pat.handle, _ptr(coords), int(coords.shape[1]), rule.ref, _ptr(coef), coef_f32,
                              int(which), int(precision), _ptr(bufs["M"]), _ptr(bufs["A"]), _ptr(bufs["MC"]),
                              None if cache_path is None else cache_path.encode(), _stream(stream),
                              ctypes.byref(best)))
    return int(best.value)


def _batch_items(meshes, which):
    """lfem_batch_item records of the meshes, with their float outputs."""
    items = (_BatchItem * len(meshes))()
    kept = []
    coef_f32 = 1
    for i, m in enumerate(meshes):
        pat, coords, rule = m["pattern"], _dev_f64(m["coords"], "coords"), as_rule(m["rule"])
        coef = m.get("coef")
        if coef is not None:
            coef_f32 = int(coef.dtype == torch.float32)
        outs = {k: (torch.empty(max(pat.nnz, 1), dtype=torch.float32, device=coords.device) if which & bit
                    else None) for k, bit in (("M", MASS), ("A", STIFF), ("MC", CMASS))}
        kept.append({"pattern": pat, "coords": coords, "rule": rule, "coef": coef, "out": outs})
        it = items[i]
        it.pattern = pat.handle.value
        it.coords = coords.data_ptr()
        it.ambient = int(coords.shape[1])
        it.quad = None if rule._c is None else ctypes.addressof(rule._c)
        it.coef = None if coef is None else coef.data_ptr()
        it.M = None if outs["M"] is None else outs["M"].data_ptr()
        it.A = None if outs["A"] is None else outs["A"].data_ptr()
        it.MC = None if outs["MC"] is None else outs["MC"].data_ptr()
    return items, kept, coef_f32


def batch_autotune(meshes, which: int = MASS | STIFF, cache_path: Optional[str] = None, stream=None):
    """lfem_batch_autotune: retile the meshes' patterns to the fastest tile
    capacity per element family; returns the capacities of
    (P1 curves, P2 curves, P1 triangles, P2 triangles), 0 for absent ones."""
    items, kept, coef_f32 = _batch_items(meshes, int(which))
    best = (ctypes.c_int32 * 4)()
    _check(_lib.lfem_batch_autotune(items, len(meshes), int(which), coef_f32,
                                    None if cache_path is None else cache_path.encode(), _stream(stream), best))
    del kept
    return tuple(int(v) for v in best)


class Batch:
    """Many meshes assembled by one persistent launch (lfem_batch_*), mixed precision.

    meshes: list of dicts with keys pattern, coords, rule and optionally coef.
    Outputs are allocated here (float [nnz] per requested matrix) and stay fixed,
    so the launch can be captured once as a CUDA graph and replayed while the
    coordinates change in place."""

    def __init__(self, meshes, which: int = MASS | STIFF, stream=None):
        self.which = int(which)
        items, self.meshes, coef_f32 = _batch_items(meshes, self.which)
        self._items = items
        h = ctypes.c_void_p()
        _check(_lib.lfem_batch_create(items, len(meshes), self.which, coef_f32, _stream(stream), ctypes.byref(h)))
        self._h = h

    def assemble(self, stream=None):
        _check(_lib.lfem_batch_assemble(self._h, _stream(stream)))

    def graph_launch(self, stream=None):
        _check(_lib.lfem_batch_graph_launch(self._h, _stream(stream)))

    def sync_status(self, stream=None):
        _check(_lib.lfem_batch_sync_status(self._h, _stream(stream)))

    def info(self):
        n, e, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(_lib.lfem_batch_info(self._h, ctypes.byref(n), ctypes.byref(e), ctypes.byref(c)))
        return {"work_items": n.value, "elements_computed": e.value, "cap_elements": c.value}

    def outputs(self, i):
        m = self.meshes[i]
        nnz = m["pattern"].nnz
        return {k: v[:nnz] for k, v in m["out"].items() if v is not None}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.lfem_batch_destroy(h)
            self._h = ctypes.c_void_p()


def assemble_adjoint(pat: Pattern, coords: torch.Tensor, rule, coef=None, gM=None, gA=None, gMC=None,
                     want_coef_grad: bool = False, stream=None, precision: int = FP64):
    """lfem_assemble_adjoint (FP64) or lfem_assemble_adjoint_mixed: returns (g_coords, g_coef or None)."""
    coords = _dev_f64(coords, "coords")
    rule = as_rule(rule)
    gx = torch.empty_like(coords)
    gc = None
    if want_coef_grad:
        gc = torch.empty(pat.n_elem, rule.n_pts, dtype=torch.float64, device=coords.device)
    fn = _lib.lfem_assemble_adjoint if precision == FP64 else _lib.lfem_assemble_adjoint_mixed
    _check(fn(pat.handle, _ptr(coords), int(coords.shape[1]), rule.ref,
                                      _ptr(_dev_f64(coef, "coef")), _ptr(_dev_f64(gM, "gM")),
                                      _ptr(_dev_f64(gA, "gA")), _ptr(_dev_f64(gMC, "gMC")), _ptr(gx), _ptr(gc),
                                      _stream(stream)))
    return gx, gc


def assemble_load(pat: Pattern, coords: torch.Tensor, rule, f: torch.Tensor, stream=None) -> torch.Tensor:
    """lfem_assemble_load: b_j = integral of f_h phi_j for nodal f ([n_nodes]); returns b (b = M f)."""
    coords = _dev_f64(coords, "coords")
    rule = as_rule(rule)
    f = _dev_f64(f, "f")
    b = torch.empty(pat.n_nodes, dtype=torch.float64, device=coords.device)
    _check(_lib.lfem_assemble_load(pat.handle, _ptr(coords), int(coords.shape[1]), rule.ref, _ptr(f), _ptr(b),
                                   _stream(stream)))
    return b


def assemble_mcf_nonlinear(pat: Pattern, coords: torch.Tensor, rule, u: torch.Tensor, stream=None) -> torch.Tensor:
    """lfem_assemble_mcf_nonlinear: u = (nu, H) at the nodes ([n_nodes][4]); returns [4][n_nodes]."""
    coords = _dev_f64(coords, "coords")
    rule = as_rule(rule)
    u = _dev_f64(u, "u")
    out = torch.empty(4, pat.n_nodes, dtype=torch.float64, device=coords.device)
    _check(_lib.lfem_assemble_mcf_nonlinear(pat.handle, _ptr(coords), rule.ref, _ptr(u), _ptr(out), _stream(stream)))
    return out


def mcf_step(pat: Pattern, coords: torch.Tensor, rule, tau: float, rtol: float = 1e-12, max_iter: int = 2000,
             out=None, stream=None):
    """lfem_mcf_step: one step of Dziuk's scheme; returns (x1, cg_iterations)."""
    coords = _dev_f64(coords, "coords")
    rule = as_rule(rule)
    x1 = torch.empty_like(coords) if out is None else _dev_f64(out, "out")
    it = ctypes.c_int()
    _check(_lib.lfem_mcf_step(pat.handle, _ptr(coords), int(coords.shape[1]), rule.ref, float(tau), float(rtol),
                              int(max_iter), _ptr(x1), ctypes.byref(it), _stream(stream)))
    return x1, int(it.value)


def lift_order(pat1: Pattern, coords: torch.Tensor, order: int, stream=None):
    """lfem_lift_order: order-p nodes of an order-1 mesh; returns (coords_p, conn_p)."""
    coords = _dev_f64(coords, "coords")
    n = ctypes.c_int64()
    _check(_lib.lfem_lift_order(pat1.handle, _ptr(coords), int(coords.shape[1]), int(order), None, None,
                                ctypes.byref(n), _stream(stream)))
    ref = math.comb(order + pat1.dim, pat1.dim)
    conn = torch.empty(pat1.n_elem, ref, dtype=torch.int32, device=coords.device)
    out = torch.empty(n.value, coords.shape[1], dtype=torch.float64, device=coords.device)
    _check(_lib.lfem_lift_order(pat1.handle, _ptr(coords), int(coords.shape[1]), int(order), _ptr(conn), _ptr(out),
                                ctypes.byref(n), _stream(stream)))
    return out, conn


def eval_points(conn, dim, order, coords, rule, stream=None):
    conn = _dev_i32(conn)
    coords = _dev_f64(coords, "coords")
    rule = as_rule(rule)
    n = int(coords.shape[1])
    out = torch.empty(conn.shape[0], rule.n_pts, n, dtype=torch.float64, device=coords.device)
    _check(_lib.lfem_eval_points(_ptr(conn), conn.shape[0], dim, order, _ptr(coords), n, rule.ref, _ptr(out),
                                 _stream(stream)))
    return out


def geometry(conn, dim, order, coords, rule, stream=None):
    conn = _dev_i32(conn)
    coords = _dev_f64(coords, "coords")
    rule = as_rule(rule)
    n = int(coords.shape[1])
    nE, Q = conn.shape[0], rule.n_pts
    J = torch.empty(nE, Q, n, dim, dtype=torch.float64, device=coords.device)
    s = torch.empty(nE, Q, dtype=torch.float64, device=coords.device)
    Gi = torch.empty(nE, Q, dim, dim, dtype=torch.float64, device=coords.device)
    _check(_lib.lfem_geometry(_ptr(conn), nE, dim, order, _ptr(coords), n, rule.ref, _ptr(J), _ptr(s), _ptr(Gi),
                              _stream(stream)))
    return J, s, Gi


def local(conn, dim, order, coords, rule, coef=None, which=MASS | STIFF, stream=None):
    conn = _dev_i32(conn)
    coords = _dev_f64(coords, "coords")
    rule = as_rule(rule)
    n = int(coords.shape[1])
    ref = int(conn.shape[1])
    U = ref * (ref + 1) // 2
    mk = lambda bit: torch.empty(conn.shape[0], U, dtype=torch.float64, device=coords.device) if which & bit else None
    M, A, C = mk(MASS), mk(STIFF), mk(CMASS)
    _check(_lib.lfem_local(_ptr(conn), conn.shape[0], dim, order, _ptr(coords), n, rule.ref,
                           _ptr(_dev_f64(coef, "coef")), _ptr(M), _ptr(A), _ptr(C), _stream(stream)))
    return M, A, C


def pattern_csr_noalloc(conn: torch.Tensor, n_nodes: int, dim: int, order: int, row_ptr: torch.Tensor,
                        col_idx: torch.Tensor, stream=None) -> int:
    """lfem_pattern_csr_noalloc: CSR pattern into caller buffers with no device
    allocation inside the library; returns nnz (raises if col_idx is too small)."""
    conn = _dev_i32(conn)
    if not (row_ptr.is_cuda and row_ptr.dtype == torch.int64 and row_ptr.numel() >= n_nodes + 1):
        raise TypeError("row_ptr must be an int64 CUDA tensor of n_nodes + 1 entries")
    if not (col_idx.is_cuda and col_idx.dtype == torch.int32):
        raise TypeError("col_idx must be an int32 CUDA tensor")
    nnz = ctypes.c_int64()
    _check(_lib.lfem_pattern_csr_noalloc(_ptr(conn), int(conn.shape[0]), int(n_nodes), int(dim), int(order),
                                         _ptr(row_ptr), _ptr(col_idx), int(col_idx.numel()), ctypes.byref(nnz),
                                         _stream(stream)))
    return int(nnz.value)


class AssembleFn(torch.autograd.Function):
    """(coords, coef) -> (M, A, MC) CSR values; backward calls the adjoint kernel.
    precision FP64 (default): FP64 values and adjoint; MIXED: float values from the
    mixed assembly and the mixed adjoint (gradients in double)."""

    @staticmethod
    def forward(ctx, coords, coef, pat: Pattern, rule, precision: int = FP64):
        rule = as_rule(rule)
        which = MASS | STIFF | (CMASS if coef is not None else 0)
        cf = None if coef is None else coef.detach().contiguous()
        if cf is not None and precision != FP64:
            cf = cf.float()
        out = assemble(pat, coords.detach().contiguous(), rule, cf, which=which, precision=precision)
        ctx.pat, ctx.rule, ctx.precision = pat, rule, precision
        ctx.save_for_backward(coords, coef if coef is not None else torch.empty(0, device=coords.device))
        ctx.has_coef = coef is not None
        mc = out.get("MC", torch.zeros_like(out["M"]))
        return out["M"], out["A"], mc

    @staticmethod
    def backward(ctx, gM, gA, gMC):
        coords, coef = ctx.saved_tensors
        coef = coef if ctx.has_coef else None
        c = lambda g: None if g is None else g.contiguous().to(torch.float64)
        gx, gc = assemble_adjoint(ctx.pat, coords.detach().contiguous(), ctx.rule,
                                  None if coef is None else coef.detach().contiguous(), c(gM), c(gA),
                                  c(gMC) if ctx.has_coef else None, want_coef_grad=ctx.has_coef,
                                  precision=ctx.precision)
        if gc is not None and coef is not None:
            gc = gc.to(coef.dtype)
        return gx, gc, None, None, None
