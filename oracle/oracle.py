"""ctypes wrapper of lfem_oracle.c plus the pattern definition in numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function cites
the passage of the paper it follows; the C file holds the element loops.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfem_oracle.c")
_lock = threading.Lock()
_libs: dict = {}


def _lib_path(mutation: int) -> str:
    tag = "" if mutation == 0 else f"_mut{mutation}"
    return os.path.join(_HERE, f"liblfem_oracle{tag}.so")


def build(mutation: int = 0, force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math).  `mutation` > 0 builds a
    copy with one planted mistake, used only by the tests that check the pins
    catch it."""
    path = _lib_path(mutation)
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = f"{path}.{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-fopenmp",
               f"-DORACLE_MUTATION={mutation}", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return path


def _lib(mutation: int = 0):
    with _lock:
        if mutation in _libs:
            return _libs[mutation]
        lib = ctypes.CDLL(build(mutation))
        P = ctypes.c_void_p
        I = ctypes.c_int
        L = ctypes.c_int64
        lib.oracle_tabulate.argtypes = [I, I, I, P, P, P]
        lib.oracle_eval_points.argtypes = [P, I, P, L, I, I, I, P, P]
        lib.oracle_geometry.argtypes = [P, I, P, L, I, I, I, P, P, P, P]
        lib.oracle_local.argtypes = [P, I, P, L, I, I, I, P, P, P, P, P, P]
        lib.oracle_assemble.argtypes = [P, I, P, L, I, I, I, P, P, P, P, P, L, P, P, P]
        lib.oracle_assemble_threads.argtypes = [P, I, P, L, L, I, I, I, P, P, P, P, P, L, P, P, P, I]
        lib.oracle_adjoint.argtypes = [P, I, P, L, L, I, I, I, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_load.argtypes = [P, I, P, L, L, I, I, I, P, P, P, P]
        lib.oracle_kll.argtypes = [P, P, L, L, I, I, P, P, P, P]
        for f in ("oracle_tabulate", "oracle_eval_points", "oracle_geometry", "oracle_local",
                  "oracle_assemble", "oracle_assemble_threads", "oracle_max_threads", "oracle_adjoint", "oracle_load",
                  "oracle_kll", "oracle_mutation_id"):
            getattr(lib, f).restype = ctypes.c_int
        _libs[mutation] = lib
        return lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def n_ref(dim: int, order: int) -> int:
    """Local nodes per element, C(p+d, d) (Sec. 4, dim(E))."""
    from math import comb

    if order in (1, 2, 3, 4) and dim in (1, 2, 3):
        return comb(order + dim, dim)
    raise ValueError((dim, order))


def tabulate(dim, order, xi, mutation=0):
    """Basis values phi [Q][ref] and reference gradients [Q][ref][dim] (Lagrange
    P1/P2 on the reference simplex; Eq. form_functions_s2dp2 read as Lagrange)."""
    xi = _f64(xi).reshape(-1, dim)
    nq = xi.shape[0]
    ref = n_ref(dim, order)
    phi = np.zeros((nq, ref))
    dphi = np.zeros((nq, ref, dim))
    rc = _lib(mutation).oracle_tabulate(dim, order, nq, _p(xi), _p(phi), _p(dphi))
    if rc:
        raise ValueError("unsupported element")
    return phi, dphi


def pattern(conn, n_nodes):
    """CSR pattern of all structural pairs (E[e,a], E[e,b]) with duplicates merged,
    the index set that sparse(I(:), J(:), .) builds (Sec. 3.4 (b), Sec. 3.3):
    sort lexicographically, unique.  Returns (row_ptr int64 [N+1], col_idx int32)."""
    conn = np.asarray(conn, dtype=np.int64)
    ref = conn.shape[1]
    I = np.repeat(conn, ref, axis=1).ravel()
    J = np.tile(conn, (1, ref)).ravel()
    key = np.unique(I * np.int64(n_nodes) + J)
    rows = key // n_nodes
    cols = (key % n_nodes).astype(np.int32)
    row_ptr = np.zeros(n_nodes + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n_nodes), out=row_ptr[1:])
    return row_ptr, cols


def p1_exact(coords, conn, dim):
    """Order-1 M and A from the exact reference matrices, the paper's P1
    precomputation (Sec. 4.2): the element map is affine, so with s_E =
    sqrt(det G_E), G_E = J_E^T J_E, J_E = [x_1 - x_0, ..., x_d - x_0],
      M_E = s_E M_ref,            M_ref(a, b) = int_ref lambda_a lambda_b
                                              = (1 + delta_ab) / (d! (d+1) (d+2)),
      A_E = s_E sum_mn (G_E^-1)_mn A_ref_mn,  A_ref_mn(a, b) = |ref| d_m lambda_a d_n lambda_b,
    with |ref| = 1 / d! and d_m lambda_0 = -1, d_m lambda_k = delta_mk.  Then
    summed into the pattern's slots (Eqs. M matrix, A matrix).  numpy, no
    quadrature.  Returns (row_ptr, col_idx, M, A)."""
    from math import factorial

    x = np.asarray(coords, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    e = np.asarray(conn, dtype=np.int64)
    assert e.shape[1] == dim + 1
    N = x.shape[0]
    X = x[e]                                         # [nE][d+1][n]
    T = X[:, 1:, :] - X[:, :1, :]                    # rows t_m = x_m - x_0 (columns of J)
    G = np.einsum("emi,eki->emk", T, T)
    s = np.sqrt(np.linalg.det(G))
    Gi = np.linalg.inv(G)
    m_ref = (1.0 + np.eye(dim + 1)) / (factorial(dim) * (dim + 1) * (dim + 2))
    dl = np.vstack([-np.ones(dim), np.eye(dim)])     # [d+1][d], d_m lambda_a
    a_ref = np.einsum("am,bn->mnab", dl, dl) / factorial(dim)
    Ml = s[:, None, None] * m_ref[None]
    Al = s[:, None, None] * np.einsum("emn,mnab->eab", Gi, a_ref)
    rp, ci = pattern(conn, N)
    rows = np.repeat(np.arange(N, dtype=np.int64), np.diff(rp))
    keys = rows * N + ci
    ref = dim + 1
    I = np.repeat(e, ref, axis=1).ravel()
    J = np.tile(e, (1, ref)).ravel()
    slot = np.searchsorted(keys, I * N + J)
    M = np.zeros(keys.size)
    A = np.zeros(keys.size)
    np.add.at(M, slot, Ml.ravel())
    np.add.at(A, slot, Al.ravel())
    return rp, ci, M, A


def eval_points(coords, conn, dim, order, xi, mutation=0):
    """Physical points F_E(xi_q) for every element (Eq. F_map): [nE][Q][n]."""
    coords = _f64(coords)
    conn = _i32(conn)
    xi = _f64(xi).reshape(-1, dim)
    n = coords.shape[1]
    out = np.zeros((conn.shape[0], xi.shape[0], n))
    rc = _lib(mutation).oracle_eval_points(_p(coords), n, _p(conn), conn.shape[0], dim, order, xi.shape[0],
                                           _p(xi), _p(out))
    if rc:
        raise ValueError("unsupported element")
    return out


def geometry(coords, conn, dim, order, xi, mutation=0):
    """J [nE][Q][n][d], s = |det DF| [nE][Q], G^{-1} [nE][Q][d][d] (Sec. 3.2.1)."""
    coords = _f64(coords)
    conn = _i32(conn)
    xi = _f64(xi).reshape(-1, dim)
    n = coords.shape[1]
    nE, nq = conn.shape[0], xi.shape[0]
    J = np.zeros((nE, nq, n, dim))
    s = np.zeros((nE, nq))
    Gi = np.zeros((nE, nq, dim, dim))
    rc = _lib(mutation).oracle_geometry(_p(coords), n, _p(conn), nE, dim, order, nq, _p(xi), _p(J), _p(s), _p(Gi))
    if rc:
        raise ValueError("unsupported element")
    return J, s, Gi


def local_matrices(coords, conn, dim, order, xi, w, coef=None, mutation=0):
    """Element matrices M_loc, A_loc, MC_loc [nE][ref][ref] by quadrature
    (Eqs. reference_quadrature_mass, reference_quadrature_stiffness)."""
    coords = _f64(coords)
    conn = _i32(conn)
    xi = _f64(xi).reshape(-1, dim)
    w = _f64(w)
    coef = _f64(coef)
    n = coords.shape[1]
    nE, nq = conn.shape[0], xi.shape[0]
    ref = n_ref(dim, order)
    M = np.zeros((nE, ref, ref))
    A = np.zeros((nE, ref, ref))
    C = np.zeros((nE, ref, ref))
    rc = _lib(mutation).oracle_local(_p(coords), n, _p(conn), nE, dim, order, nq, _p(xi), _p(w), _p(coef),
                                     _p(M), _p(A), _p(C))
    if rc:
        raise ValueError("unsupported element")
    return M, A, C


def assemble(coords, conn, dim, order, xi, w, coef=None, pat=None, mutation=0):
    """Global M, A, MC values over the CSR pattern (Eqs. M matrix, A matrix).
    Returns (row_ptr, col_idx, M, A, MC); MC is zero when coef is None."""
    coords = _f64(coords)
    conn = _i32(conn)
    xi = _f64(xi).reshape(-1, dim)
    w = _f64(w)
    coef = _f64(coef)
    n = coords.shape[1]
    if pat is None:
        pat = pattern(conn, coords.shape[0])
    row_ptr, col_idx = pat
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = _i32(col_idx)
    nnz = col_idx.shape[0]
    M = np.zeros(nnz)
    A = np.zeros(nnz)
    C = np.zeros(nnz)
    rc = _lib(mutation).oracle_assemble(_p(coords), n, _p(conn), conn.shape[0], dim, order, xi.shape[0], _p(xi),
                                        _p(w), _p(coef), _p(row_ptr), _p(col_idx), nnz, _p(M), _p(A), _p(C))
    if rc:
        raise ValueError(f"oracle_assemble failed ({rc})")
    return row_ptr, col_idx, M, A, C


def assemble_threads(coords, conn, dim, order, xi, w, coef=None, pat=None, n_nodes=None, threads=0):
    """The same global assembly on every host core (or `threads`): bit-identical
    to assemble() -- each slot's contributions are added in the same order with
    the same compensated sums.  Returns (row_ptr, col_idx, M, A, MC)."""
    coords = _f64(coords)
    conn = _i32(conn)
    xi = _f64(xi).reshape(-1, dim)
    w = _f64(w)
    coef = _f64(coef)
    n = coords.shape[1]
    nn = coords.shape[0] if n_nodes is None else n_nodes
    if pat is None:
        pat = pattern(conn, nn)
    row_ptr, col_idx = pat
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = _i32(col_idx)
    nnz = col_idx.shape[0]
    M = np.zeros(nnz)
    A = np.zeros(nnz)
    C = np.zeros(nnz)
    rc = _lib().oracle_assemble_threads(_p(coords), n, _p(conn), conn.shape[0], nn, dim, order, xi.shape[0], _p(xi),
                                        _p(w), _p(coef), _p(row_ptr), _p(col_idx), nnz, _p(M), _p(A), _p(C),
                                        int(threads))
    if rc:
        raise ValueError(f"oracle_assemble_threads failed ({rc})")
    return row_ptr, col_idx, M, A, C


def max_threads():
    """Threads the all-core oracle uses by default."""
    return int(_lib().oracle_max_threads())


def load(coords, conn, dim, order, xi, w, f, mutation=0):
    """Load vector b_j = int f_h phi_j with f_h the interpolant of nodal f (Sec. 2; b = M f)."""
    coords = _f64(coords)
    conn = _i32(conn)
    xi = _f64(xi).reshape(-1, dim)
    w = _f64(w)
    f = _f64(f)
    b = np.zeros(coords.shape[0])
    rc = _lib(mutation).oracle_load(_p(coords), coords.shape[1], _p(conn), conn.shape[0], coords.shape[0], dim, order,
                                    xi.shape[0], _p(xi), _p(w), _p(f), _p(b))
    if rc:
        raise ValueError(f"oracle_load failed ({rc})")
    return b


def kll(coords, conn, order, xi, w, u, mutation=0):
    """Non-linear vectors of the mean curvature flow system (Sec. 5.1): u = (nu, H) nodal [N][4];
    returns [4][N]: rows 0..2 = int alpha^2 (nu_h)_k phi_j, row 3 = int alpha^2 H_h phi_j."""
    coords = _f64(coords)
    conn = _i32(conn)
    xi = _f64(xi).reshape(-1, 2)
    w = _f64(w)
    u = _f64(u).reshape(-1, 4)
    out = np.zeros((4, coords.shape[0]))
    rc = _lib(mutation).oracle_kll(_p(coords), _p(conn), conn.shape[0], coords.shape[0], order, xi.shape[0], _p(xi),
                                   _p(w), _p(u), _p(out))
    if rc:
        raise ValueError(f"oracle_kll failed ({rc})")
    return out


def mcf_step(coords, conn, dim, order, xi, w, tau, mutation=0):
    """One step of Dziuk's scheme (the starting point of the flow example, Sec. 5.1):
    (M(x0) + tau A(x0)) x1 = M(x0) x0, per coordinate, with the oracle's FP64 M and A
    and a sparse direct solve (library primitive).  Returns x1 [N][n]."""
    import scipy.sparse as sps
    import scipy.sparse.linalg as spl

    coords = _f64(coords)
    rp, ci, M, A, _ = assemble(coords, conn, dim, order, xi, w, mutation=mutation)
    n = coords.shape[0]
    Mm = sps.csr_matrix((M, ci, rp), shape=(n, n))
    Km = sps.csr_matrix((M + tau * A, ci, rp), shape=(n, n))
    rhs = Mm @ coords
    out = np.empty_like(coords)
    used = np.diff(rp) > 0
    K_used = Km[used][:, used].tocsc()
    sol = spl.spsolve(K_used, rhs[used])
    out[used] = sol.reshape(-1, coords.shape[1])
    out[~used] = coords[~used]
    return out


def adjoint(coords, conn, dim, order, xi, w, coef, pat, gM=None, gA=None, gMC=None, mutation=0):
    """dL/dx [N][n] and dL/dc [nE][Q] for L = gM.M + gA.A + gMC.MC (closed forms in
    lfem_oracle.c; derived from Eqs. reference_quadrature_mass / _stiffness)."""
    coords = _f64(coords)
    conn = _i32(conn)
    xi = _f64(xi).reshape(-1, dim)
    w = _f64(w)
    coef = _f64(coef)
    row_ptr, col_idx = pat
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = _i32(col_idx)
    n = coords.shape[1]
    gx = np.zeros_like(coords)
    gc = np.zeros((conn.shape[0], xi.shape[0]))
    rc = _lib(mutation).oracle_adjoint(_p(coords), n, _p(conn), conn.shape[0], coords.shape[0], dim, order,
                                       xi.shape[0], _p(xi), _p(w), _p(coef), _p(row_ptr), _p(col_idx),
                                       _p(_f64(gM)), _p(_f64(gA)), _p(_f64(gMC)), _p(gx), _p(gc))
    if rc:
        raise ValueError(f"oracle_adjoint failed ({rc})")
    return gx, gc


if __name__ == "__main__":  # pragma: no cover
    print(build(int(sys.argv[1]) if len(sys.argv) > 1 else 0))
