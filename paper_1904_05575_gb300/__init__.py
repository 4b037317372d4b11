"""Python binding of libbse.so: ctypes marshalling of torch CUDA tensors onto
the C ABI declared in include/bse.h.  Every step of the computation runs in
the library's CUDA kernels (and the cuSOLVER / cuBLAS calls it makes); this
module only checks tensor placement and passes pointers.  It raises if the
library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbse.so")

BSE_OK, BSE_ERR_ARG, BSE_ERR_CUDA, BSE_ERR_NOMEM = 0, -1, -2, -3
BSE_ERR_NOT_PD, BSE_ERR_NO_CONV, BSE_ERR_TIMEOUT, BSE_ERR_UNSUPPORTED = -4, -5, -6, -7
BSE_PREC_FP64, BSE_PREC_BF16X6, BSE_PREC_BF16X3 = 0, 2, 3
BSE_C128, BSE_C64 = 0, 1   # bse_problem.in_dtype
BSE_PLAN_AUTOTUNE = 1
BSE_PLAN_UNFUSED = 2
BSE_PLAN_CUDA_CORE_STAGE2 = 4
BSE_PLAN_HERMITIAN = 8
BSE_PLAN_FP64_DIAGONAL = 16
HARTREE_EV = 27.211386245988

STATUS_NAMES = {0: "BSE_OK", -1: "BSE_ERR_ARG", -2: "BSE_ERR_CUDA", -3: "BSE_ERR_NOMEM",
                -4: "BSE_ERR_NOT_PD", -5: "BSE_ERR_NO_CONV", -6: "BSE_ERR_TIMEOUT",
                -7: "BSE_ERR_UNSUPPORTED"}


class BSEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class bse_problem(ctypes.Structure):
    _fields_ = [
        ("nk", ctypes.c_int32), ("nv", ctypes.c_int32), ("nc", ctypes.c_int32),
        ("ng", ctypes.c_int32), ("nq_w", ctypes.c_int32),
        ("omega_cell", ctypes.c_double), ("gamma_x", ctypes.c_double),
        ("gamma_c", ctypes.c_double), ("coupling", ctypes.c_int32),
        ("e_v", ctypes.c_void_p), ("e_c", ctypes.c_void_p),
        ("m_x", ctypes.c_void_p), ("m_vv", ctypes.c_void_p), ("m_cc", ctypes.c_void_p),
        ("n_vc", ctypes.c_void_p), ("w", ctypes.c_void_p),
        ("q_minus", ctypes.c_void_p), ("q_plus", ctypes.c_void_p),
        ("v_bar", ctypes.c_void_p),
        ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("ld", ctypes.c_int64),
        ("k_begin", ctypes.c_int32), ("k_count", ctypes.c_int32),
        ("in_dtype", ctypes.c_int32),
    ]


_lib: Optional[ctypes.CDLL] = None

EXPORTED = ("bse_build_kernel", "bse_reduce", "bse_spectrum", "bse_last_error", "bse_version",
            "bse_kernel_launches", "bse_precision_supported", "bse_phase_timing",
            "bse_phase_report", "bse_build_kernel_fp64_static", "bse_lowest_excitons",
            "bse_mlp_create", "bse_mlp_destroy", "bse_mlp_num_params", "bse_mlp_get_params",
            "bse_mlp_set_params", "bse_mlp_samples", "bse_mlp_loss_grad", "bse_mlp_train",
            "bse_mlp_predict", "bse_xpy", "bse_mlp_trajectory_samples", "bse_mlp_set_neighbours",
            "bse_mlp_features", "bse_plan_create",
            "bse_plan_execute", "bse_plan_status", "bse_plan_tile_cols", "bse_plan_destroy",
            "bse_plan_stage2_shape", "bse_spectrum_lanczos",
            "bse_plan_fused", "bse_spectrum_tensor", "bse_loss_function",
            "bse_lowest_excitons_from", "bse_rpa_screening", "bse_plan_set_wait_limit",
            "bse_pair_elements")


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libbse.so (built by build.py / __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.bse_build_kernel.argtypes = [ctypes.POINTER(bse_problem), i32, i32, vp]
    lib.bse_reduce.argtypes = [i32, vp, vp, i64, vp, vp, ctypes.POINTER(i32), vp]
    lib.bse_spectrum.argtypes = [i32, vp, vp, i64, vp, dbl, dbl, i32, vp, dbl, vp, vp, vp, vp]
    lib.bse_spectrum_lanczos.argtypes = [i32, vp, vp, i64, vp, dbl, dbl, i32, vp, dbl, dbl, i32,
                                         i32, vp, ctypes.POINTER(i32), vp]
    lib.bse_spectrum_lanczos.restype = ctypes.c_int
    lib.bse_spectrum_tensor.argtypes = [i32, vp, vp, i64, vp, i64, dbl, dbl, i32, vp, dbl, vp, vp,
                                        vp]
    lib.bse_spectrum_tensor.restype = ctypes.c_int
    lib.bse_loss_function.argtypes = [i32, vp, dbl, vp, vp, vp]
    lib.bse_loss_function.restype = ctypes.c_int
    lib.bse_last_error.restype = ctypes.c_char_p
    lib.bse_kernel_launches.restype = ctypes.c_int64
    lib.bse_build_kernel_fp64_static.argtypes = [ctypes.POINTER(bse_problem), vp]
    lib.bse_build_kernel_fp64_static.restype = ctypes.c_int
    lib.bse_lowest_excitons.argtypes = [i32, vp, vp, i64, i32, dbl, i32, i32, vp, i32, vp, vp,
                                        ctypes.POINTER(i32), vp]
    lib.bse_lowest_excitons.restype = ctypes.c_int
    lib.bse_lowest_excitons_from.argtypes = [i32, vp, vp, i64, i32, dbl, i32, i32, vp, i32, vp,
                                             i32, vp, vp, ctypes.POINTER(i32), vp]
    lib.bse_lowest_excitons_from.restype = ctypes.c_int
    lib.bse_rpa_screening.argtypes = [i32, i32, i32, i32, dbl, vp, vp, vp, vp, i32, vp, vp]
    lib.bse_rpa_screening.restype = ctypes.c_int
    lib.bse_xpy.argtypes = [i32, i32, vp, vp, i64, vp, vp, vp]
    lib.bse_xpy.restype = ctypes.c_int
    lib.bse_plan_create.argtypes = [ctypes.POINTER(bse_problem), i32, i32, i32,
                                    ctypes.POINTER(vp), vp]
    lib.bse_plan_execute.argtypes = [vp, vp]
    lib.bse_plan_status.argtypes = [vp, vp]
    lib.bse_plan_tile_cols.argtypes = [vp]
    lib.bse_plan_stage2_shape.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.bse_plan_stage2_shape.restype = ctypes.c_int
    lib.bse_plan_fused.argtypes = [vp]
    lib.bse_plan_destroy.argtypes = [vp]
    lib.bse_plan_destroy.restype = None
    lib.bse_plan_set_wait_limit.argtypes = [vp, dbl]
    lib.bse_pair_elements.argtypes = [i32, i32, i32, i32, i32, vp, vp, vp, vp, i32, i32, vp, vp,
                                      vp, vp, vp]
    lib.bse_pair_elements.restype = ctypes.c_int
    lib.bse_plan_set_wait_limit.restype = ctypes.c_int
    for name in ("bse_plan_create", "bse_plan_execute", "bse_plan_status", "bse_plan_tile_cols",
                 "bse_plan_fused"):
        getattr(lib, name).restype = ctypes.c_int
    f32p = ctypes.POINTER(ctypes.c_float)
    lib.bse_mlp_create.argtypes = [ctypes.POINTER(vp), i32, i32, ctypes.c_uint64]
    lib.bse_mlp_destroy.argtypes = [vp]
    lib.bse_mlp_destroy.restype = None
    lib.bse_mlp_num_params.argtypes = [vp]
    lib.bse_mlp_num_params.restype = ctypes.c_int64
    lib.bse_mlp_get_params.argtypes = [vp, f32p, i64]
    lib.bse_mlp_set_params.argtypes = [vp, f32p, i64]
    lib.bse_mlp_samples.argtypes = [i32, vp, vp, i64, i32, vp, vp, vp, dbl, vp, vp, vp, vp]
    lib.bse_mlp_trajectory_samples.argtypes = [i32, vp, vp, i64, i32, vp, vp, dbl, i32, vp, vp,
                                               i32, i64, vp, vp, vp, ctypes.POINTER(i64), vp]
    lib.bse_mlp_set_neighbours.argtypes = [vp, i32, i32, vp, i32, vp]
    lib.bse_mlp_set_neighbours.restype = ctypes.c_int
    lib.bse_mlp_features.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp]
    lib.bse_mlp_features.restype = ctypes.c_int
    lib.bse_mlp_trajectory_samples.restype = ctypes.c_int
    lib.bse_mlp_loss_grad.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(dbl), f32p, vp]
    lib.bse_mlp_train.argtypes = [vp, vp, vp, vp, i64, i32, dbl, ctypes.POINTER(dbl), vp]
    lib.bse_mlp_predict.argtypes = [vp, vp, i64, vp, vp]
    for name in ("bse_mlp_create", "bse_mlp_get_params", "bse_mlp_set_params", "bse_mlp_samples",
                 "bse_mlp_loss_grad", "bse_mlp_train", "bse_mlp_predict"):
        getattr(lib, name).restype = ctypes.c_int
    lib.bse_phase_timing.argtypes = [i32]
    lib.bse_phase_report.argtypes = [ctypes.c_char_p, i64]
    lib.bse_precision_supported.argtypes = [i32]
    lib.bse_precision_supported.restype = ctypes.c_int
    for name in ("bse_build_kernel", "bse_reduce", "bse_spectrum", "bse_version"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != BSE_OK:
        msg = load().bse_last_error().decode(errors="replace")
        raise BSEError(status, msg)


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _matrix_ptr(t, n, name):
    """Column-major N x N with ld: a torch tensor of shape [n_cols, ld] (row r of
    the tensor is column r of the matrix)."""
    import torch
    if t.dim() != 2 or t.shape[0] != n or t.shape[1] < n:
        raise ValueError(f"{name} must have shape [n, ld] with ld >= n")
    return _ptr(t, torch.complex128, name), t.shape[1]


def _check_shapes(d: Dict, kn: int, coupling: bool) -> None:
    """The array shapes include/bse.h states (the library reads them through
    bare pointers and cannot check them): raises ValueError on a mismatch."""
    nk, nv, nc, ng = d["nk"], d["nv"], d["nc"], d["ng"]
    nq = d["w"].shape[0] if d.get("w") is not None else 0
    want = {"e_v": (nk, nv), "e_c": (nk, nc), "m_x": (nk, nv, nc, ng), "v_bar": (ng,),
            "w": (nq, ng, ng), "q_minus": (nk, nk), "m_vv": (kn, nk, nv, nv, ng),
            "m_cc": (kn, nk, nc, nc, ng)}
    if coupling:
        want.update(n_vc=(nk, nk, nv, nc, ng), q_plus=(nk, nk))
    for name, shape in want.items():
        t = d.get(name)
        if t is not None and tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")


def make_problem_struct(d: Dict, gamma_x: float = 1.0, gamma_c: float = 1.0,
                        coupling: bool = True, k_begin: int = 0,
                        k_count: int = 0) -> bse_problem:
    """bse_problem from a dict of CUDA tensors (see upload_problem) and outputs A, B.

    k_count > 0 builds only the rows k_begin <= k < k_begin + k_count of A and
    B; m_vv and m_cc then hold only those k rows ([k_count, nk, ...]) while
    n_vc stays whole ([nk, nk, ...])."""
    import torch
    f64, i32 = torch.float64, torch.int32
    # the complex inputs' storage: complex128 (BSE_C128) or complex64 (BSE_C64)
    c128 = d["m_x"].dtype
    if c128 not in (torch.complex128, torch.complex64):
        raise TypeError(f"m_x must be complex128 or complex64, got {c128}")
    n = d["nk"] * d["nv"] * d["nc"]
    nk = d["nk"]
    kn = k_count if k_count > 0 else nk
    if not (0 <= k_begin and k_count >= 0 and k_begin + k_count <= nk and (k_count > 0 or k_begin == 0)):
        raise ValueError(f"k-row slab [{k_begin}, {k_begin + k_count}) outside [0, {nk})")
    for name, rows in (("m_vv", kn), ("m_cc", kn), ("n_vc", nk)):
        t = d.get(name)
        if t is not None and (name != "n_vc" or coupling) and tuple(t.shape[:2]) != (rows, nk):
            raise ValueError(f"{name} must have leading shape ({rows}, {nk}), got {tuple(t.shape[:2])}")
    _check_shapes(d, kn, coupling)
    a_ptr, ld = _matrix_ptr(d["A"], n, "A")
    b_ptr = None
    if coupling:
        b_ptr, ldb = _matrix_ptr(d["B"], n, "B")
        if ldb != ld:
            raise ValueError("A and B must share ld")
    return bse_problem(
        nk=d["nk"], nv=d["nv"], nc=d["nc"], ng=d["ng"], nq_w=d["w"].shape[0],
        omega_cell=float(d["omega_cell"]), gamma_x=float(gamma_x), gamma_c=float(gamma_c),
        coupling=1 if coupling else 0,
        e_v=_ptr(d["e_v"], f64, "e_v"), e_c=_ptr(d["e_c"], f64, "e_c"),
        m_x=_ptr(d["m_x"], c128, "m_x"), m_vv=_ptr(d["m_vv"], c128, "m_vv"),
        m_cc=_ptr(d["m_cc"], c128, "m_cc"),
        n_vc=_ptr(d["n_vc"], c128, "n_vc") if coupling else None,
        w=_ptr(d["w"], c128, "w"), q_minus=_ptr(d["q_minus"], i32, "q_minus"),
        q_plus=_ptr(d["q_plus"], i32, "q_plus") if coupling else None,
        v_bar=_ptr(d["v_bar"], f64, "v_bar"), A=a_ptr, B=b_ptr, ld=ld,
        k_begin=int(k_begin), k_count=int(k_count),
        in_dtype=BSE_C64 if c128 == torch.complex64 else BSE_C128)


def bse_build_kernel(problems: Sequence[bse_problem], precision: int = BSE_PREC_FP64,
                     stream=None) -> None:
    lib = load()
    arr = (bse_problem * len(problems))(*problems)
    _check(lib.bse_build_kernel(arr, len(problems), int(precision), _stream(stream)))


def bse_build_kernel_fp64_static(problem: bse_problem, stream=None) -> None:
    """FP64 build of one problem using the library's fixed 16 MiB scratch array
    instead of allocating device memory (for callers that cannot allocate)."""
    lib = load()
    _check(lib.bse_build_kernel_fp64_static(ctypes.byref(problem), _stream(stream)))


def bse_reduce(n: int, A, B, S, L, stream=None) -> int:
    """A-B = L L^H, S = L^H (A+B) L.  B may be None (TDA).  Returns 0 or raises
    BSEError (status BSE_ERR_NOT_PD carries the failing minor in .minor)."""
    lib = load()
    a, ld = _matrix_ptr(A, n, "A")
    b = _matrix_ptr(B, n, "B")[0] if B is not None else None
    s, _ = _matrix_ptr(S, n, "S")
    l, _ = _matrix_ptr(L, n, "L")
    minor = ctypes.c_int32(0)
    st = lib.bse_reduce(n, a, b, ld, s, l, ctypes.byref(minor), _stream(stream))
    if st != BSE_OK:
        err = BSEError(st, lib.bse_last_error().decode(errors="replace"))
        err.minor = minor.value
        raise err
    return 0


def bse_spectrum(n: int, S, L, rho, c_q: float, vc: float, omega, delta: float,
                 E_out, osc_out, eps_out, stream=None) -> None:
    import torch
    lib = load()
    s, ld = _matrix_ptr(S, n, "S")
    l, _ = _matrix_ptr(L, n, "L")
    n_omega = 0 if omega is None else omega.numel()
    _check(lib.bse_spectrum(n, s, l, ld, _ptr(rho, torch.complex128, "rho"), float(c_q),
                            float(vc), n_omega, _ptr(omega, torch.float64, "omega"),
                            float(delta), _ptr(E_out, torch.float64, "E_out"),
                            _ptr(osc_out, torch.float64, "osc_out"),
                            _ptr(eps_out, torch.complex128, "eps_out"), _stream(stream)))


def bse_spectrum_lanczos(n: int, A, B, rho, c_q: float, vc: float, omega, delta: float, eps_out,
                         tol: float = 1e-8, max_steps: int = 4000,
                         matvec_precision: int = BSE_PREC_FP64, stream=None) -> int:
    """eps on the grid by the Lanczos recursion on (A-B)(A+B) (no reduction,
    no eigensolve); returns the steps taken.  On BSE_ERR_NO_CONV the raised
    error carries .steps and eps_out holds the last estimate."""
    import torch
    lib = load()
    a, ld = _matrix_ptr(A, n, "A")
    b = _matrix_ptr(B, n, "B")[0] if B is not None else None
    steps = ctypes.c_int32(0)
    st = lib.bse_spectrum_lanczos(n, a, b, ld, _ptr(rho, torch.complex128, "rho"), float(c_q),
                                  float(vc), omega.numel(), _ptr(omega, torch.float64, "omega"),
                                  float(delta), float(tol), int(max_steps), int(matvec_precision),
                                  _ptr(eps_out, torch.complex128, "eps_out"), ctypes.byref(steps),
                                  _stream(stream))
    if st != BSE_OK:
        err = BSEError(st, lib.bse_last_error().decode(errors="replace"))
        err.steps = steps.value
        raise err
    return steps.value


def bse_spectrum_tensor(n: int, Z, L, D, c_q: float, vc: float, omega, delta: float, E,
                        eps_out, stream=None) -> None:
    """Cartesian dielectric tensor eps_out [n_omega, 3, 3] from bse_spectrum's
    eigenvectors Z (its S after the call), L and energies E; D [3, n] holds the
    three directions' matrix elements (row i = direction i)."""
    import torch
    lib = load()
    z, ld = _matrix_ptr(Z, n, "Z")
    l, _ = _matrix_ptr(L, n, "L")
    if tuple(D.shape) != (3, n) or not D.is_contiguous():
        raise ValueError("D must be a contiguous [3, n] tensor")
    n_omega = omega.numel()
    if tuple(eps_out.shape) != (n_omega, 3, 3) or not eps_out.is_contiguous():
        raise ValueError("eps_out must be a contiguous [n_omega, 3, 3] tensor")
    _check(lib.bse_spectrum_tensor(n, z, l, ld, _ptr(D, torch.complex128, "D"), n, float(c_q),
                                   float(vc), n_omega, _ptr(omega, torch.float64, "omega"),
                                   float(delta), _ptr(E, torch.float64, "E"),
                                   _ptr(eps_out, torch.complex128, "eps_out"), _stream(stream)))


def bse_loss_function(eps, v_inv: float, loss_out=None, sqw_out=None, stream=None) -> None:
    """Loss function -Im 1/eps and S(Q, w) = v_inv L / pi for eps [n_omega]."""
    import torch
    _check(load().bse_loss_function(eps.numel(), _ptr(eps, torch.complex128, "eps"), float(v_inv),
                                    _ptr(loss_out, torch.float64, "loss_out"),
                                    _ptr(sqw_out, torch.float64, "sqw_out"), _stream(stream)))


def bse_lowest_excitons(n: int, A, B, nev: int, E_out, XpY_out=None, tol_ev: float = 1e-4,
                        max_iter: int = 100, precond: int = 0, mlp=None, stream=None,
                        matvec_precision: int = BSE_PREC_FP64, start=None) -> int:
    """Lowest nev excitons by block Davidson; returns the iterations used.  On
    BSE_ERR_NO_CONV the raised error carries .iters.  start: optional [k0, n]
    complex128 CUDA tensor (column-major n x k0, e.g. the X+Y found at a
    neighbouring Q) that seeds the basis (bse_lowest_excitons_from)."""
    import torch
    lib = load()
    a, ld = _matrix_ptr(A, n, "A")
    b = _matrix_ptr(B, n, "B")[0] if B is not None else None
    x = None
    if XpY_out is not None:
        if XpY_out.shape != (nev, n):
            raise ValueError("XpY_out must have shape [nev, n] (column-major n x nev)")
        x = _ptr(XpY_out, torch.complex128, "XpY_out")
    iters = ctypes.c_int32(0)
    handle = mlp.handle if mlp is not None else None
    if start is None:
        st = lib.bse_lowest_excitons(n, a, b, ld, nev, float(tol_ev), int(max_iter), int(precond),
                                     handle, int(matvec_precision),
                                     _ptr(E_out, torch.float64, "E_out"), x, ctypes.byref(iters),
                                     _stream(stream))
    else:
        if start.dim() != 2 or start.shape[1] != n:
            raise ValueError("start must have shape [k0, n] (column-major n x k0)")
        st = lib.bse_lowest_excitons_from(n, a, b, ld, nev, float(tol_ev), int(max_iter),
                                          int(precond), handle, int(matvec_precision),
                                          _ptr(start, torch.complex128, "start"), start.shape[0],
                                          _ptr(E_out, torch.float64, "E_out"), x,
                                          ctypes.byref(iters), _stream(stream))
    if st != BSE_OK:
        err = BSEError(st, lib.bse_last_error().decode(errors="replace"))
        err.iters = iters.value
        raise err
    return iters.value


def exciton_bands(problems: Sequence[tuple], nev: int, tol_ev: float = 1e-4, max_iter: int = 200,
                  matvec_precision: int = BSE_PREC_FP64, warm: bool = True, stream=None):
    """Lowest nev exciton energies along a line of momentum transfers: problems
    is a sequence of (n, A, B) built for consecutive Q (same n and transition
    order).  Each Q after the first starts Davidson from the X+Y found at the
    previous one (warm=False: from unit vectors).  Returns (E [nQ, nev] host
    numpy array, iterations per Q)."""
    import torch
    out, iters, prev = [], [], None
    for n, A, B in problems:
        E = torch.empty(nev, dtype=torch.float64, device=A.device)
        X = torch.empty((nev, n), dtype=torch.complex128, device=A.device)
        it = bse_lowest_excitons(n, A, B, nev, E, X, tol_ev=tol_ev, max_iter=max_iter,
                                 matvec_precision=matvec_precision, stream=stream,
                                 start=prev if warm else None)
        out.append(E.cpu().numpy())
        iters.append(it)
        prev = X
    return np.stack(out), iters


def bse_rpa_screening(e_v, e_c_kq, m, v, omega_cell: float, w_out, stream=None,
                      precision: int = BSE_PREC_FP64) -> None:
    """Static RPA screened interaction w = v eps^-1 for one q (include/bse.h):
    e_v [nk, nv], e_c_kq [nk, nc] float64, m [nk, nv, nc, ng] complex128,
    v [ng] float64, w_out [ng, ng] complex128 (row-major), CUDA tensors;
    precision of the polarisability contraction (FP64 or a tensor-core split)."""
    import torch
    nk, nv, nc, ng = m.shape
    if tuple(e_v.shape) != (nk, nv) or tuple(e_c_kq.shape) != (nk, nc) or tuple(v.shape) != (ng,):
        raise ValueError("e_v [nk, nv], e_c_kq [nk, nc] and v [ng] must match m [nk, nv, nc, ng]")
    if tuple(w_out.shape) != (ng, ng):
        raise ValueError("w_out must have shape [ng, ng]")
    f64, c128 = torch.float64, torch.complex128
    _check(load().bse_rpa_screening(nk, nv, nc, ng, float(omega_cell), _ptr(e_v, f64, "e_v"),
                                    _ptr(e_c_kq, f64, "e_c_kq"), _ptr(m, c128, "m"),
                                    _ptr(v, f64, "v"), int(precision), _ptr(w_out, c128, "w_out"),
                                    _stream(stream)))


def bse_pair_elements(grid: int, cv, cc, basis, gout, m_x=None, m_vv=None, m_cc=None, n_vc=None,
                      k_begin: int = 0, k_count: int = 0, stream=None) -> None:
    """Pair matrix elements from plane-wave coefficients (include/bse.h):
    cv [nk, nv, npw], cc [nk, nc, npw] complex128 CUDA tensors; basis [npw, 3]
    and gout [ng, 3] integer coordinates (host, any integer array); outputs
    complex128 CUDA tensors of the bse_problem shapes, or None."""
    import torch
    nk, nv, npw = cv.shape
    nc = cc.shape[1]
    b = np.ascontiguousarray(basis, np.int32)
    g = np.ascontiguousarray(gout, np.int32)
    ng = g.shape[0]
    if nk != grid ** 3 or tuple(cc.shape) != (nk, nc, npw) or b.shape != (npw, 3) or g.shape[1] != 3:
        raise ValueError("cv [nk, nv, npw], cc [nk, nc, npw], basis [npw, 3], gout [ng, 3], nk = grid^3")
    kn = k_count if k_count > 0 else nk
    shapes = {"m_x": (nk, nv, nc, ng), "m_vv": (kn, nk, nv, nv, ng), "m_cc": (kn, nk, nc, nc, ng),
              "n_vc": (nk, nk, nv, nc, ng)}
    outs = {"m_x": m_x, "m_vv": m_vv, "m_cc": m_cc, "n_vc": n_vc}
    for name, t in outs.items():
        if t is not None and tuple(t.shape) != shapes[name]:
            raise ValueError(f"{name} must have shape {shapes[name]}")
    c128 = torch.complex128
    ptr = lambda t, name: _ptr(t, c128, name) if t is not None else None
    _check(load().bse_pair_elements(
        grid, nv, nc, npw, ng, _ptr(cv, c128, "cv"), _ptr(cc, c128, "cc"),
        b.ctypes.data_as(ctypes.c_void_p), g.ctypes.data_as(ctypes.c_void_p), int(k_begin),
        int(k_count), ptr(m_x, "m_x"), ptr(m_vv, "m_vv"), ptr(m_cc, "m_cc"), ptr(n_vc, "n_vc"),
        _stream(stream)))


def bse_phase_timing(enable: bool) -> None:
    load().bse_phase_timing(1 if enable else 0)


def bse_phase_report() -> Dict[str, tuple]:
    """{phase: (launches, total_ms)} since the last report; clears the record."""
    buf = ctypes.create_string_buffer(1 << 16)
    n = load().bse_phase_report(buf, len(buf))
    if n < 0:
        _check(n)
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def bse_xpy(n: int, k: int, Z, L, E, XpY_out, stream=None) -> None:
    """X+Y = L Z E^-1/2 for the first k eigenvectors (XpY_out [k, n] CUDA complex128)."""
    import torch
    z, ld = _matrix_ptr(Z, n, "Z")
    l, _ = _matrix_ptr(L, n, "L")
    if XpY_out.shape != (k, n):
        raise ValueError("XpY_out must have shape [k, n]")
    _check(load().bse_xpy(n, k, z, l, ld, _ptr(E, torch.float64, "E"),
                          _ptr(XpY_out, torch.complex128, "XpY_out"), _stream(stream)))


def bse_kernel_launches() -> int:
    return int(load().bse_kernel_launches())


def upload_problem(p: Dict, device="cuda", ld: Optional[int] = None, pin: bool = False,
                   complex_dtype=None) -> Dict:
    """Copy a bse_inputs problem (numpy arrays, or torch tensors already on a
    device) to contiguous CUDA tensors and allocate A, B [n, ld].
    complex_dtype = torch.complex64 stores m_x, m_vv, m_cc, n_vc and w as
    complex64 (BSE_C64; make_problem_struct sets in_dtype from it)."""
    import torch
    ct = complex_dtype or torch.complex128
    cn = np.complex64 if ct == torch.complex64 else np.complex128

    def dev(x, npt, tt):
        if isinstance(x, torch.Tensor):
            return x.to(device=device, dtype=tt).contiguous()
        return torch.as_tensor(np.ascontiguousarray(x, npt)).to(device)

    out = {}
    for k in ("e_v", "e_c", "v_bar"):
        out[k] = dev(p[k], np.float64, torch.float64)
    for k in ("m_x", "m_vv", "m_cc", "n_vc", "w"):
        out[k] = dev(p[k], cn, ct)
    for k in ("q_minus", "q_plus"):
        out[k] = dev(p[k], np.int32, torch.int32)
    for k in ("nk", "nv", "nc", "ng"):
        out[k] = int(p[k])
    out["omega_cell"] = float(p["omega_cell"])
    n = out["nk"] * out["nv"] * out["nc"]
    ld = ld or n
    out["A"] = torch.zeros((n, ld), dtype=torch.complex128, device=device)
    out["B"] = torch.zeros((n, ld), dtype=torch.complex128, device=device)
    return out


def matrix_to_numpy(t, n: int) -> np.ndarray:
    """Column-major [n, ld] tensor -> numpy N x N (row i, column j)."""
    return t[:, :n].cpu().numpy().T.copy()


def mixed_available() -> bool:
    """True when this library serves the split-precision tensor-core build."""
    return bool(load().bse_precision_supported(BSE_PREC_BF16X6))


class MLP:
    """Handle of the learned Davidson preconditioner (bse_mlp_* in include/bse.h)."""

    def __init__(self, seed: int = 1, n_features: int = 4, hidden: int = 128):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.bse_mlp_create(ctypes.byref(h), n_features, hidden, seed))
        self.handle = h
        self.n_features = n_features
        self.num_params = int(lib.bse_mlp_num_params(h))
        self._nbr = None

    def set_neighbours(self, nbr, stream=None) -> None:
        """The 10-feature set's neighbouring-Q X+Y: a CUDA complex128 tensor
        [count, nev, n] (block i, exciton lambda: column-major n x nev per
        block), count 1 or 2, kept alive by this object; None clears."""
        import torch
        if nbr is None:
            _check(load().bse_mlp_set_neighbours(self.handle, 0, 0, None, 0, _stream(stream)))
            self._nbr = None
            return
        if nbr.dim() != 3:
            raise ValueError("nbr must have shape [count, nev, n]")
        nbr = nbr.contiguous()
        cnt, nev, n = nbr.shape
        _check(load().bse_mlp_set_neighbours(self.handle, n, nev,
                                             _ptr(nbr, torch.complex128, "nbr"), cnt,
                                             _stream(stream)))
        self._nbr = nbr

    def features(self, A, B, eq, lam, theta, R, X, stream=None):
        """Input features (bse_mlp_features) of the residual columns R [ncol, n]
        correcting X [ncol, n]; eq, lam int32 and theta float64 CUDA tensors of
        ncol; returns a float32 CUDA tensor [ncol n, F]."""
        import torch
        ncol, n = R.shape
        a, ld = _matrix_ptr(A, n, "A")
        b = _matrix_ptr(B, n, "B")[0] if B is not None else None
        feat = torch.empty((ncol * n, self.n_features), dtype=torch.float32, device="cuda")
        _check(load().bse_mlp_features(self.handle, n, ncol, _ptr(eq, torch.int32, "eq"),
                                       _ptr(lam, torch.int32, "lam"),
                                       _ptr(theta, torch.float64, "theta"), a, b, ld,
                                       _ptr(R, torch.complex128, "R"),
                                       _ptr(X, torch.complex128, "X"), _ptr(feat),
                                       _stream(stream)))
        return feat

    def close(self):
        if self.handle:
            load().bse_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, np.float32)
        _check(load().bse_mlp_get_params(self.handle, out.ctypes.data_as(
            ctypes.POINTER(ctypes.c_float)), self.num_params))
        return out

    def set_params(self, v: np.ndarray) -> None:
        v = np.ascontiguousarray(v, np.float32)
        _check(load().bse_mlp_set_params(self.handle, v.ctypes.data_as(
            ctypes.POINTER(ctypes.c_float)), self.num_params))

    def loss_grad(self, feat, target, weight, stream=None):
        import torch
        g = np.empty(self.num_params, np.float32)
        L = ctypes.c_double(0.0)
        _check(load().bse_mlp_loss_grad(self.handle, _ptr(feat, torch.float32, "feat"),
                                        _ptr(target, torch.float32, "target"),
                                        _ptr(weight, torch.float32, "weight"), target.numel(),
                                        ctypes.byref(L), g.ctypes.data_as(
                                            ctypes.POINTER(ctypes.c_float)), _stream(stream)))
        return L.value, g

    def train(self, feat, target, weight, steps: int, lr: float, stream=None) -> float:
        import torch
        L = ctypes.c_double(0.0)
        _check(load().bse_mlp_train(self.handle, _ptr(feat, torch.float32, "feat"),
                                    _ptr(target, torch.float32, "target"),
                                    _ptr(weight, torch.float32, "weight"), target.numel(),
                                    int(steps), float(lr), ctypes.byref(L), _stream(stream)))
        return L.value

    def predict(self, feat, out, stream=None) -> None:
        import torch
        _check(load().bse_mlp_predict(self.handle, _ptr(feat, torch.float32, "feat"),
                                      feat.shape[0], _ptr(out, torch.float32, "out"),
                                      _stream(stream)))


def bse_mlp_samples(n: int, A, B, E, XpY, noise, eps: float, stream=None):
    """Training samples (feat [2 nev n, 4], target, weight: CUDA float32 tensors)."""
    import torch
    lib = load()
    a, ld = _matrix_ptr(A, n, "A")
    b = _matrix_ptr(B, n, "B")[0] if B is not None else None
    nev = E.numel()
    if XpY.shape != (nev, n) or noise.shape != (nev, n):
        raise ValueError("XpY and noise must have shape [nev, n] (column-major n x nev)")
    ns = 2 * nev * n
    feat = torch.empty((ns, 4), dtype=torch.float32, device="cuda")
    target = torch.empty(ns, dtype=torch.float32, device="cuda")
    weight = torch.empty(ns, dtype=torch.float32, device="cuda")
    _check(lib.bse_mlp_samples(n, a, b, ld, nev, _ptr(E, torch.float64, "E"),
                               _ptr(XpY, torch.complex128, "XpY"),
                               _ptr(noise, torch.complex128, "noise"), float(eps),
                               _ptr(feat), _ptr(target), _ptr(weight), _stream(stream)))
    return feat, target, weight


def bse_mlp_trajectory_samples(n: int, A, B, E, XpY, tol_ev: float = 1e-6, max_iter: int = 60,
                               capacity: int = 1 << 20, mlp=None, start=None, stream=None):
    """Samples recorded along a diagonal-preconditioned Davidson run whose exact
    pairs (E, XpY [nev, n]) are known, with mlp's feature set (None: 4
    features) and started from start ([k0, n], None: unit vectors); returns
    (feat, target, weight) trimmed."""
    import torch
    lib = load()
    a, ld = _matrix_ptr(A, n, "A")
    b = _matrix_ptr(B, n, "B")[0] if B is not None else None
    nev = E.numel()
    if XpY.shape != (nev, n):
        raise ValueError("XpY must have shape [nev, n]")
    nf = mlp.n_features if mlp is not None else 4
    feat = torch.empty((capacity, nf), dtype=torch.float32, device="cuda")
    target = torch.empty(capacity, dtype=torch.float32, device="cuda")
    weight = torch.empty(capacity, dtype=torch.float32, device="cuda")
    cnt = ctypes.c_int64(0)
    v0, k0 = None, 0
    if start is not None:
        if start.dim() != 2 or start.shape[1] != n:
            raise ValueError("start must have shape [k0, n] (column-major n x k0)")
        v0, k0 = _ptr(start, torch.complex128, "start"), start.shape[0]
    _check(lib.bse_mlp_trajectory_samples(n, a, b, ld, nev, _ptr(E, torch.float64, "E"),
                                          _ptr(XpY, torch.complex128, "XpY"), float(tol_ev),
                                          int(max_iter), mlp.handle if mlp is not None else None,
                                          v0, k0, int(capacity), _ptr(feat), _ptr(target),
                                          _ptr(weight), ctypes.byref(cnt), _stream(stream)))
    c = cnt.value
    return feat[:c].contiguous(), target[:c].contiguous(), weight[:c].contiguous()


class Plan:
    """Batched build of several problems (bse_plan_* in include/bse.h); the
    problem structs (and the tensors behind them) must outlive the plan."""

    def __init__(self, problems: Sequence[bse_problem], precision: int = BSE_PREC_BF16X6,
                 autotune: bool = False, fused: bool = True, tc_stage2: bool = True,
                 hermitian: bool = False, fp64_diagonal: bool = False, stream=None):
        lib = load()
        self._problems = list(problems)
        arr = (bse_problem * len(self._problems))(*self._problems)
        h = ctypes.c_void_p()
        flags = ((BSE_PLAN_AUTOTUNE if autotune else 0) | (0 if fused else BSE_PLAN_UNFUSED)
                 | (0 if tc_stage2 else BSE_PLAN_CUDA_CORE_STAGE2)
                 | (BSE_PLAN_HERMITIAN if hermitian else 0)
                 | (BSE_PLAN_FP64_DIAGONAL if fp64_diagonal else 0))
        _check(lib.bse_plan_create(arr, len(self._problems), int(precision), flags,
                                   ctypes.byref(h), _stream(stream)))
        self.handle = h

    def execute(self, stream=None) -> None:
        _check(load().bse_plan_execute(self.handle, _stream(stream)))

    def status(self, stream=None) -> None:
        _check(load().bse_plan_status(self.handle, _stream(stream)))

    def set_wait_limit(self, seconds: float) -> None:
        """Clock budget of the bounded device waits of later executes."""
        _check(load().bse_plan_set_wait_limit(self.handle, float(seconds)))

    @property
    def tile_cols(self) -> int:
        return int(load().bse_plan_tile_cols(self.handle))

    @property
    def stage2_shape(self):
        """(tile width, pipeline depth) of the tensor-core stage 2, (0, 0) if none."""
        t, st = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(load().bse_plan_stage2_shape(self.handle, ctypes.byref(t), ctypes.byref(st)))
        return t.value, st.value

    @property
    def fused(self) -> bool:
        """True if the direct terms run as one fused launch."""
        return bool(load().bse_plan_fused(self.handle))

    def close(self) -> None:
        if self.handle:
            load().bse_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
