"""Thin Python binding of the libcdsigma C ABI (``include/cdsigma.h``).

Argument marshalling only: torch tensors supply device memory and the
current CUDA stream; every step of the method runs in the library's CUDA
kernels.  There is no CPU fallback: if the library is missing or no GPU is
present the calls raise.

Function names are those of the C entry points.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcdsigma.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "cdsigma.h")

CDS_OK = 0
STATUS_NAMES = {0: "CDS_OK", 1: "CDS_ERR_ARG", 2: "CDS_ERR_CUDA", 3: "CDS_ERR_NOT_PD",
                4: "CDS_ERR_RANK_CAP", 5: "CDS_ERR_NO_CONVERGENCE", 6: "CDS_ERR_WORKSPACE",
                7: "CDS_ERR_UNSUPPORTED", 8: "CDS_ERR_TIMEOUT", 9: "CDS_ERR_CAPACITY"}
SCHEMES = {"full": 0, "atomic": 1}
PRECISIONS = {"fp64": 0, "bf16x3": 2, "fp16x3": 3, "f32x2": 4}
QP_OK, QP_NO_CONVERGENCE, QP_NONFINITE = 0, 1, 2

_lib: Optional[ctypes.CDLL] = None

_i32, _f64, _sz, _vp = ctypes.c_int32, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p
_SIGNATURES = {
    "cds_version": (ctypes.c_int, []),
    "cds_errstr": (ctypes.c_char_p, [ctypes.c_int]),
    "cds_launch_count": (ctypes.c_ulonglong, []),
    "cds_eri_diag": (ctypes.c_int, [_i32, _vp, _vp, _vp, _vp]),
    "cds_eri_columns": (ctypes.c_int, [_i32, _vp, _vp, _vp, _i32, _vp, _vp]),
    "cds_cd_workspace_bytes": (_sz, [_i32]),
    "cds_cd_decompose": (ctypes.c_int, [_i32, _vp, _vp, _vp, _f64, _i32, _i32, _vp, _vp, _vp,
                                        ctypes.POINTER(_i32), ctypes.POINTER(_f64), _vp, _sz,
                                        _vp]),
    "cds_cd_decompose_static": (ctypes.c_int, [_i32, _vp, _vp, _vp, _f64, _i32, _i32, _vp, _vp,
                                               _vp, ctypes.POINTER(_i32), ctypes.POINTER(_f64),
                                               _vp]),
    "cds_cd_static_max_nbf": (ctypes.c_int, []),
    "cds_cd_to_mo_workspace_bytes": (_sz, [_i32, _i32, _i32, _i32, _i32]),
    "cds_cd_to_mo": (ctypes.c_int, [_i32, _i32, _i32, _i32, _vp, _vp, _vp, _i32, _i32, _vp, _vp,
                                    _vp, _sz, _vp]),
    "cds_sigma2_workspace_bytes": (_sz, [_i32, _i32, _i32, _i32, _i32, _i32]),
    "cds_sigma2_diag": (ctypes.c_int, [_i32, _i32, _i32, _vp, _vp, _i32, _vp, _vp, _i32, _i32,
                                       _vp, _vp, _vp, _sz, _vp]),
    "cds_qp_workspace_bytes": (_sz, [_i32, _i32, _i32, _i32, _i32]),
    "cds_qp_solve": (ctypes.c_int, [_i32, _i32, _i32, _vp, _vp, _vp, _i32, _vp, _f64, _i32, _i32,
                                    _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
}


class CdsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({errstr(status)})")


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run __graft_entry__.build() first")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def declared_symbols(header: str = HEADER) -> list[str]:
    """Every function name declared in the public header."""
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:int|size_t|const char\*|unsigned long long)\s+(cds_\w+)\s*\(",
                                 text, re.M)))


def errstr(status: int) -> str:
    return load().cds_errstr(status).decode()


def _check(status: int, where: str) -> None:
    if status != CDS_OK:
        raise CdsError(status, where)


def _dev(t: torch.Tensor, dtype: torch.dtype, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


def _p(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device: torch.device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _workspace(nbytes: int, device: torch.device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def npair(nbf: int) -> int:
    return nbf * (nbf + 1) // 2


def cds_version() -> int:
    return int(load().cds_version())


def cds_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().cds_launch_count())


def cds_eri_diag(xyz: torch.Tensor, alpha: torch.Tensor) -> torch.Tensor:
    """(rho_I|rho_I) for every product density (paper Eq. integral)."""
    lib = load()
    xyz = _dev(xyz, torch.float64, "xyz")
    alpha = _dev(alpha, torch.float64, "alpha")
    n = alpha.shape[0]
    D = torch.empty(npair(n), dtype=torch.float64, device=alpha.device)
    _check(lib.cds_eri_diag(n, _p(xyz), _p(alpha), _p(D), _stream(alpha.device)), "cds_eri_diag")
    return D


def cds_eri_columns(xyz: torch.Tensor, alpha: torch.Tensor, piv: torch.Tensor) -> torch.Tensor:
    """cols[c][I] = (rho_I|rho_piv[c]) (paper Eq. integral)."""
    lib = load()
    xyz = _dev(xyz, torch.float64, "xyz")
    alpha = _dev(alpha, torch.float64, "alpha")
    piv = _dev(piv, torch.int32, "piv")
    n = alpha.shape[0]
    cols = torch.empty((piv.shape[0], npair(n)), dtype=torch.float64, device=alpha.device)
    _check(lib.cds_eri_columns(n, _p(xyz), _p(alpha), _p(piv), piv.shape[0], _p(cols),
                               _stream(alpha.device)), "cds_eri_columns")
    return cols


def default_max_rank(nbf: int) -> int:
    return min(npair(nbf), max(6 * nbf, 512))


def cds_cd_decompose(xyz: torch.Tensor, alpha: torch.Tensor, atom: torch.Tensor, delta: float,
                     scheme: str = "full", max_rank: Optional[int] = None,
                     L_out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None):
    """Pivoted Cholesky decomposition of the ERI supermatrix (paper Sec. II.A).

    Returns (L [M, npair], piv [M] int32, D [npair] residual diagonal, delta_eff).
    ``L_out`` ([max_rank, npair] float64) and ``workspace`` may be passed to
    reuse device memory across calls."""
    lib = load()
    xyz = _dev(xyz, torch.float64, "xyz")
    alpha = _dev(alpha, torch.float64, "alpha")
    atom = _dev(atom, torch.int32, "atom")
    dev = alpha.device
    n = alpha.shape[0]
    npr = npair(n)
    if max_rank is None:
        max_rank = L_out.shape[0] if L_out is not None else default_max_rank(n)
    if L_out is None:
        L_out = torch.empty((max_rank, npr), dtype=torch.float64, device=dev)
    if L_out.shape[0] < max_rank or L_out.shape[1] != npr or not L_out.is_contiguous():
        raise ValueError("L_out must be a contiguous [max_rank, npair] float64 tensor")
    piv = torch.empty(max(max_rank, 1), dtype=torch.int32, device=dev)
    D = torch.empty(npr, dtype=torch.float64, device=dev)
    need = lib.cds_cd_workspace_bytes(n)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    M = _i32(0)
    de = _f64(0.0)
    st = lib.cds_cd_decompose(n, _p(xyz), _p(alpha), _p(atom), float(delta), SCHEMES[scheme],
                              int(max_rank), _p(L_out), _p(piv), _p(D), ctypes.byref(M),
                              ctypes.byref(de), _p(workspace), workspace.numel(), _stream(dev))
    _check(st, "cds_cd_decompose")
    return L_out[:M.value], piv[:M.value], D, de.value


def cds_cd_decompose_static(xyz: torch.Tensor, alpha: torch.Tensor, atom: torch.Tensor,
                            delta: float, scheme: str, L_out: torch.Tensor, piv_out: torch.Tensor,
                            D_out: torch.Tensor):
    """The allocation-free decomposition: outputs are caller tensors
    (L_out [max_rank, npair] float64, piv_out [max_rank] int32, D_out [npair]
    float64); the library's fixed device scratch replaces the workspace.
    Returns (M, delta_eff)."""
    lib = load()
    xyz = _dev(xyz, torch.float64, "xyz")
    alpha = _dev(alpha, torch.float64, "alpha")
    atom = _dev(atom, torch.int32, "atom")
    for t, dt, nm in ((L_out, torch.float64, "L_out"), (piv_out, torch.int32, "piv_out"),
                      (D_out, torch.float64, "D_out")):
        if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise ValueError(f"{nm} must be a contiguous CUDA {dt} tensor")
    n = alpha.shape[0]
    M = _i32(0)
    de = _f64(0.0)
    st = lib.cds_cd_decompose_static(n, _p(xyz), _p(alpha), _p(atom), float(delta),
                                     SCHEMES[scheme], int(L_out.shape[0]), _p(L_out),
                                     _p(piv_out), _p(D_out), ctypes.byref(M), ctypes.byref(de),
                                     _stream(alpha.device))
    _check(st, "cds_cd_decompose_static")
    return M.value, de.value


def cds_cd_to_mo(L: torch.Tensor, C: torch.Tensor, nocc: int, orbitals: torch.Tensor,
                 workspace: Optional[torch.Tensor] = None, precision: str = "fp64"):
    """AO->MO transform of the Cholesky vectors (paper Eq. transformation).

    precision: "fp64" or "f32x2" (float-pair arithmetic on the FP32 units).
    Returns (Lov [o, v, M], Lp [np, nmo, M])."""
    lib = load()
    L = _dev(L, torch.float64, "L")
    C = _dev(C, torch.float64, "C")
    orb = _dev(orbitals, torch.int32, "orbitals")
    dev = L.device
    nbf, nmo = C.shape
    M = L.shape[0]
    np_ = orb.shape[0]
    Lov = torch.empty((nocc, nmo - nocc, M), dtype=torch.float64, device=dev)
    Lp = torch.empty((np_, nmo, M), dtype=torch.float64, device=dev)
    need = lib.cds_cd_to_mo_workspace_bytes(nbf, nmo, nocc, M, np_)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    _check(lib.cds_cd_to_mo(nbf, nmo, nocc, M, _p(L), _p(C), _p(orb), np_, PRECISIONS[precision],
                            _p(Lov), _p(Lp), _p(workspace), workspace.numel(), _stream(dev)),
           "cds_cd_to_mo")
    return Lov, Lp


def cds_sigma2_diag(Lov: torch.Tensor, Lp: torch.Tensor, eps: torch.Tensor, nocc: int,
                    E: torch.Tensor, precision: str = "fp64",
                    workspace: Optional[torch.Tensor] = None):
    """Sigma_qq(E) and dSigma/dE for the orbitals of Lp (paper Eq. SE).

    E: [np, nE].  Returns (sigma [np, nE], dsigma [np, nE])."""
    lib = load()
    Lov = _dev(Lov, torch.float64, "Lov")
    Lp = _dev(Lp, torch.float64, "Lp")
    eps = _dev(eps, torch.float64, "eps")
    E = _dev(E, torch.float64, "E")
    dev = Lp.device
    np_, nmo, M = Lp.shape
    nE = E.shape[1]
    prec = PRECISIONS[precision]
    sig = torch.empty((np_, nE), dtype=torch.float64, device=dev)
    dsig = torch.empty((np_, nE), dtype=torch.float64, device=dev)
    need = lib.cds_sigma2_workspace_bytes(nmo, nocc, M, np_, nE, prec)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    _check(lib.cds_sigma2_diag(nmo, nocc, M, _p(Lov), _p(Lp), np_, _p(eps), _p(E), nE, prec,
                               _p(sig), _p(dsig), _p(workspace), workspace.numel(),
                               _stream(dev)), "cds_sigma2_diag")
    return sig, dsig


def cds_qp_solve(Lov: torch.Tensor, Lp: torch.Tensor, orbitals: torch.Tensor, eps: torch.Tensor,
                 nocc: int, conv: float = 1e-5, max_iter: int = 50, precision: str = "fp64",
                 workspace: Optional[torch.Tensor] = None, raise_on_nonconvergence: bool = False):
    """Newton quasiparticle solve (paper Eq. iter, Eq. ps, Eq. NR).

    Returns (omega, pole, iters, status), each [np]."""
    lib = load()
    Lov = _dev(Lov, torch.float64, "Lov")
    Lp = _dev(Lp, torch.float64, "Lp")
    orb = _dev(orbitals, torch.int32, "orbitals")
    eps = _dev(eps, torch.float64, "eps")
    dev = Lp.device
    np_, nmo, M = Lp.shape
    prec = PRECISIONS[precision]
    omega = torch.empty(np_, dtype=torch.float64, device=dev)
    pole = torch.empty(np_, dtype=torch.float64, device=dev)
    iters = torch.empty(np_, dtype=torch.int32, device=dev)
    status = torch.empty(np_, dtype=torch.int32, device=dev)
    need = lib.cds_qp_workspace_bytes(nmo, nocc, M, np_, prec)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    st = lib.cds_qp_solve(nmo, nocc, M, _p(Lov), _p(Lp), _p(orb), np_, _p(eps), float(conv),
                          int(max_iter), prec, _p(omega), _p(pole), _p(iters), _p(status),
                          _p(workspace), workspace.numel(), _stream(dev))
    if st == 5 and not raise_on_nonconvergence:
        st = CDS_OK
    _check(st, "cds_qp_solve")
    return omega, pole, iters, status
