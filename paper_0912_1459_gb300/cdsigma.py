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
PRECISIONS = {"fp64": 0, "bf16x3": 2, "fp16x3": 3, "f32x2": 4, "tf32x3": 5, "ozaki": 6}
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
    "cds_cd_decompose": (ctypes.c_int, [_i32, _vp, _vp, _vp, _f64, _i32, _i32, _i32, _vp, _vp,
                                        _vp, ctypes.POINTER(_i32), ctypes.POINTER(_f64), _vp, _sz,
                                        _vp]),
    "cds_cd_decompose_static": (ctypes.c_int, [_i32, _vp, _vp, _vp, _f64, _i32, _i32, _vp, _vp,
                                               _vp, ctypes.POINTER(_i32), ctypes.POINTER(_f64),
                                               _vp]),
    "cds_cd_static_max_nbf": (ctypes.c_int, []),
    "cds_cd_candidates": (ctypes.c_int, [_i32]),
    "cds_cd_live_pairs": (ctypes.c_int, [_i32, _vp, _i32, ctypes.POINTER(ctypes.c_int64), _vp]),
    "cds_cd_gemm_timing": (ctypes.c_int, [_i32]),
    "cds_cd_gemm_time": (ctypes.c_int, [ctypes.POINTER(_f64), ctypes.POINTER(ctypes.c_int64)]),
    "cds_cd_decompose_shells": (ctypes.c_int, [_i32, _vp, _vp, _vp, _vp, _vp, _vp, _f64, _i32, _i32,
                                               _vp, _vp, _vp, ctypes.POINTER(_i32),
                                               ctypes.POINTER(_f64), _vp, _sz, _vp]),
    "cds_cd_workspace_bytes_prec": (_sz, [_i32, _i32, _i32]),
    "cds_cd_to_mo_workspace_bytes": (_sz, [_i32, _i32, _i32, _i32, _i32]),
    "cds_cd_to_mo": (ctypes.c_int, [_i32, _i32, _i32, _i32, _vp, _vp, _vp, _i32, _i32, _vp, _vp,
                                    _vp, _sz, _vp]),
    "cds_sigma2_workspace_bytes": (_sz, [_i32, _i32, _i32, _i32, _i32, _i32]),
    "cds_sigma2_diag": (ctypes.c_int, [_i32, _i32, _i32, _vp, _vp, _i32, _vp, _vp, _i32, _i32,
                                       _vp, _vp, _vp, _sz, _vp]),
    "cds_qp_workspace_bytes": (_sz, [_i32, _i32, _i32, _i32, _i32]),
    "cds_qp_solve": (ctypes.c_int, [_i32, _i32, _i32, _vp, _vp, _vp, _i32, _vp, _f64, _i32, _i32,
                                    _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "cds_cd_stats": (ctypes.c_int, [_i32, _vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_int64), _vp]),
    "cds_cd_decompose_to_mo_workspace_bytes": (_sz, [_i32, _i32, _i32, _i32, _i32, _i32]),
    "cds_cd_decompose_to_mo": (ctypes.c_int, [_i32, _vp, _vp, _vp, _f64, _i32, _i32, _vp, _i32, _i32,
                                              _vp, _i32, _i32, _i32, _vp, _vp, _vp, ctypes.POINTER(_i32),
                                              ctypes.POINTER(_f64), _vp, _vp, _vp, _sz, _vp]),
    "cds_acd_workspace_bytes": (_sz, [_i32]),
    "cds_acd_aux_pairs": (ctypes.c_int, [_i32, _vp, _vp, _f64, _vp, _i32, ctypes.POINTER(_i32), _vp,
                                         _sz, _vp]),
    "cds_ri_workspace_bytes": (_sz, [_i32, _i32, _i32]),
    "cds_ri_factors": (ctypes.c_int, [_i32, _vp, _vp, _vp, _i32, _i32, _vp, _vp, _sz, _vp]),
    "cds_sigma2_cache_bytes": (_sz, [_i32, _i32, _i32, _i32]),
    "cds_sigma2_diag_cache": (ctypes.c_int, [_i32, _i32, _i32, _vp, _vp, _i32, _vp, _vp, _i32, _i32,
                                             _vp, _vp, _vp, _sz, _vp, _sz, _vp]),
    "cds_qp_cached_workspace_bytes": (_sz, [_i32, _i32, _i32]),
    "cds_qp_solve_cached": (ctypes.c_int, [_i32, _i32, _i32, _vp, _vp, _f64, _i32, _vp, _sz, _i32, _vp,
                                           _vp, _vp, _vp, _vp, _sz, _vp]),
    "cds_qp_solve_bracketed_cached": (ctypes.c_int, [_i32, _i32, _i32, _vp, _vp, _f64, _i32, _vp, _sz,
                                                     _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "cds_qp_solve_bracketed": (ctypes.c_int, [_i32, _i32, _i32, _vp, _vp, _vp, _i32, _vp, _f64, _i32,
                                              _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "cds_wait_check": (ctypes.c_int, [_f64, _vp, _vp]),
    "cds_mp2_workspace_bytes": (_sz, [_i32, _i32, _i32, _i32]),
    "cds_mp2_energy": (ctypes.c_int, [_i32, _i32, _i32, _vp, _vp, _i32, _vp, _vp, _vp, _sz, _vp]),
}


class CdsMol(ctypes.Structure):
    """One molecule of a batch (the C struct cds_mol)."""
    _fields_ = [("nbf", ctypes.c_int32), ("nocc", ctypes.c_int32), ("np", ctypes.c_int32),
                ("nE", ctypes.c_int32), ("max_rank", ctypes.c_int32)]


BATCH_NOFF = 10
BATCH_KEYS = ("basis", "pair", "L", "piv", "C", "eps", "orb", "E", "ov", "p")

_mp = ctypes.POINTER(CdsMol)
_SIGNATURES.update({
    "cds_batch_offsets": (ctypes.c_int, [_i32, _mp, ctypes.POINTER(ctypes.c_int64)]),
    "cds_batch_workspace_bytes": (_sz, [_i32, _mp, _i32]),
    "cds_batch_cd_decompose": (ctypes.c_int, [_i32, _mp, _vp, _vp, _vp, _f64, _i32, _i32, _vp, _vp, _vp,
                                              ctypes.POINTER(_i32), _vp, _sz, _vp]),
    "cds_batch_cd_to_mo": (ctypes.c_int, [_i32, _mp, ctypes.POINTER(_i32), _vp, _vp, _vp, _i32, _vp,
                                          _vp, _vp, _sz, _vp]),
    "cds_batch_sigma2": (ctypes.c_int, [_i32, _mp, ctypes.POINTER(_i32), _vp, _vp, _vp, _vp, _i32,
                                        _vp, _vp, _vp, _vp, _sz, _vp]),
    "cds_batch_qp_solve": (ctypes.c_int, [_i32, _mp, ctypes.POINTER(_i32), _vp, _vp, _vp, _vp, _f64,
                                          _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "cds_batch_graph_create": (ctypes.c_int, [_i32, _mp, ctypes.POINTER(_i32), _vp, _vp, _vp, _vp,
                                              _vp, _i32, _f64, _i32, _vp, _vp, _vp, _vp, _vp, _vp,
                                              _vp, _vp, _sz, ctypes.POINTER(_vp)]),
    "cds_graph_launch": (ctypes.c_int, [_vp, _vp]),
    "cds_tune_set": (ctypes.c_int, [_i32, _i32]),
    "cds_tune_get": (ctypes.c_int, [_i32]),
    "cds_graph_destroy": (ctypes.c_int, [_vp]),
})


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
                     L_out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                     precision: str = "fp64"):
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
    need = lib.cds_cd_workspace_bytes_prec(n, int(max_rank), PRECISIONS[precision])
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    M = _i32(0)
    de = _f64(0.0)
    st = lib.cds_cd_decompose(n, _p(xyz), _p(alpha), _p(atom), float(delta), SCHEMES[scheme],
                              int(max_rank), PRECISIONS[precision], _p(L_out), _p(piv), _p(D),
                              ctypes.byref(M),
                              ctypes.byref(de), _p(workspace), workspace.numel(), _stream(dev))
    _check(st, "cds_cd_decompose")
    return L_out[:M.value], piv[:M.value], D, de.value


def cds_cd_decompose_to_mo(xyz: torch.Tensor, alpha: torch.Tensor, atom: torch.Tensor,
                           delta: float, C: torch.Tensor, nocc: int, orbitals: torch.Tensor,
                           scheme: str = "full", max_rank: Optional[int] = None,
                           L_out: Optional[torch.Tensor] = None,
                           Lov_out: Optional[torch.Tensor] = None,
                           Lp_out: Optional[torch.Tensor] = None,
                           workspace: Optional[torch.Tensor] = None,
                           transform: str = "f32x2", cd_precision: str = "f32x2"):
    """Float-pair decomposition and transform in one pipelined call.

    transform: the transform's precision, "f32x2" (float pairs on the FP32
    units), "ozaki" (exact-slice tensor-core GEMMs), "tf32x3" or "bf16x3"
    (split-precision tensor-core GEMMs, for well-conditioned C only).
    cd_precision: "f32x2" (speculative float-pair passes) or "ozaki" (the
    passes on the tensor cores, 64 candidates).

    Returns (L [M, npair], piv [M], D, delta_eff, Lov [o, v, M], Lp [np, nmo, M])."""
    lib = load()
    xyz = _dev(xyz, torch.float64, "xyz")
    alpha = _dev(alpha, torch.float64, "alpha")
    atom = _dev(atom, torch.int32, "atom")
    C = _dev(C, torch.float64, "C")
    orb = _dev(orbitals, torch.int32, "orbitals")
    dev = alpha.device
    n = alpha.shape[0]
    nbf, nmo = C.shape
    if nbf != n:
        raise ValueError("C must be [nbf, nmo]")
    npr = npair(n)
    if max_rank is None:
        max_rank = L_out.shape[0] if L_out is not None else default_max_rank(n)
    if L_out is None:
        L_out = torch.empty((max_rank, npr), dtype=torch.float64, device=dev)
    np_ = orb.shape[0]
    nv = nmo - nocc
    if Lov_out is None or Lov_out.numel() < nocc * nv * max_rank:
        Lov_out = torch.empty(max(nocc * nv * max_rank, 1), dtype=torch.float64, device=dev)
    if Lp_out is None or Lp_out.numel() < np_ * nmo * max_rank:
        Lp_out = torch.empty(max(np_ * nmo * max_rank, 1), dtype=torch.float64, device=dev)
    piv = torch.empty(max(max_rank, 1), dtype=torch.int32, device=dev)
    D = torch.empty(npr, dtype=torch.float64, device=dev)
    need = lib.cds_cd_decompose_to_mo_workspace_bytes(n, nmo, nocc, max_rank, np_,
                                                      PRECISIONS[cd_precision])
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    M, de = _i32(0), _f64(0.0)
    st = lib.cds_cd_decompose_to_mo(n, _p(xyz), _p(alpha), _p(atom), float(delta),
                                    SCHEMES[scheme], int(max_rank), _p(C), nmo, nocc, _p(orb),
                                    np_, PRECISIONS[transform], PRECISIONS[cd_precision], _p(L_out),
                                    _p(piv), _p(D), ctypes.byref(M),
                                    ctypes.byref(de), _p(Lov_out), _p(Lp_out), _p(workspace),
                                    workspace.numel(), _stream(dev))
    _check(st, "cds_cd_decompose_to_mo")
    Mv = M.value
    Lov = Lov_out.view(-1)[:nocc * nv * Mv].view(nocc, nv, Mv)
    Lp = Lp_out.view(-1)[:np_ * nmo * Mv].view(np_, nmo, Mv)
    return L_out[:Mv], piv[:Mv], D, de.value, Lov, Lp


def cds_acd_aux_pairs(alpha: torch.Tensor, atom: torch.Tensor, delta: float) -> torch.Tensor:
    """Packed pair indices of the atomic Cholesky basis (Sec. II.A, atomic CD),
    as an int32 tensor on the basis' device."""
    lib = load()
    alpha = _dev(alpha, torch.float64, "alpha")
    atom = _dev(atom, torch.int32, "atom")
    dev = alpha.device
    n = alpha.shape[0]
    na = int(torch.bincount(atom.long()).max().item()) if n else 1
    ws = _workspace(lib.cds_acd_workspace_bytes(na), dev)
    cap = n * (n + 1) // 2
    out = (ctypes.c_int32 * max(cap, 1))()
    cnt = _i32(0)
    st = lib.cds_acd_aux_pairs(n, _p(alpha), _p(atom), float(delta), out, cap, ctypes.byref(cnt),
                               _p(ws), ws.numel(), _stream(dev))
    _check(st, "cds_acd_aux_pairs")
    return torch.tensor(list(out[:cnt.value]), dtype=torch.int32, device=dev)


def cds_ri_factors(xyz: torch.Tensor, alpha: torch.Tensor, aux: torch.Tensor,
                   precision: str = "fp64") -> torch.Tensor:
    """B [naux, npair]: the V-approximation (Eq. int_approx) over the basis
    densities aux, in the factor form of the Cholesky vectors.

    precision: "fp64" or "f32x2" (integrals and substitution in float pairs)."""
    lib = load()
    xyz = _dev(xyz, torch.float64, "xyz")
    alpha = _dev(alpha, torch.float64, "alpha")
    aux = _dev(aux, torch.int32, "aux")
    dev = alpha.device
    n = alpha.shape[0]
    naux = aux.shape[0]
    B = torch.empty((naux, npair(n)), dtype=torch.float64, device=dev)
    prec = PRECISIONS[precision]
    ws = _workspace(lib.cds_ri_workspace_bytes(n, naux, prec), dev)
    st = lib.cds_ri_factors(n, _p(xyz), _p(alpha), _p(aux), naux, prec, _p(B), _p(ws), ws.numel(),
                            _stream(dev))
    _check(st, "cds_ri_factors")
    return B


def cds_cd_stats(nbf: int, workspace: torch.Tensor, precision: str = "fp64") -> dict:
    """Work counters of the last decomposition run in ``workspace``: streaming
    passes, vectors streamed by them, vectors added between passes."""
    lib = load()
    p, st_, ex = _i32(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.cds_cd_stats(int(nbf), _p(workspace), PRECISIONS[precision], ctypes.byref(p),
                            ctypes.byref(st_), ctypes.byref(ex), _stream(workspace.device)),
           "cds_cd_stats")
    return {"passes": p.value, "streamed": st_.value, "extra": ex.value}


def cds_cd_decompose_shells(xyz: torch.Tensor, lmn: torch.Tensor, start: torch.Tensor,
                            exps: torch.Tensor, coefs: torch.Tensor, atom: torch.Tensor,
                            delta: float, scheme: str = "full", max_rank: Optional[int] = None):
    """The decomposition over contracted Cartesian shells (FP64).

    Returns (L [M, npair], piv [M] int32, D [npair], delta_eff)."""
    lib = load()
    xyz = _dev(xyz, torch.float64, "xyz")
    lmn = _dev(lmn, torch.int32, "lmn")
    start = _dev(start, torch.int32, "start")
    exps = _dev(exps, torch.float64, "exps")
    coefs = _dev(coefs, torch.float64, "coefs")
    atom = _dev(atom, torch.int32, "atom")
    dev = xyz.device
    n = lmn.shape[0]
    npr = npair(n)
    if max_rank is None:
        max_rank = default_max_rank(n)
    L = torch.empty((max(max_rank, 1), npr), dtype=torch.float64, device=dev)
    piv = torch.empty(max(max_rank, 1), dtype=torch.int32, device=dev)
    D = torch.empty(npr, dtype=torch.float64, device=dev)
    ws = _workspace(lib.cds_cd_workspace_bytes(n), dev)
    M, de = _i32(0), _f64(0.0)
    st = lib.cds_cd_decompose_shells(n, _p(xyz), _p(lmn), _p(start), _p(exps), _p(coefs),
                                     _p(atom), float(delta), SCHEMES[scheme], int(max_rank),
                                     _p(L), _p(piv), _p(D), ctypes.byref(M), ctypes.byref(de),
                                     _p(ws), ws.numel(), _stream(dev))
    _check(st, "cds_cd_decompose_shells")
    return L[:M.value], piv[:M.value], D, de.value


def cds_cd_gemm_timing(enable: bool) -> None:
    """Switch the event timing of the OZAKI decomposition's projection GEMM
    (every launch, on its stream) and clear its totals."""
    _check(load().cds_cd_gemm_timing(1 if enable else 0), "cds_cd_gemm_timing")


def cds_cd_gemm_time() -> tuple[float, int]:
    """(milliseconds summed, launches) of the GEMM since timing was switched."""
    ms, n = _f64(0.0), ctypes.c_int64(0)
    _check(load().cds_cd_gemm_time(ctypes.byref(ms), ctypes.byref(n)), "cds_cd_gemm_time")
    return ms.value, n.value


def cds_cd_live_pairs(nbf: int, workspace: torch.Tensor, precision: str = "ozaki") -> int:
    """Pairs the last decomposition in ``workspace`` kept after screening."""
    n = ctypes.c_int64(0)
    _check(load().cds_cd_live_pairs(nbf, _p(workspace), PRECISIONS[precision], ctypes.byref(n),
                                    _stream(workspace.device)), "cds_cd_live_pairs")
    return n.value


def cd_candidates(precision: str = "f32x2") -> int:
    """Candidate pivots per streaming pass of the decomposition's precision."""
    return int(load().cds_cd_candidates(PRECISIONS[precision]))


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

    precision: "fp64", "f32x2" (float-pair arithmetic on the FP32 units),
    "ozaki" (exact-slice tcgen05 GEMMs, nbf <= 1040), or "tf32x3" / "bf16x3"
    (split-precision tcgen05 GEMMs, for well-conditioned C only).
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


def cds_qp_solve_bracketed(Lov: torch.Tensor, Lp: torch.Tensor, orbitals: torch.Tensor,
                           eps: torch.Tensor, nocc: int, conv: float = 1e-5, max_iter: int = 100,
                           precision: str = "fp64", workspace: Optional[torch.Tensor] = None,
                           raise_on_nonconvergence: bool = False):
    """Safeguarded Newton inside the pole-free interval around each e_q, Sigma
    recomputed from the factors.  Returns (omega, pole, iters, status, bracket [np, 2])."""
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
    bracket = torch.empty((np_, 2), dtype=torch.float64, device=dev)
    need = lib.cds_qp_workspace_bytes(nmo, nocc, M, np_, prec)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    st = lib.cds_qp_solve_bracketed(nmo, nocc, M, _p(Lov), _p(Lp), _p(orb), np_, _p(eps),
                                    float(conv), int(max_iter), prec, _p(omega), _p(pole),
                                    _p(iters), _p(status), _p(bracket), _p(workspace),
                                    workspace.numel(), _stream(dev))
    if st == 5 and not raise_on_nonconvergence:
        st = CDS_OK
    _check(st, "cds_qp_solve_bracketed")
    return omega, pole, iters, status, bracket


def cds_wait_check(seconds: float = 0.05, device: Optional[torch.device] = None) -> int:
    """Run the tensor-core kernels' bounded wait on a barrier nothing completes;
    returns the status word it leaves (CDS_ERR_TIMEOUT = 8 when it gave up)."""
    lib = load()
    dev = device or torch.device("cuda", torch.cuda.current_device())
    err = torch.full((1,), -1, dtype=torch.int32, device=dev)
    return int(lib.cds_wait_check(float(seconds), _p(err), _stream(dev)))


def cds_sigma2_diag_cache(Lov: torch.Tensor, Lp: torch.Tensor, eps: torch.Tensor, nocc: int,
                          E: torch.Tensor, precision: str = "bf16x3",
                          cache: Optional[torch.Tensor] = None,
                          workspace: Optional[torch.Tensor] = None):
    """cds_sigma2_diag that also keeps every work item's numerators.

    Returns (sigma, dsigma, cache); pass the cache to cds_qp_solve_cached."""
    lib = load()
    Lov = _dev(Lov, torch.float64, "Lov")
    Lp = _dev(Lp, torch.float64, "Lp")
    eps = _dev(eps, torch.float64, "eps")
    E = _dev(E, torch.float64, "E")
    dev = Lp.device
    np_, nmo, M = Lp.shape
    nE = E.shape[1]
    prec = PRECISIONS[precision]
    sigma = torch.empty((np_, nE), dtype=torch.float64, device=dev)
    dsigma = torch.empty((np_, nE), dtype=torch.float64, device=dev)
    cb = lib.cds_sigma2_cache_bytes(nmo, nocc, np_, prec)
    if cache is None or cache.numel() < cb:
        cache = torch.empty(max(cb, 1), dtype=torch.uint8, device=dev)
    need = lib.cds_sigma2_workspace_bytes(nmo, nocc, M, np_, nE, prec)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    st = lib.cds_sigma2_diag_cache(nmo, nocc, M, _p(Lov), _p(Lp), np_, _p(eps), _p(E), nE, prec,
                                   _p(sigma), _p(dsigma), _p(cache), cache.numel(),
                                   _p(workspace), workspace.numel(), _stream(dev))
    _check(st, "cds_sigma2_diag_cache")
    return sigma, dsigma, cache


def cds_qp_solve_cached(cache: torch.Tensor, orbitals: torch.Tensor, eps: torch.Tensor, nmo: int,
                        nocc: int, conv: float = 1e-5, max_iter: int = 50,
                        workspace: Optional[torch.Tensor] = None,
                        raise_on_nonconvergence: bool = False, precision: str = "bf16x3"):
    """Newton quasiparticle solve (Eq. iter, Eq. ps, Eq. NR) with Sigma from the
    numerators cds_sigma2_diag_cache stored (in `precision`, the cache's form).
    Returns (omega, pole, iters, status)."""
    lib = load()
    orb = _dev(orbitals, torch.int32, "orbitals")
    eps = _dev(eps, torch.float64, "eps")
    dev = orb.device
    np_ = orb.shape[0]
    omega = torch.empty(np_, dtype=torch.float64, device=dev)
    pole = torch.empty(np_, dtype=torch.float64, device=dev)
    iters = torch.empty(np_, dtype=torch.int32, device=dev)
    status = torch.empty(np_, dtype=torch.int32, device=dev)
    need = lib.cds_qp_cached_workspace_bytes(nmo, nocc, np_)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    st = lib.cds_qp_solve_cached(nmo, nocc, np_, _p(orb), _p(eps), float(conv), int(max_iter),
                                 _p(cache), cache.numel(), PRECISIONS[precision], _p(omega),
                                 _p(pole), _p(iters),
                                 _p(status), _p(workspace), workspace.numel(), _stream(dev))
    if st == 5 and not raise_on_nonconvergence:
        st = CDS_OK
    _check(st, "cds_qp_solve_cached")
    return omega, pole, iters, status


def cds_qp_solve_bracketed_cached(cache: torch.Tensor, orbitals: torch.Tensor, eps: torch.Tensor,
                                  nmo: int, nocc: int, conv: float = 1e-5, max_iter: int = 100,
                                  workspace: Optional[torch.Tensor] = None,
                                  raise_on_nonconvergence: bool = False,
                                  precision: str = "bf16x3"):
    """Safeguarded Newton inside the pole-free interval around each e_q, Sigma
    from cached numerators.  Returns (omega, pole, iters, status, bracket [np, 2])."""
    lib = load()
    orb = _dev(orbitals, torch.int32, "orbitals")
    eps = _dev(eps, torch.float64, "eps")
    dev = orb.device
    np_ = orb.shape[0]
    omega = torch.empty(np_, dtype=torch.float64, device=dev)
    pole = torch.empty(np_, dtype=torch.float64, device=dev)
    iters = torch.empty(np_, dtype=torch.int32, device=dev)
    status = torch.empty(np_, dtype=torch.int32, device=dev)
    bracket = torch.empty((np_, 2), dtype=torch.float64, device=dev)
    need = lib.cds_qp_cached_workspace_bytes(nmo, nocc, np_)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    st = lib.cds_qp_solve_bracketed_cached(nmo, nocc, np_, _p(orb), _p(eps), float(conv),
                                           int(max_iter), _p(cache), cache.numel(),
                                           PRECISIONS[precision], _p(omega),
                                           _p(pole), _p(iters), _p(status), _p(bracket),
                                           _p(workspace), workspace.numel(), _stream(dev))
    if st == 5 and not raise_on_nonconvergence:
        st = CDS_OK
    _check(st, "cds_qp_solve_bracketed_cached")
    return omega, pole, iters, status, bracket


def cds_mp2_energy(Lov: torch.Tensor, eps: torch.Tensor, nocc: int, precision: str = "fp64",
                   workspace: Optional[torch.Tensor] = None):
    """MP2 correlation energy (paper Eq. MP2) from the factors.

    Returns (e_total [1], e_pair [nocc]) as device tensors: e_pair[i] is the
    sum over j, a, b for occupied i."""
    lib = load()
    Lov = _dev(Lov, torch.float64, "Lov")
    eps = _dev(eps, torch.float64, "eps")
    dev = Lov.device
    o, v, M = Lov.shape
    if o != nocc:
        raise ValueError("Lov must be [nocc, nvirt, M]")
    nmo = nocc + v
    prec = PRECISIONS[precision]
    e_total = torch.empty(1, dtype=torch.float64, device=dev)
    e_pair = torch.empty(max(nocc, 1), dtype=torch.float64, device=dev)
    need = lib.cds_mp2_workspace_bytes(nmo, nocc, M, prec)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    st = lib.cds_mp2_energy(nmo, nocc, M, _p(Lov), _p(eps), prec, _p(e_pair), _p(e_total),
                            _p(workspace), workspace.numel(), _stream(dev))
    _check(st, "cds_mp2_energy")
    return e_total, e_pair[:nocc]


# ---------------------------------------------------------------------------
# batched form
# ---------------------------------------------------------------------------
class Batch:
    """A batch of molecules in concatenated device buffers (cds_mol layout).

    ``mols``: list of (nbf, nocc, np, nE, max_rank).  Holds the offsets, the
    workspace and the output buffers; the methods call the cds_batch_* entry
    points and return per-molecule views.  ``cd_precision="ozaki"`` sizes the
    workspace for the tensor-core decomposition of every molecule."""

    def __init__(self, mols, device, precision: str = "bf16x3", cd_precision: str = "f32x2"):
        self.lib = load()
        self.dev = torch.device(device)
        self.n = len(mols)
        self.mols = (CdsMol * self.n)(*[CdsMol(*m) for m in mols])
        offs = (ctypes.c_int64 * ((self.n + 1) * BATCH_NOFF))()
        _check(self.lib.cds_batch_offsets(self.n, self.mols, offs), "cds_batch_offsets")
        o = list(offs)
        self.off = [dict(zip(BATCH_KEYS, o[i * BATCH_NOFF:(i + 1) * BATCH_NOFF]))
                    for i in range(self.n + 1)]
        self.total = self.off[self.n]
        self.prec = precision
        need = self.lib.cds_batch_workspace_bytes(self.n, self.mols, PRECISIONS[precision])
        if cd_precision == "ozaki":
            need = max(need, self.lib.cds_batch_workspace_bytes(self.n, self.mols,
                                                                PRECISIONS["ozaki"]))
        self.ws = _workspace(need, self.dev)
        f64 = dict(dtype=torch.float64, device=self.dev)
        i32 = dict(dtype=torch.int32, device=self.dev)
        t = self.total
        self.L = torch.empty(max(t["L"], 1), **f64)
        self.piv = torch.empty(max(t["piv"], 1), **i32)
        self.D = torch.empty(max(t["pair"], 1), **f64)
        self.Lov = torch.zeros(max(t["ov"], 1), **f64)
        self.Lp = torch.zeros(max(t["p"], 1), **f64)
        self.sigma = torch.empty(max(t["E"], 1), **f64)
        self.dsigma = torch.empty(max(t["E"], 1), **f64)
        self.omega = torch.empty(max(t["orb"], 1), **f64)
        self.pole = torch.empty(max(t["orb"], 1), **f64)
        self.iters = torch.empty(max(t["orb"], 1), **i32)
        self.status = torch.empty(max(t["orb"], 1), **i32)
        self.stamps = torch.zeros(self.n + 1, dtype=torch.int64, device=self.dev)
        self.M = (_i32 * self.n)()

    def _s(self):
        return _stream(self.dev)

    def cd_decompose(self, xyz, alpha, atom, delta, scheme="full", precision="fp64"):
        st = self.lib.cds_batch_cd_decompose(self.n, self.mols, _p(xyz), _p(alpha), _p(atom),
                                             float(delta), SCHEMES[scheme], PRECISIONS[precision],
                                             _p(self.L), _p(self.piv),
                                             _p(self.D), self.M, _p(self.ws), self.ws.numel(),
                                             self._s())
        _check(st, "cds_batch_cd_decompose")
        return list(self.M)

    def cd_to_mo(self, C, orb, precision="f32x2"):
        _check(self.lib.cds_batch_cd_to_mo(self.n, self.mols, self.M, _p(self.L), _p(C), _p(orb),
                                           PRECISIONS[precision], _p(self.Lov), _p(self.Lp),
                                           _p(self.ws), self.ws.numel(), self._s()),
               "cds_batch_cd_to_mo")

    def sigma2(self, eps, E):
        _check(self.lib.cds_batch_sigma2(self.n, self.mols, self.M, _p(self.Lov), _p(self.Lp), _p(eps),
                                         _p(E), PRECISIONS[self.prec], _p(self.sigma), _p(self.dsigma),
                                         None, _p(self.ws), self.ws.numel(), self._s()),
               "cds_batch_sigma2")

    def qp_solve(self, orb, eps, conv=1e-5, max_iter=50):
        st = self.lib.cds_batch_qp_solve(self.n, self.mols, self.M, _p(self.Lov), _p(self.Lp), _p(orb),
                                         _p(eps), float(conv), int(max_iter), PRECISIONS[self.prec],
                                         _p(self.omega), _p(self.pole), _p(self.iters),
                                         _p(self.status), _p(self.stamps), _p(self.ws),
                                         self.ws.numel(), self._s())
        if st not in (CDS_OK, 5):
            _check(st, "cds_batch_qp_solve")

    def graph(self, orb, eps, E, conv=1e-5, max_iter=50):
        """Capture the Sigma-grid + Newton stage as a CUDA graph (BatchGraph)."""
        h = ctypes.c_void_p()
        st = self.lib.cds_batch_graph_create(self.n, self.mols, self.M, _p(self.Lov), _p(self.Lp),
                                             _p(orb), _p(eps), _p(E), PRECISIONS[self.prec],
                                             float(conv), int(max_iter), _p(self.sigma),
                                             _p(self.dsigma), _p(self.omega), _p(self.pole),
                                             _p(self.iters), _p(self.status), _p(self.stamps),
                                             _p(self.ws), self.ws.numel(), ctypes.byref(h))
        _check(st, "cds_batch_graph_create")
        return BatchGraph(self.lib, h, self)

    def view(self, key: str, c: int, shape):
        """Molecule c's part of a concatenated buffer."""
        buf = {"L": self.L, "piv": self.piv, "D": self.D, "ov": self.Lov, "p": self.Lp,
               "sigma": self.sigma, "dsigma": self.dsigma, "omega": self.omega, "pole": self.pole,
               "iters": self.iters, "status": self.status}[key]
        base = {"L": "L", "piv": "piv", "D": "pair", "ov": "ov", "p": "p", "sigma": "E",
                "dsigma": "E", "omega": "orb", "pole": "orb", "iters": "orb", "status": "orb"}[key]
        o = self.off[c][base]
        size = 1
        for d in shape:
            size *= d
        return buf[o:o + size].view(*shape)


class BatchGraph:
    def __init__(self, lib, handle, batch):
        self.lib, self.h, self.batch = lib, handle, batch

    def launch(self):
        _check(self.lib.cds_graph_launch(self.h, _stream(self.batch.dev)), "cds_graph_launch")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.cds_graph_destroy(self.h)
            self.h = None


TUNE_ENERGY_CHUNK, TUNE_ITEM_ORDER, TUNE_NEWTON_CACHE, TUNE_CD_GRAPH, TUNE_PIPE_SPLIT, TUNE_GRID_EC = (
    0, 1, 2, 3, 4, 5)


def cds_tune_set(knob: int, value: int) -> None:
    _check(load().cds_tune_set(knob, value), "cds_tune_set")


def cds_tune_get(knob: int) -> int:
    return int(load().cds_tune_get(knob))


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------
_SIGNATURES.update({
    "cds_qp_gradient_workspace_bytes": (_sz, [_i32, _i32, _i32, _i32, _i32]),
    "cds_qp_gradient": (ctypes.c_int, [_i32, _i32, _i32, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _i32,
                                       _vp, _vp, _vp, _vp, _sz, _vp]),
    "cds_cd_to_mo_backward_workspace_bytes": (_sz, [_i32, _i32, _i32]),
    "cds_cd_to_mo_backward": (ctypes.c_int, [_i32, _i32, _i32, _i32, _vp, _vp, _vp, _i32, _vp, _vp,
                                             _vp, _vp, _sz, _vp]),
})


def cds_qp_gradient(Lov, Lp, orbitals, eps, nocc, omega, g, precision: str = "fp64"):
    """dl/d(eps, Lov, Lp) for upstream gradients g of converged roots omega.

    precision "fp64" (FP64 CUDA cores) or "bf16x3" / "tf32x3" (tensor cores,
    FP32 accumulation)."""
    lib = load()
    Lov = _dev(Lov, torch.float64, "Lov")
    Lp = _dev(Lp, torch.float64, "Lp")
    orb = _dev(orbitals, torch.int32, "orbitals")
    eps = _dev(eps, torch.float64, "eps")
    omega = _dev(omega, torch.float64, "omega")
    g = _dev(g, torch.float64, "g")
    dev = Lp.device
    np_, nmo, M = Lp.shape
    d_eps = torch.empty(nmo, dtype=torch.float64, device=dev)
    d_Lov = torch.empty_like(Lov)
    d_Lp = torch.empty_like(Lp)
    prec = PRECISIONS[precision]
    ws = _workspace(lib.cds_qp_gradient_workspace_bytes(nmo, nocc, M, np_, prec), dev)
    _check(lib.cds_qp_gradient(nmo, nocc, M, _p(Lov), _p(Lp), _p(orb), np_, _p(eps), _p(omega),
                               _p(g), prec, _p(d_eps), _p(d_Lov), _p(d_Lp), _p(ws), ws.numel(),
                               _stream(dev)), "cds_qp_gradient")
    return d_eps, d_Lov, d_Lp


def cds_cd_to_mo_backward(L, C, nocc, orbitals, d_Lov, d_Lp):
    """dl/dC from dl/dLov and dl/dLp through the AO->MO transform."""
    lib = load()
    L = _dev(L, torch.float64, "L")
    C = _dev(C, torch.float64, "C")
    orb = _dev(orbitals, torch.int32, "orbitals")
    d_Lov = _dev(d_Lov, torch.float64, "d_Lov")
    d_Lp = _dev(d_Lp, torch.float64, "d_Lp")
    nbf, nmo = C.shape
    dC = torch.empty_like(C)
    ws = _workspace(lib.cds_cd_to_mo_backward_workspace_bytes(nbf, nmo, orb.shape[0]), C.device)
    _check(lib.cds_cd_to_mo_backward(nbf, nmo, nocc, L.shape[0], _p(L), _p(C), _p(orb), orb.shape[0],
                                     _p(d_Lov), _p(d_Lp), _p(dC), _p(ws), ws.numel(),
                                     _stream(C.device)), "cds_cd_to_mo_backward")
    return dC


class QPEnergies(torch.autograd.Function):
    """Quasiparticle energies of the given orbitals as a differentiable
    function of (eps, Lov, Lp): forward = cds_qp_solve (or the safeguarded
    cds_qp_solve_bracketed), backward = the hand-written adjoint
    (cds_qp_gradient) at the converged roots, in grad_precision (default: FP64
    after an FP64 solve, BF16X3 tensor cores after a split-precision one)."""

    @staticmethod
    def forward(ctx, eps, Lov, Lp, orbitals, nocc, conv=1e-12, max_iter=100, precision="fp64",
                bracketed=False, grad_precision=None):
        solve = cds_qp_solve_bracketed if bracketed else cds_qp_solve
        w, P, it, st = solve(Lov, Lp, orbitals, eps, nocc, conv=conv, max_iter=max_iter,
                             precision=precision)[:4]
        ctx.save_for_backward(eps, Lov, Lp, orbitals, w)
        ctx.nocc = nocc
        ctx.grad_precision = grad_precision or ("fp64" if precision == "fp64" else "bf16x3")
        ctx.mark_non_differentiable(st)
        return w, st

    @staticmethod
    def backward(ctx, gw, gst):
        eps, Lov, Lp, orbitals, w = ctx.saved_tensors
        if gw is None:
            return (None,) * 10
        d_eps, d_Lov, d_Lp = cds_qp_gradient(Lov, Lp, orbitals, eps, ctx.nocc, w, gw.contiguous(),
                                             ctx.grad_precision)
        return d_eps, d_Lov, d_Lp, None, None, None, None, None, None, None


class MOFactors(torch.autograd.Function):
    """(Lov, Lp) = cds_cd_to_mo(L, C) with the transform adjoint for dC."""

    @staticmethod
    def forward(ctx, C, L, nocc, orbitals):
        Lov, Lp = cds_cd_to_mo(L, C, nocc, orbitals)
        ctx.save_for_backward(C, L, orbitals)
        ctx.nocc = nocc
        return Lov, Lp

    @staticmethod
    def backward(ctx, g_ov, g_p):
        C, L, orbitals = ctx.saved_tensors
        g_ov = torch.zeros((ctx.nocc, C.shape[1] - ctx.nocc, L.shape[0]), dtype=torch.float64,
                           device=C.device) if g_ov is None else g_ov.contiguous()
        g_p = torch.zeros((orbitals.shape[0], C.shape[1], L.shape[0]), dtype=torch.float64,
                          device=C.device) if g_p is None else g_p.contiguous()
        return cds_cd_to_mo_backward(L, C, ctx.nocc, orbitals, g_ov, g_p), None, None, None
