"""gwas_b300: per-SNP generalized least squares on one B300 GPU.

Thin Python binding of the C ABI in include/gwas_b300.h (libgwas_b300.so).
It only marshals arguments: every step of the computation runs in the
library's CUDA kernels.  There is no CPU fallback: if the library or a CUDA
device is missing, calls raise.

Array convention (the C ABI's column-major layout):
  * a matrix with n rows is a numpy array in Fortran order, or a torch tensor
    whose first dimension has stride 1 (e.g. ``t.T`` of a contiguous tensor);
  * results b and se come back as (p, ncols) arrays in the same layout.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgwas_b300.so")

GWAS_OK = 0
ERRORS = {
    -1: "GWAS_ERR_ARG", -2: "GWAS_ERR_NOT_SPD", -3: "GWAS_ERR_CUDA", -4: "GWAS_ERR_TIMEOUT",
    -5: "GWAS_ERR_IO", -6: "GWAS_ERR_NOMEM", -7: "GWAS_ERR_UNSUPPORTED",
}
GWAS_ERR_ARG, GWAS_ERR_NOT_SPD, GWAS_ERR_CUDA, GWAS_ERR_TIMEOUT = -1, -2, -3, -4
GWAS_ERR_IO, GWAS_ERR_NOMEM, GWAS_ERR_UNSUPPORTED = -5, -6, -7
PRECISIONS = {"fp64": 0, "tf32x3": 1, "bf16x3": 2, "f16x2": 3, "sliced64": 4}
# split modes: how the solve's tiles map onto SMs (gwas_config.tile_mode)
TILE_MODES = {"auto": 0, "single": 1, "pair_mma": 3, "inverse": 4}
BUILT_PRECISIONS = ("fp64", "bf16x3", "tf32x3", "f16x2", "sliced64")
# the split precisions (tensor-core solves to the 1e-5 bar; batches take these)
SPLIT_PRECISIONS = ("bf16x3", "tf32x3", "f16x2")
SNP_OK, SNP_SINGULAR = 0, 1

# Every symbol the header declares (checked by the CPU test suite).
EXPORTS = (
    "gwas_config_default", "gwas_init", "gwas_solve_block", "gwas_solve_block_f64", "gwas_solve_stream",
    "gwas_synchronize", "gwas_set_stream", "gwas_get_info", "gwas_solve_shape", "gwas_not_spd_index", "gwas_copy_factor",
    "gwas_kernel_launches", "gwas_strerror", "gwas_last_error_detail", "gwas_destroy",
    "gwas_timing_enable", "gwas_timing_read", "gwas_solve_block_static", "gwas_adjoint_block",
    "gwas_reml_eval", "gwas_reml_fit", "gwas_batch_create", "gwas_batch_solve", "gwas_batch_synchronize",
    "gwas_batch_set_order", "gwas_batch_autotune", "gwas_batch_autotune_ex", "gwas_batch_solve_k",
    "gwas_batch_solve_files", "gwas_batch_solve_files_packed", "gwas_batch_kernel_launches",
    "gwas_batch_last_error_detail",
    "gwas_batch_destroy", "gwas_solve_file", "gwas_solve_file_out", "gwas_reader_open", "gwas_reader_next",
    "gwas_reader_release", "gwas_reader_error_detail", "gwas_reader_close", "gwas_check_timeout",
    "gwas_pack_dosages2", "gwas_h2d_bytes", "gwas_solve_stream_packed",
)
GWAS_RESUME = 1
GWAS_PACKED_INPUT = 2
STAGES = ("h2d", "trsm", "reduce", "d2h", "solve")


class GwasError(RuntimeError):
    def __init__(self, code: int, detail: str = ""):
        self.code = code
        self.name = ERRORS.get(code, f"code {code}")
        super().__init__(f"{self.name}: {detail}" if detail else self.name)


class NotSPDError(GwasError):
    def __init__(self, code, detail, index):
        super().__init__(code, detail)
        self.index = index


class _Config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("bs", ctypes.c_int), ("ring_depth", ctypes.c_int),
                ("device", ctypes.c_int), ("strip_group", ctypes.c_int), ("tile_mode", ctypes.c_int),
                ("traits", ctypes.c_int), ("separate_sums", ctypes.c_int),
                ("single_piece", ctypes.c_int), ("stream_pack", ctypes.c_int)]


_lib = None


class _Tuning(ctypes.Structure):
    _fields_ = [("cols", ctypes.c_int), ("tile_mode", ctypes.c_int), ("stages", ctypes.c_int),
                ("order", ctypes.c_int), ("strip_group", ctypes.c_int), ("snps_per_s", ctypes.c_double)]


def load(path: str | None = None):
    """Loads libgwas_b300.so (built by paper_1302_4332_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1302_4332_b300.build`")
    lib = ctypes.CDLL(path)
    vp, i64, c_int, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.gwas_config_default.argtypes = [ctypes.POINTER(_Config)]
    lib.gwas_config_default.restype = None
    lib.gwas_init.argtypes = [ctypes.POINTER(vp), c_int, c_int, vp, c_int, vp, vp, dp, dp,
                              ctypes.POINTER(_Config), vp]
    lib.gwas_init.restype = c_int
    lib.gwas_solve_block.argtypes = [vp, vp, i64, c_int, vp, vp, vp]
    lib.gwas_solve_block.restype = c_int
    lib.gwas_solve_block_f64.argtypes = [vp, vp, i64, c_int, vp, vp, vp]
    lib.gwas_solve_block_f64.restype = c_int
    lib.gwas_solve_stream.argtypes = [vp, vp, i64, i64, vp, vp, vp]
    lib.gwas_solve_stream.restype = c_int
    lib.gwas_synchronize.argtypes = [vp]
    lib.gwas_synchronize.restype = c_int
    lib.gwas_check_timeout.argtypes = [vp, c_int, c_int]
    lib.gwas_check_timeout.restype = c_int
    lib.gwas_set_stream.argtypes = [vp, vp]
    lib.gwas_set_stream.restype = c_int
    lib.gwas_get_info.argtypes = [vp] + [ctypes.POINTER(c_int)] * 5
    lib.gwas_get_info.restype = c_int
    lib.gwas_solve_shape.argtypes = [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
    lib.gwas_solve_shape.restype = c_int
    lib.gwas_not_spd_index.argtypes = [vp]
    lib.gwas_not_spd_index.restype = i64
    lib.gwas_copy_factor.argtypes = [vp, vp, i64]
    lib.gwas_copy_factor.restype = c_int
    lib.gwas_kernel_launches.argtypes = [vp]
    lib.gwas_kernel_launches.restype = i64
    lib.gwas_h2d_bytes.argtypes = [vp]
    lib.gwas_h2d_bytes.restype = i64
    lib.gwas_pack_dosages2.argtypes = [vp, i64, c_int, c_int, vp, i64]
    lib.gwas_pack_dosages2.restype = c_int
    lib.gwas_solve_stream_packed.argtypes = [vp, vp, i64, i64, vp, vp, vp]
    lib.gwas_solve_stream_packed.restype = c_int
    lib.gwas_strerror.argtypes = [c_int]
    lib.gwas_strerror.restype = ctypes.c_char_p
    lib.gwas_last_error_detail.argtypes = [vp]
    lib.gwas_last_error_detail.restype = ctypes.c_char_p
    lib.gwas_timing_enable.argtypes = [vp, c_int]
    lib.gwas_timing_enable.restype = c_int
    lib.gwas_timing_read.argtypes = [vp, ctypes.POINTER(dp), ctypes.POINTER(i64)]
    lib.gwas_timing_read.restype = c_int
    lib.gwas_solve_block_static.argtypes = [vp, vp, i64, c_int, vp, vp, vp]
    lib.gwas_solve_block_static.restype = c_int
    lib.gwas_adjoint_block.argtypes = [vp, vp, i64, c_int, vp, vp, vp, vp]
    lib.gwas_adjoint_block.restype = c_int
    lib.gwas_reml_eval.argtypes = [c_int, c_int, vp, vp, vp, dp, ctypes.POINTER(_Config), vp, ctypes.POINTER(dp)]
    lib.gwas_reml_eval.restype = c_int
    lib.gwas_reml_fit.argtypes = [c_int, c_int, vp, vp, vp, dp, dp, c_int, ctypes.POINTER(_Config), vp,
                                  ctypes.POINTER(dp), ctypes.POINTER(dp), ctypes.POINTER(c_int)]
    lib.gwas_reml_fit.restype = c_int
    P = ctypes.POINTER
    lib.gwas_batch_create.argtypes = [P(vp), P(vp), c_int, vp]
    lib.gwas_batch_create.restype = c_int
    lib.gwas_batch_solve.argtypes = [vp, P(vp), P(i64), P(c_int), P(vp), P(vp), P(vp)]
    lib.gwas_batch_solve.restype = c_int
    lib.gwas_batch_synchronize.argtypes = [vp]
    lib.gwas_batch_synchronize.restype = c_int
    lib.gwas_batch_set_order.argtypes = [vp, c_int]
    lib.gwas_batch_set_order.restype = c_int
    lib.gwas_batch_autotune.argtypes = [vp, c_int, P(c_int), P(c_int), P(dp)]
    lib.gwas_batch_autotune.restype = c_int
    lib.gwas_batch_autotune_ex.argtypes = [vp, c_int, P(_Tuning)]
    lib.gwas_batch_autotune_ex.restype = c_int
    lib.gwas_batch_solve_k.argtypes = [vp, c_int, P(vp), P(i64), P(c_int), P(vp), P(vp), P(vp)]
    lib.gwas_batch_solve_k.restype = c_int
    lib.gwas_batch_solve_files.argtypes = [vp, P(ctypes.c_char_p), P(i64), P(i64), P(i64), P(i64), c_int, P(vp),
                                           P(vp), P(vp)]
    lib.gwas_batch_solve_files.restype = c_int
    lib.gwas_batch_solve_files_packed.argtypes = lib.gwas_batch_solve_files.argtypes
    lib.gwas_batch_solve_files_packed.restype = c_int
    lib.gwas_batch_kernel_launches.argtypes = [vp]
    lib.gwas_batch_kernel_launches.restype = i64
    lib.gwas_batch_last_error_detail.argtypes = [vp]
    lib.gwas_batch_last_error_detail.restype = ctypes.c_char_p
    lib.gwas_batch_destroy.argtypes = [vp]
    lib.gwas_batch_destroy.restype = None
    lib.gwas_solve_file.argtypes = [vp, ctypes.c_char_p, i64, i64, i64, i64, vp, vp, vp]
    lib.gwas_solve_file.restype = c_int
    lib.gwas_solve_file_out.argtypes = [vp, ctypes.c_char_p, i64, i64, i64, i64, ctypes.c_char_p, c_int,
                                        ctypes.POINTER(i64)]
    lib.gwas_solve_file_out.restype = c_int
    lib.gwas_reader_open.argtypes = [P(vp), ctypes.c_char_p, i64, i64, i64, i64, c_int]
    lib.gwas_reader_open.restype = c_int
    lib.gwas_reader_next.argtypes = [vp, P(vp), P(i64), c_int]
    lib.gwas_reader_next.restype = c_int
    lib.gwas_reader_release.argtypes = [vp]
    lib.gwas_reader_release.restype = c_int
    lib.gwas_reader_error_detail.argtypes = [vp]
    lib.gwas_reader_error_detail.restype = ctypes.c_char_p
    lib.gwas_reader_close.argtypes = [vp]
    lib.gwas_reader_close.restype = None
    lib.gwas_destroy.argtypes = [vp]
    lib.gwas_destroy.restype = None
    _lib = lib
    return lib


def _host_f64(a, name):
    arr = np.asfortranarray(np.asarray(a.detach().cpu() if _is_torch(a) else a, dtype=np.float64))
    return arr


def reml_eval(phi, XL, y, h: float, bs: int = 4096):
    """REML log-likelihood of the null model, its derivative in h and s2 (GPU, FP64)."""
    lib = load()
    phi, y = _host_f64(phi, "phi"), _host_f64(y, "y")
    n = y.shape[0]
    XL = _host_f64(XL, "XL").reshape(n, -1, order="F") if XL is not None else np.zeros((n, 0), order="F")
    cfg = _Config()
    lib.gwas_config_default(ctypes.byref(cfg))
    cfg.bs = int(bs)
    out = (ctypes.c_double * 3)()
    rc = lib.gwas_reml_eval(n, XL.shape[1], phi.ctypes.data, XL.ctypes.data if XL.size else None, y.ctypes.data,
                            float(h), ctypes.byref(cfg), None, out)
    if rc != GWAS_OK:
        raise GwasError(rc, (lib.gwas_last_error_detail(None) or b"").decode())
    return out[0], out[1], out[2]


def reml_fit(phi, XL, y, h0: float = 0.2, tol: float = 1e-8, max_evals: int = 60, bs: int = 4096):
    """Gradient-based REML fit of h (GPU, FP64).  Returns (h_hat, loglik, evaluations)."""
    lib = load()
    phi, y = _host_f64(phi, "phi"), _host_f64(y, "y")
    n = y.shape[0]
    XL = _host_f64(XL, "XL").reshape(n, -1, order="F") if XL is not None else np.zeros((n, 0), order="F")
    cfg = _Config()
    lib.gwas_config_default(ctypes.byref(cfg))
    cfg.bs = int(bs)
    h = ctypes.c_double()
    ll = ctypes.c_double()
    ev = ctypes.c_int()
    rc = lib.gwas_reml_fit(n, XL.shape[1], phi.ctypes.data, XL.ctypes.data if XL.size else None, y.ctypes.data,
                           float(h0), float(tol), int(max_evals), ctypes.byref(cfg), None, ctypes.byref(h),
                           ctypes.byref(ll), ctypes.byref(ev))
    if rc != GWAS_OK:
        raise GwasError(rc, (lib.gwas_last_error_detail(None) or b"").decode())
    return h.value, ll.value, ev.value


def _torch():
    import torch
    return torch


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _colmajor(a, dtype, rows: int, name: str, allow_none=False):
    """(pointer, leading dimension, keep-alive) of a column-major matrix argument."""
    if a is None:
        if allow_none:
            return None, 0, None
        raise ValueError(f"{name} is required")
    if _is_torch(a):
        torch = _torch()
        tdt = {np.int8: torch.int8, np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if a.dtype != tdt:
            raise TypeError(f"{name} must be {tdt}, got {a.dtype}")
        if a.dim() == 1:
            a = a.reshape(-1, 1)
        if a.shape[0] != rows:
            raise ValueError(f"{name} must have {rows} rows, got {tuple(a.shape)}")
        if a.shape[1] > 1 and a.stride(0) != 1:
            raise ValueError(f"{name} must be column-major (stride 1 along rows)")
        ld = a.stride(1) if a.shape[1] > 1 else rows
        return a.data_ptr(), ld, a
    arr = np.asarray(a)
    if arr.dtype != dtype:
        arr = arr.astype(dtype)
    if arr.ndim == 1:
        arr = arr.reshape(-1, 1)
    if arr.shape[0] != rows:
        raise ValueError(f"{name} must have {rows} rows, got {arr.shape}")
    arr = np.asfortranarray(arr)
    return arr.ctypes.data, rows, arr


def pack_dosages2(X) -> np.ndarray:
    """The 2-bit encoding of gwas_solve_stream's transport (gwas_pack_dosages2):
    X n x m int8 with values 0..3 -> ceil(n/4) x m uint8 (column-major), row
    4k + i of a column in bits 2i .. 2i+1 of its byte k.  Raises GwasError
    (GWAS_ERR_ARG) for any other value."""
    x = np.asfortranarray(X, dtype=np.int8)
    if x.ndim == 1:
        x = x.reshape(-1, 1, order="F")
    n, m = x.shape
    ldp = (n + 3) // 4
    out = np.zeros((ldp, m), dtype=np.uint8, order="F")
    rc = load().gwas_pack_dosages2(x.ctypes.data, n, n, m, out.ctypes.data, ldp)
    if rc != GWAS_OK:
        raise GwasError(rc, "values outside 0..3")
    return out


def read_results(path: str):
    """A result file of GLS.solve_file_out: (header dict, b, se p x m, status m);
    b is p x m, or p x m x t for t phenotypes."""
    raw = np.fromfile(path, dtype=np.uint8)
    if raw.size < 64 or bytes(raw[:8]) != b"GWASRES\0":
        raise ValueError(f"{path}: not a result file")
    p, n, col0, m, rec, prec = (int(raw[12:16].view("<u4")[0]), int(raw[16:24].view("<u8")[0]),
                                int(raw[24:32].view("<u8")[0]), int(raw[32:40].view("<u8")[0]),
                                int(raw[40:44].view("<u4")[0]), int(raw[44:48].view("<u4")[0]))
    t = int(raw[56:64].view("<u8")[0]) or 1
    dt = np.dtype([("b", "<f8", (t, p)), ("se", "<f8", (p,)), ("status", "<i4"), ("pad", "<i4")])
    assert dt.itemsize == rec
    recs = raw[64:64 + m * rec].view(dt)
    head = dict(p=p, n=n, col0=col0, m=m, record_bytes=rec, precision=prec)
    if t > 1:
        head["traits"] = t
    b = np.asfortranarray(np.transpose(recs["b"], (2, 0, 1)))  # (p, m, t)
    return head, (b[:, :, 0].copy(order="F") if t == 1 else b), np.asfortranarray(recs["se"].T), \
        recs["status"].copy()


class GLS:
    """One study on the GPU: Listing 1's loop-invariant part at construction,
    then per-block solves.

    phi_or_L: n x n kinship Phi (or, with is_L=True, the lower factor L of M).
    XL: n x (p-1) covariates; y: n phenotypes; M = sigma2 (h Phi + (1-h) I).
    precision: "fp64", "tf32x3", "bf16x3" or "f16x2" (the inverse tile mode's
    row-scaled FP16 pieces of L^-1) for the blocked triangular solve, or
    "sliced64" (FP64-class results from exact integer products of a sliced
    M^-1 on the tensor cores; tile options do not apply).
    stream_pack: how solve_stream moves int8 host columns (-1: 2-bit codes
    packed by host threads when the CPU has AVX-512 and the solve outruns the
    int8 link, i.e. bf16x3 / f16x2 in the inverse form; 0: int8; 1: packed
    wherever the values lie in 0..3); results are identical either way.
    """

    def __init__(self, phi_or_L, XL, y, h: float, sigma2: float = 1.0, *, precision: str = "fp64",
                 bs: int = 4096, ring_depth: int = 3, is_L: bool = False, device: int = -1, stream=None,
                 strip_group: int = 0, tiles: str = "auto", separate_sums: bool = False,
                 single_piece: bool = False, stream_pack: int = -1):
        lib = load()
        n = int(np.shape(y)[0]) if not _is_torch(y) else int(y.shape[0])
        q = 0 if XL is None else (int(XL.shape[1]) if np.ndim(XL) == 2 or _is_torch(XL) else 1)
        self.n, self.p = n, q + 1
        phi_p, ldphi, self._k1 = _colmajor(phi_or_L, np.float64, n, "phi_or_L")
        if ldphi != n:
            raise ValueError("phi_or_L must be a contiguous n x n column-major matrix")
        xl_p, ldxl, self._k2 = _colmajor(XL, np.float64, n, "XL", allow_none=True) if q else (None, n, None)
        if q and ldxl != n:
            raise ValueError("XL must be contiguous with leading dimension n")
        y_p, ldy, self._k3 = _colmajor(y, np.float64, n, "y")
        self.t = int(self._k3.shape[1])  # phenotypes: y is n or n x t
        if ldy != n:
            raise ValueError("y must be contiguous with leading dimension n")
        cfg = _Config()
        lib.gwas_config_default(ctypes.byref(cfg))
        cfg.precision = PRECISIONS[precision]
        cfg.bs = int(bs)
        cfg.ring_depth = int(ring_depth)
        cfg.device = int(device)
        cfg.strip_group = int(strip_group)
        cfg.tile_mode = TILE_MODES[tiles]
        cfg.traits = self.t
        cfg.separate_sums = int(bool(separate_sums))
        cfg.single_piece = int(bool(single_piece))
        cfg.stream_pack = int(stream_pack)
        self.precision, self.bs = precision, int(bs)
        stream_p = None
        if stream is not None:
            stream_p = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        ctx = ctypes.c_void_p()
        rc = lib.gwas_init(ctypes.byref(ctx), n, self.p, phi_p, int(bool(is_L)), xl_p, y_p, float(h),
                           float(sigma2), ctypes.byref(cfg), stream_p)
        self._k1 = self._k2 = self._k3 = None
        if rc != GWAS_OK:
            detail = (lib.gwas_last_error_detail(None) or b"").decode()
            if rc == -2:
                raise NotSPDError(rc, detail, int(lib.gwas_not_spd_index(None)))
            raise GwasError(rc, detail)
        self._ctx = ctx
        info = [ctypes.c_int() for _ in range(5)]
        lib.gwas_get_info(ctx, *[ctypes.byref(i) for i in info])
        self.n_pad = info[2].value

    def solve_shape(self) -> tuple[int, int, str]:
        """(CTAs, cluster size, resolved tile mode) of the blocked triangular solve over a full block."""
        ctas, cl, mode = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(load().gwas_solve_shape(self._ctx, ctypes.byref(ctas), ctypes.byref(cl), ctypes.byref(mode)))
        names = {v: k for k, v in TILE_MODES.items()}
        return ctas.value, cl.value, names[mode.value]

    # -- helpers ---------------------------------------------------------------
    def _check(self, rc: int):
        if rc != GWAS_OK:
            detail = (load().gwas_last_error_detail(self._ctx) or b"").decode()
            raise GwasError(rc, detail)

    def _outputs(self, ncols: int, like, b, se, status):
        p, t = self.p, self.t
        if b is None:
            if _is_torch(like) and like.is_cuda:
                torch = _torch()
                b = torch.empty((t, ncols, p), dtype=torch.float64, device=like.device).permute(2, 1, 0)
                if t == 1:
                    b = b[:, :, 0]
                se = torch.empty((ncols, p), dtype=torch.float64, device=like.device).T
                status = torch.empty(ncols, dtype=torch.int32, device=like.device)
            else:
                b = np.empty((p, ncols) if t == 1 else (p, ncols, t), order="F")
                se = np.empty((p, ncols), order="F")
                status = np.empty(ncols, dtype=np.int32)
        if t > 1:  # p x ncols x t, column-major: phenotype k at + k p ncols
            strides = tuple(b.stride()) if _is_torch(b) else tuple(x // 8 for x in np.asarray(b).strides)
            if tuple(b.shape) != (p, ncols, t) or strides != (1, p, p * ncols):
                raise ValueError(f"b must be a contiguous p x ncols x t column-major array, got {tuple(b.shape)}")
            bptr = b.data_ptr() if _is_torch(b) else np.asarray(b).ctypes.data
            sp, lds, _ = _colmajor(se, np.float64, p, "se", allow_none=True)
            if sp is not None and lds != p:
                raise ValueError("se must be contiguous p x ncols column-major")
            if status is not None and not _is_torch(status):
                status = np.ascontiguousarray(status, dtype=np.int32)
            stp = None if status is None else (status.data_ptr() if _is_torch(status) else status.ctypes.data)
            return (b, se, status), (bptr, sp, stp)
        bp, ldb, _ = _colmajor(b, np.float64, p, "b")
        sp, lds, _ = _colmajor(se, np.float64, p, "se", allow_none=True)
        if ldb != p or (sp is not None and lds != p):
            raise ValueError("b and se must be contiguous p x ncols column-major")
        if status is not None and not _is_torch(status):
            status = np.ascontiguousarray(status, dtype=np.int32)
        stp = None if status is None else (status.data_ptr() if _is_torch(status) else status.ctypes.data)
        return (b, se, status), (bp, sp, stp)

    # -- the path ----------------------------------------------------------------
    def solve_block(self, XR, b=None, se=None, status=None):
        """b, se, status for the SNP columns of XR (n x ncols int8 dosages)."""
        xp, ldx, keep = _colmajor(XR, np.int8, self.n, "XR")
        ncols = int(keep.shape[1])
        outs, ptrs = self._outputs(ncols, keep, b, se, status)
        self._check(load().gwas_solve_block(self._ctx, xp, ldx, ncols, *ptrs))
        return outs

    def solve_block_f64(self, XR, b=None, se=None, status=None):
        """As solve_block with FP64 SNP values."""
        xp, ldx, keep = _colmajor(XR, np.float64, self.n, "XR")
        ncols = int(keep.shape[1])
        outs, ptrs = self._outputs(ncols, keep, b, se, status)
        self._check(load().gwas_solve_block_f64(self._ctx, xp, ldx, ncols, *ptrs))
        return outs

    def solve_stream(self, XR_host, b=None, se=None, status=None):
        """All m SNP columns of a HOST array, streamed block by block through the device ring."""
        xp, ldx, keep = _colmajor(XR_host, np.int8, self.n, "XR_host")
        if _is_torch(keep) and keep.is_cuda:
            raise ValueError("solve_stream takes host memory")
        m = int(keep.shape[1])
        if b is None:
            b = np.empty((self.p, m) if self.t == 1 else (self.p, m, self.t), order="F")
            se = np.empty((self.p, m), order="F")
            status = np.empty(m, dtype=np.int32)
        _, ptrs = self._outputs(m, keep, b, se, status)
        self._check(load().gwas_solve_stream(self._ctx, xp, ldx, m, *ptrs))
        return b, se, status

    def solve_stream_packed(self, P_host, b=None, se=None, status=None):
        """As solve_stream over 2-bit packed HOST columns (ceil(n/4) x m uint8,
        column-major, as pack_dosages2 returns them)."""
        P = P_host
        if _is_torch(P):
            if P.is_cuda:
                raise ValueError("solve_stream_packed takes host memory")
            ptr, m, ldp = P.data_ptr(), int(P.shape[1]), int(P.stride(1))
            if P.stride(0) != 1 or P.dtype != _torch().uint8:
                raise ValueError("P_host must be column-major uint8")
        else:
            P = np.asfortranarray(P, dtype=np.uint8)
            ptr, m, ldp = P.ctypes.data, int(P.shape[1]), int(P.shape[0])
        if int(P.shape[0]) < (self.n + 3) // 4:
            raise ValueError("P_host needs ceil(n/4) rows")
        if b is None:
            b = np.empty((self.p, m) if self.t == 1 else (self.p, m, self.t), order="F")
            se = np.empty((self.p, m), order="F")
            status = np.empty(m, dtype=np.int32)
        _, ptrs = self._outputs(m, P, b, se, status)
        self._check(load().gwas_solve_stream_packed(self._ctx, ptr, ldp, m, *ptrs))
        return b, se, status

    def adjoint_block(self, XR, dh_accum=None, dy_accum=None, chi2=None, dchi2_dh=None):
        """Wald chi2 per SNP and the gradient of their sum w.r.t. h and y (FP64).

        dh_accum (1 element) and dy_accum (n) are ADDED to; numpy arrays are
        created when not given.  Returns (chi2, dchi2_dh, dh_accum, dy_accum)."""
        xp, ldx, keep = _colmajor(XR, np.int8, self.n, "XR")
        ncols = int(keep.shape[1])
        on_dev = _is_torch(keep) and keep.is_cuda
        if on_dev:
            torch = _torch()
            mk = lambda k: torch.zeros(k, dtype=torch.float64, device=keep.device)
        else:
            mk = lambda k: np.zeros(k)
        chi2 = mk(ncols) if chi2 is None else chi2
        dchi2_dh = mk(ncols) if dchi2_dh is None else dchi2_dh
        dh_accum = mk(1) if dh_accum is None else dh_accum
        dy_accum = mk(self.n) if dy_accum is None else dy_accum
        ptr = lambda a: a.data_ptr() if _is_torch(a) else a.ctypes.data
        for a in (chi2, dchi2_dh, dh_accum, dy_accum):
            if (a.dtype != np.float64) if not _is_torch(a) else (str(a.dtype) != "torch.float64"):
                raise TypeError("adjoint outputs must be float64")
        self._check(load().gwas_adjoint_block(self._ctx, xp, ldx, ncols, ptr(chi2), ptr(dchi2_dh), ptr(dh_accum),
                                              ptr(dy_accum)))
        return chi2, dchi2_dh, dh_accum, dy_accum

    def solve_file(self, path: str, m: int, ldx: int | None = None, col0: int = 0, header_bytes: int = 0):
        """Columns col0 .. col0+m-1 of an n x M int8 column-major file (leading
        dimension ldx bytes, default n), streamed disk -> pinned host -> GPU."""
        b = np.empty((self.p, m) if self.t == 1 else (self.p, m, self.t), order="F")
        se = np.empty((self.p, m), order="F")
        st = np.empty(m, dtype=np.int32)
        self._check(load().gwas_solve_file(self._ctx, os.fsencode(path), int(header_bytes), int(ldx or self.n),
                                           int(col0), int(m), b.ctypes.data, se.ctypes.data, st.ctypes.data))
        return b, se, st

    def solve_file_out(self, path: str, m: int, out_path: str, ldx: int | None = None, col0: int = 0,
                       header_bytes: int = 0, resume: bool = False, packed: bool = False) -> int:
        """Columns col0 .. col0+m-1 of the dosage file, disk to disk: results
        written to out_path (read them with read_results), with a checkpoint
        beside it; resume=True continues an interrupted run; packed=True reads
        2-bit packed columns (pack_dosages2's encoding, ldx default ceil(n/4)).
        Returns the number of columns on disk."""
        done = ctypes.c_int64(0)
        ld = int(ldx or ((self.n + 3) // 4 if packed else self.n))
        flags = (GWAS_RESUME if resume else 0) | (GWAS_PACKED_INPUT if packed else 0)
        self._check(load().gwas_solve_file_out(self._ctx, os.fsencode(path), int(header_bytes), ld, int(col0),
                                               int(m), os.fsencode(out_path), flags, ctypes.byref(done)))
        return done.value

    def synchronize(self):
        self._check(load().gwas_synchronize(self._ctx))

    def check_timeout(self, kind: int = 0, limit_us: int = 20000) -> int:
        """Diagnostic: a device-side wait on something that never happens,
        bounded by limit_us; returns the library's code (GWAS_ERR_TIMEOUT is
        the expected outcome) and leaves the context usable."""
        return int(load().gwas_check_timeout(self._ctx, int(kind), int(limit_us)))

    def set_stream(self, stream):
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        self._check(load().gwas_set_stream(self._ctx, sp))

    def factor(self) -> np.ndarray:
        """The device factor L (n x n, lower) copied to the host."""
        L = np.empty((self.n, self.n), order="F")
        self._check(load().gwas_copy_factor(self._ctx, L.ctypes.data, self.n))
        return L

    def timing(self, enable: bool = True):
        """Starts (clearing) or stops the per-stage CUDA-event timers."""
        self._check(load().gwas_timing_enable(self._ctx, int(bool(enable))))

    def timing_read(self) -> dict:
        """{stage: (total ms, timed launches)} for h2d, trsm, reduce, d2h, and
        solve (the solve kernel alone, inside trsm)."""
        ms = (ctypes.c_double * len(STAGES))()
        cnt = (ctypes.c_int64 * len(STAGES))()
        self._check(load().gwas_timing_read(self._ctx, ms, cnt))
        return {name: (ms[i], int(cnt[i])) for i, name in enumerate(STAGES)}

    @property
    def kernel_launches(self) -> int:
        return int(load().gwas_kernel_launches(self._ctx))

    @property
    def h2d_bytes(self) -> int:
        """SNP-block bytes this context has copied host -> device (packed blocks count packed bytes)."""
        return int(load().gwas_h2d_bytes(self._ctx))

    def close(self):
        if getattr(self, "_ctx", None):
            load().gwas_destroy(self._ctx)
            self._ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GLSBatch:
    """The batching form: several split-precision studies (GLS objects) solved
    by one persistent tensor-core launch, replayed from a captured CUDA graph.
    The GLS objects must outlive the batch."""

    def __init__(self, studies, stream=None):
        lib = load()
        self.studies = list(studies)
        arr = (ctypes.c_void_p * len(self.studies))(*[g._ctx for g in self.studies])
        B = ctypes.c_void_p()
        sp = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        rc = lib.gwas_batch_create(ctypes.byref(B), arr, len(self.studies), sp)
        if rc != GWAS_OK:
            raise GwasError(rc, (lib.gwas_last_error_detail(None) or b"").decode())
        self._B = B

    def _check(self, rc):
        if rc != GWAS_OK:
            raise GwasError(rc, (load().gwas_batch_last_error_detail(self._B) or b"").decode())

    def solve_files(self, paths, m, cols: int, ldx=None, col0=None, header_bytes=None, packed=False):
        """Out of core: study i's columns col0[i] .. col0[i]+m[i]-1 of the n_i x M int8
        column-major file paths[i] (leading dimension ldx[i] bytes, default n_i, after
        header_bytes[i]), streamed disk -> pinned host -> batched solves of `cols`
        columns per study per step.  packed=True: the files hold 2-bit packed columns
        (pack_dosages2's encoding; ldx default ceil(n_i/4)), expanded on the GPU.
        Returns a list of (b, se, status) per study."""
        ns = len(self.studies)
        m = [int(v) for v in m]
        ldx = [int(v) for v in (ldx or [(g.n + 3) // 4 if packed else g.n for g in self.studies])]
        col0 = [int(v) for v in (col0 or [0] * ns)]
        header_bytes = [int(v) for v in (header_bytes or [0] * ns)]
        outs = [(np.empty((g.p, mi), order="F"), np.empty((g.p, mi), order="F"), np.empty(mi, dtype=np.int32))
                for g, mi in zip(self.studies, m)]
        arr = lambda t, v: (t * ns)(*v)
        fn = load().gwas_batch_solve_files_packed if packed else load().gwas_batch_solve_files
        rc = fn(
            self._B, arr(ctypes.c_char_p, [os.fsencode(p) for p in paths]), arr(ctypes.c_int64, header_bytes),
            arr(ctypes.c_int64, ldx), arr(ctypes.c_int64, col0), arr(ctypes.c_int64, m), int(cols),
            arr(ctypes.c_void_p, [o[0].ctypes.data for o in outs]), arr(ctypes.c_void_p, [o[1].ctypes.data for o in outs]),
            arr(ctypes.c_void_p, [o[2].ctypes.data for o in outs]))
        self._check(rc)
        return outs

    def solve(self, blocks):
        """blocks[i]: n_i x ncols_i int8 (column-major; None or 0 columns skips study i).
        Returns a list of (b, se, status) per study (None for skipped studies)."""
        return self.solve_k([blocks])[0]

    def solve_k(self, steps):
        """steps[j][i]: study i's block of step j; all k = len(steps) steps of
        every study in one graph replay.  Returns outs[j][i] = (b, se, status)."""
        ns, k = len(self.studies), len(steps)
        xs, lds, ncs, outs, keep = [], [], [], [], []
        for g, X in ((g, X) for blocks in steps for g, X in zip(self.studies, blocks)):
            if X is None or (hasattr(X, "shape") and X.shape[1] == 0):
                xs.append(None); lds.append(g.n); ncs.append(0); outs.append(None)
                continue
            xp, ld, xk = _colmajor(X, np.int8, g.n, "XR")
            keep.append(xk)
            nc = int(xk.shape[1])
            if _is_torch(xk) and xk.is_cuda:
                torch = _torch()
                o = (torch.empty((nc, g.p), dtype=torch.float64, device=xk.device).T,
                     torch.empty((nc, g.p), dtype=torch.float64, device=xk.device).T,
                     torch.empty(nc, dtype=torch.int32, device=xk.device))
            else:
                o = (np.empty((g.p, nc), order="F"), np.empty((g.p, nc), order="F"), np.empty(nc, dtype=np.int32))
            xs.append(xp); lds.append(ld); ncs.append(nc); outs.append(o)
        ptr = lambda a: None if a is None else (a.data_ptr() if _is_torch(a) else a.ctypes.data)
        VP = ctypes.c_void_p * (k * ns)
        rc = load().gwas_batch_solve_k(self._B, k, VP(*xs), (ctypes.c_int64 * (k * ns))(*lds),
                                       (ctypes.c_int * (k * ns))(*ncs),
                                       VP(*[ptr(o[0]) if o else None for o in outs]),
                                       VP(*[ptr(o[1]) if o else None for o in outs]),
                                       VP(*[ptr(o[2]) if o else None for o in outs]))
        self._check(rc)
        return [outs[j * ns:(j + 1) * ns] for j in range(k)]

    def synchronize(self):
        self._check(load().gwas_batch_synchronize(self._B))

    def set_order(self, mode: int):
        self._check(load().gwas_batch_set_order(self._B, int(mode)))

    def autotune(self, reps: int = 3):
        """(columns per study per launch, tile order, SNPs/s) of the fastest measured configuration."""
        t = self.autotune_ex(reps)
        return t["cols"], t["order"], t["snps_per_s"]

    def autotune_ex(self, reps: int = 3) -> dict:
        """The autotuner's choice: columns per study, tile mode, operand stages,
        tile order, strip group, and its measured rate (SNPs/s over all studies)."""
        t = _Tuning()
        self._check(load().gwas_batch_autotune_ex(self._B, int(reps), ctypes.byref(t)))
        names = {v: k for k, v in TILE_MODES.items()}
        return dict(cols=t.cols, tile_mode=names.get(t.tile_mode, t.tile_mode), stages=t.stages, order=t.order,
                    strip_group=t.strip_group, snps_per_s=t.snps_per_s)

    @property
    def kernel_launches(self) -> int:
        return int(load().gwas_batch_kernel_launches(self._B))

    def close(self):
        if getattr(self, "_B", None):
            load().gwas_batch_destroy(self._B)
            self._B = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Reader:
    """Prefetching file reader (disk -> pinned host buffers on a host thread)."""

    def __init__(self, path: str, offset: int, block_bytes: int, nblocks: int, last_bytes: int = 0, depth: int = 3):
        lib = load()
        r = ctypes.c_void_p()
        rc = lib.gwas_reader_open(ctypes.byref(r), os.fsencode(path), int(offset), int(block_bytes), int(nblocks),
                                  int(last_bytes), int(depth))
        if rc != GWAS_OK:
            raise GwasError(rc, f"cannot open {path}")
        self._r = r

    def next(self, timeout_ms: int = 120000):
        """(pointer, bytes) of the next block; valid until release()."""
        buf, nb = ctypes.c_void_p(), ctypes.c_int64()
        rc = load().gwas_reader_next(self._r, ctypes.byref(buf), ctypes.byref(nb), int(timeout_ms))
        if rc != GWAS_OK:
            raise GwasError(rc, (load().gwas_reader_error_detail(self._r) or b"").decode())
        return buf.value, nb.value

    def release(self):
        rc = load().gwas_reader_release(self._r)
        if rc != GWAS_OK:
            raise GwasError(rc, "release without a taken block")

    def close(self):
        if getattr(self, "_r", None):
            load().gwas_reader_close(self._r)
            self._r = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
