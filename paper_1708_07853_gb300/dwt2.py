"""Python binding of libdwt2.so (the C ABI in include/dwt2.h).

Argument marshalling only: tensors are passed as device pointers with the current CUDA stream;
every step of the transform runs in the library's kernels.  There is no CPU path: a missing
library or a non-CUDA tensor raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdwt2.so")

WAVELETS = {"cdf53_int": 0, "cdf53": 1, "cdf97": 2, "dd97": 3, "dd137": 4}
SCHEMES = {"nonsep": 0, "sep_fused": 1, "sep_twopass": 2, "adapted": 3, "conv": 4}
DT_I32, DT_F32, DT_BF16, DT_F16 = 0, 1, 2, 3
TORCH_DT = {torch.int32: DT_I32, torch.float32: DT_F32, torch.bfloat16: DT_BF16,
            torch.float16: DT_F16}
DT_TORCH = {v: k for k, v in TORCH_DT.items()}
ESIZE = {DT_I32: 4, DT_F32: 4, DT_BF16: 2, DT_F16: 2}
STATUS = {0: "ok", 1: "EINVAL", 2: "EUNSUPPORTED", 3: "ENOMEM", 4: "ECUDA", 5: "ETIMEOUT",
          6: "EINTERNAL"}

# Every symbol the header declares (checked by the tests without a GPU).
EXPORTS = ["dwt2_status_string", "dwt2_last_error", "dwt2_max_levels", "dwt2_layout",
           "dwt2_workspace_bytes", "dwt2_workspace_bytes_scheme", "dwt2_workspace_init",
           "dwt2_check_status", "dwt2_forward", "dwt2_forward_scheme", "dwt2_inverse",
           "dwt2_forward_static", "dwt2_forward_adjoint", "dwt2_inverse_adjoint",
           "dwt2_plan_workspace_bytes", "dwt2_plan_create", "dwt2_plan_execute", "dwt2_plan_info",
           "dwt2_plan_destroy", "dwt2_workspace_bytes_batch", "dwt2_forward_batch",
           "dwt2_inverse_batch", "dwt2_forward_adjoint_batch", "dwt2_inverse_adjoint_batch",
           "dwt2_selftest_wait_timeout"]
DIRECTIONS = {"forward": 0, "inverse": 1, "forward_adjoint": 2, "inverse_adjoint": 3}


class Dwt2Error(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = f"{what}: {STATUS.get(status, status)}"
        err = _lib().dwt2_last_error().decode()
        super().__init__(msg + (f" ({err})" if err and status in (3, 4, 6) else ""))


class ImageDesc(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("img_pitch_bytes", ctypes.c_int64),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("coeffs", ctypes.c_void_p)]


class Band(ctypes.Structure):
    _fields_ = [("offset_bytes", ctypes.c_int64), ("h", ctypes.c_int32), ("w", ctypes.c_int32),
                ("pitch_bytes", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("level", ctypes.c_int32), ("kind", ctypes.c_char),
                ("reserved", ctypes.c_char * 3)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_1708_07853_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        lib.dwt2_status_string.restype = ctypes.c_char_p
        lib.dwt2_status_string.argtypes = [i]
        lib.dwt2_last_error.restype = ctypes.c_char_p
        lib.dwt2_last_error.argtypes = []
        lib.dwt2_max_levels.argtypes = [i, i]
        lib.dwt2_layout.argtypes = [i, i, i, i, ctypes.POINTER(Band), ctypes.POINTER(sz)]
        lib.dwt2_workspace_bytes.restype = sz
        lib.dwt2_workspace_bytes.argtypes = [i, i, i, i, i]
        lib.dwt2_workspace_bytes_scheme.restype = sz
        lib.dwt2_workspace_bytes_scheme.argtypes = [i, i, i, i, i, i]
        lib.dwt2_workspace_init.argtypes = [vp, sz, vp]
        lib.dwt2_check_status.argtypes = [vp, vp]
        lib.dwt2_forward.argtypes = [vp, i64, i, i, i, vp, vp, sz, i, i, i, vp]
        lib.dwt2_forward_scheme.argtypes = [vp, i64, i, i, i, vp, vp, sz, i, i, i, i, vp]
        lib.dwt2_inverse.argtypes = [vp, vp, i64, i, i, i, vp, sz, i, i, i, vp]
        lib.dwt2_forward_static.argtypes = [vp, i64, i, i, i, vp, i, i, i, vp]
        lib.dwt2_forward_adjoint.argtypes = [vp, vp, i64, i, i, i, vp, sz, i, i, i, vp]
        pd = ctypes.POINTER(ImageDesc)
        lib.dwt2_plan_workspace_bytes.restype = sz
        lib.dwt2_plan_workspace_bytes.argtypes = [pd, i, i, i, i]
        lib.dwt2_plan_create.argtypes = [pd, i, i, i, i, i, i, vp, sz, ctypes.c_char_p,
                                         ctypes.POINTER(vp)]
        lib.dwt2_plan_execute.argtypes = [vp, vp]
        lib.dwt2_plan_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        lib.dwt2_plan_destroy.argtypes = [vp]
        lib.dwt2_inverse_adjoint.argtypes = [vp, i64, i, i, i, vp, vp, sz, i, i, i, vp]
        lib.dwt2_workspace_bytes_batch.restype = sz
        lib.dwt2_workspace_bytes_batch.argtypes = [i, i, i, i, i, i]
        lib.dwt2_forward_batch.argtypes = [vp, i64, i64, i, i, i, i, vp, i64, vp, sz, i, i, i, vp]
        lib.dwt2_inverse_batch.argtypes = [vp, i64, vp, i64, i64, i, i, i, i, vp, sz, i, i, i, vp]
        lib.dwt2_forward_adjoint_batch.argtypes = [vp, i64, vp, i64, i64, i, i, i, i, vp, sz, i, i,
                                                   i, vp]
        lib.dwt2_inverse_adjoint_batch.argtypes = [vp, i64, i64, i, i, i, i, vp, i64, vp, sz, i, i,
                                                   i, vp]
        lib.dwt2_selftest_wait_timeout.argtypes = [i, vp, sz, vp]
        for f in ("dwt2_max_levels", "dwt2_layout", "dwt2_workspace_init", "dwt2_check_status",
                  "dwt2_forward", "dwt2_forward_scheme", "dwt2_inverse", "dwt2_forward_static",
                  "dwt2_forward_adjoint", "dwt2_inverse_adjoint", "dwt2_plan_create",
                  "dwt2_plan_execute", "dwt2_plan_info", "dwt2_plan_destroy",
                  "dwt2_forward_batch", "dwt2_inverse_batch", "dwt2_forward_adjoint_batch",
                  "dwt2_inverse_adjoint_batch", "dwt2_selftest_wait_timeout"):
            getattr(lib, f).restype = i
        _LIB = lib
    return _LIB


def lib():
    """The loaded ctypes library (raises if it has not been built)."""
    return _lib()


def _wid(wavelet) -> int:
    return WAVELETS[wavelet] if isinstance(wavelet, str) else int(wavelet)


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def max_levels(H: int, W: int) -> int:
    return _lib().dwt2_max_levels(H, W)


def layout(H: int, W: int, levels: int, band_dtype: int):
    """(list of Band, coeff_bytes) of the coefficient buffer."""
    arr = (Band * (1 + 3 * levels))()
    nbytes = ctypes.c_size_t(0)
    rc = _lib().dwt2_layout(H, W, levels, band_dtype, arr, ctypes.byref(nbytes))
    if rc:
        raise Dwt2Error(rc, "dwt2_layout")
    return list(arr), nbytes.value


def workspace_bytes(H: int, W: int, levels: int, wavelet, band_dtype: int,
                    scheme: str = "nonsep") -> int:
    n = _lib().dwt2_workspace_bytes_scheme(H, W, levels, _wid(wavelet), band_dtype,
                                           SCHEMES[scheme])
    if n == 0:
        raise Dwt2Error(1, "dwt2_workspace_bytes")
    return n


def new_workspace(nbytes: int, device=None) -> torch.Tensor:
    """A device workspace whose status header is zeroed."""
    ws = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")
    rc = _lib().dwt2_workspace_init(ws.data_ptr(), nbytes, _stream_ptr())
    if rc:
        raise Dwt2Error(rc, "dwt2_workspace_init")
    return ws


def check_status(ws: torch.Tensor) -> int:
    """Synchronise, read and clear the workspace status word (0 = ok, 5 = a wait timed out)."""
    return _lib().dwt2_check_status(ws.data_ptr(), _stream_ptr())


@dataclass
class Coeffs:
    """A coefficient buffer and its band views (band-list order: LL_J, then HL_j, LH_j, HH_j
    for j = J..1)."""
    buffer: torch.Tensor
    H: int
    W: int
    wavelet: int
    levels: int
    band_dtype: int
    layout: list = field(default_factory=list)

    def band_views(self):
        out = []
        for b in self.layout:
            dt = DT_TORCH[b.dtype]
            es = ESIZE[b.dtype]
            if b.h == 0 or b.w == 0:
                out.append(torch.empty((b.h, b.w), dtype=dt, device=self.buffer.device))
                continue
            raw = self.buffer[b.offset_bytes:b.offset_bytes + b.h * b.pitch_bytes]
            out.append(raw.view(dt).view(b.h, b.pitch_bytes // es)[:, :b.w])
        return out

    def band(self, kind: str, level: int):
        k = {"LL": b"A", "HL": b"H", "LH": b"V", "HH": b"D"}[kind]
        for b, v in zip(self.layout, self.band_views()):
            if b.kind == k and b.level == level:
                return v
        raise KeyError((kind, level))


def _check_img(x: torch.Tensor):
    if not x.is_cuda:
        raise ValueError("dwt2 needs a CUDA tensor (there is no CPU implementation)")
    if x.dim() != 2 or x.stride(1) != 1:
        raise ValueError("image must be 2-D with unit column stride")
    if x.dtype not in TORCH_DT:
        raise ValueError(f"unsupported dtype {x.dtype}")


def alloc_coeffs(H, W, levels, wavelet, band_dtype, device) -> Coeffs:
    lay, nbytes = layout(H, W, levels, band_dtype)
    buf = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=device)
    return Coeffs(buf, H, W, _wid(wavelet), levels, band_dtype, lay)


def forward(x: torch.Tensor, wavelet="cdf53", levels: int = 1, band_dtype=None,
            scheme: str = "nonsep", out: Coeffs | None = None,
            workspace: torch.Tensor | None = None, stream=None) -> Coeffs:
    """dwt2_forward / dwt2_forward_scheme on a CUDA image; returns the coefficient buffer."""
    _check_img(x)
    H, W = x.shape
    wid = _wid(wavelet)
    img_dt = TORCH_DT[x.dtype]
    bdt = TORCH_DT[band_dtype] if isinstance(band_dtype, torch.dtype) else (
        band_dtype if band_dtype is not None else img_dt)
    if out is None:
        out = alloc_coeffs(H, W, levels, wid, bdt, x.device)
    nws = workspace_bytes(H, W, levels, wid, bdt, scheme)
    if workspace is None:
        workspace = new_workspace(nws, x.device)
    rc = _lib().dwt2_forward_scheme(
        x.data_ptr(), x.stride(0) * x.element_size(), H, W, img_dt, out.buffer.data_ptr(),
        workspace.data_ptr(), workspace.numel(), wid, levels, bdt, SCHEMES[scheme],
        _stream_ptr(stream))
    if rc:
        raise Dwt2Error(rc, "dwt2_forward")
    return out


def inverse(c: Coeffs, out: torch.Tensor | None = None, img_dtype=None,
            workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """dwt2_inverse: reconstruct the H x W image from a coefficient buffer."""
    if out is None:
        dt = img_dtype or (torch.int32 if c.wavelet == 0 else torch.float32)
        out = torch.empty((c.H, c.W), dtype=dt, device=c.buffer.device)
    _check_img(out)
    nws = workspace_bytes(c.H, c.W, c.levels, c.wavelet, c.band_dtype)
    if workspace is None:
        workspace = new_workspace(nws, out.device)
    rc = _lib().dwt2_inverse(
        c.buffer.data_ptr(), out.data_ptr(), out.stride(0) * out.element_size(), c.H, c.W,
        TORCH_DT[out.dtype], workspace.data_ptr(), workspace.numel(), c.wavelet, c.levels,
        c.band_dtype, _stream_ptr(stream))
    if rc:
        raise Dwt2Error(rc, "dwt2_inverse")
    return out


def forward_adjoint(g: Coeffs, out: torch.Tensor | None = None,
                    workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """dwt2_forward_adjoint: W^T applied to a band-gradient buffer; returns the H x W gradient."""
    if out is None:
        out = torch.empty((g.H, g.W), dtype=torch.float32, device=g.buffer.device)
    _check_img(out)
    nws = workspace_bytes(g.H, g.W, g.levels, g.wavelet, g.band_dtype)
    if workspace is None:
        workspace = new_workspace(nws, out.device)
    rc = _lib().dwt2_forward_adjoint(
        g.buffer.data_ptr(), out.data_ptr(), out.stride(0) * out.element_size(), g.H, g.W,
        TORCH_DT[out.dtype], workspace.data_ptr(), workspace.numel(), g.wavelet, g.levels,
        g.band_dtype, _stream_ptr(stream))
    if rc:
        raise Dwt2Error(rc, "dwt2_forward_adjoint")
    return out


def inverse_adjoint(x: torch.Tensor, wavelet="cdf97", levels: int = 1, out: Coeffs | None = None,
                    workspace: torch.Tensor | None = None, stream=None) -> Coeffs:
    """dwt2_inverse_adjoint: W^-T applied to an image-shaped gradient; returns band gradients."""
    _check_img(x)
    H, W = x.shape
    wid = _wid(wavelet)
    if out is None:
        out = alloc_coeffs(H, W, levels, wid, DT_F32, x.device)
    nws = workspace_bytes(H, W, levels, wid, DT_F32)
    if workspace is None:
        workspace = new_workspace(nws, x.device)
    rc = _lib().dwt2_inverse_adjoint(
        x.data_ptr(), x.stride(0) * x.element_size(), H, W, TORCH_DT[x.dtype],
        out.buffer.data_ptr(), workspace.data_ptr(), workspace.numel(), wid, levels, DT_F32,
        _stream_ptr(stream))
    if rc:
        raise Dwt2Error(rc, "dwt2_inverse_adjoint")
    return out



# ------------------------------------------------------------------ uniform batches (N x H x W)
def workspace_bytes_batch(N: int, H: int, W: int, levels: int, wavelet, band_dtype: int) -> int:
    n = _lib().dwt2_workspace_bytes_batch(N, H, W, levels, _wid(wavelet), band_dtype)
    if n == 0:
        raise Dwt2Error(1, f"dwt2_workspace_bytes_batch({N}, {H}, {W}, {levels})")
    return n


def _check_batch_img(x: torch.Tensor):
    if not x.is_cuda or x.dim() != 3 or x.stride(2) != 1:
        raise ValueError("batched images must be CUDA tensors (N, H, W) with unit column stride")
    if x.dtype not in TORCH_DT:
        raise ValueError(f"unsupported image dtype {x.dtype}")


def _check_batch_coeffs(c: torch.Tensor, N: int, nbytes: int):
    if not c.is_cuda or c.dim() != 2 or c.shape[0] != N or c.stride(1) != 1:
        raise ValueError("batched coefficients must be CUDA tensors (N, n) with unit stride")
    if c.shape[1] * c.element_size() < nbytes:
        raise ValueError(f"coefficient rows hold {c.shape[1] * c.element_size()} bytes, "
                         f"the layout needs {nbytes}")


def forward_batch(x: torch.Tensor, wavelet="cdf97", levels: int = 1, band_dtype=None,
                  out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """dwt2_forward_batch on N images (N, H, W); returns (N, layout bytes) uint8 coefficients
    (or fills `out`, any (N, n) CUDA tensor whose rows hold the layout)."""
    _check_batch_img(x)
    N, H, W = x.shape
    wid = _wid(wavelet)
    img_dt = TORCH_DT[x.dtype]
    bdt = TORCH_DT[band_dtype] if isinstance(band_dtype, torch.dtype) else (
        band_dtype if band_dtype is not None else img_dt)
    _, nbytes = layout(H, W, levels, bdt)
    if out is None:
        out = torch.empty((N, max(nbytes, 16)), dtype=torch.uint8, device=x.device)
    _check_batch_coeffs(out, N, nbytes)
    if workspace is None:
        workspace = new_workspace(workspace_bytes_batch(N, H, W, levels, wid, bdt), x.device)
    es = x.element_size()
    rc = _lib().dwt2_forward_batch(
        x.data_ptr(), x.stride(1) * es, x.stride(0) * es, N, H, W, img_dt, out.data_ptr(),
        out.stride(0) * out.element_size(), workspace.data_ptr(), workspace.numel(), wid, levels,
        bdt, _stream_ptr(stream))
    if rc:
        raise Dwt2Error(rc, "dwt2_forward_batch")
    return out


def inverse_batch(c: torch.Tensor, H: int, W: int, wavelet="cdf97", levels: int = 1,
                  band_dtype=None, out: torch.Tensor | None = None, img_dtype=None,
                  workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """dwt2_inverse_batch: (N, n) coefficient rows -> (N, H, W) images."""
    N = c.shape[0]
    wid = _wid(wavelet)
    bdt = band_dtype if band_dtype is not None else (DT_I32 if wid == 0 else DT_F32)
    _, nbytes = layout(H, W, levels, bdt)
    _check_batch_coeffs(c, N, nbytes)
    if out is None:
        dt = img_dtype or (torch.int32 if wid == 0 else torch.float32)
        out = torch.empty((N, H, W), dtype=dt, device=c.device)
    _check_batch_img(out)
    if workspace is None:
        workspace = new_workspace(workspace_bytes_batch(N, H, W, levels, wid, bdt), c.device)
    es = out.element_size()
    rc = _lib().dwt2_inverse_batch(
        c.data_ptr(), c.stride(0) * c.element_size(), out.data_ptr(), out.stride(1) * es,
        out.stride(0) * es, N, H, W, TORCH_DT[out.dtype], workspace.data_ptr(), workspace.numel(),
        wid, levels, bdt, _stream_ptr(stream))
    if rc:
        raise Dwt2Error(rc, "dwt2_inverse_batch")
    return out


def forward_adjoint_batch(g: torch.Tensor, H: int, W: int, wavelet="cdf97", levels: int = 1,
                          out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                          stream=None) -> torch.Tensor:
    """dwt2_forward_adjoint_batch: W^T on (N, n) float32 band-gradient rows -> (N, H, W)."""
    N = g.shape[0]
    wid = _wid(wavelet)
    _, nbytes = layout(H, W, levels, DT_F32)
    _check_batch_coeffs(g, N, nbytes)
    if out is None:
        out = torch.empty((N, H, W), dtype=torch.float32, device=g.device)
    _check_batch_img(out)
    if workspace is None:
        workspace = new_workspace(workspace_bytes_batch(N, H, W, levels, wid, DT_F32), g.device)
    es = out.element_size()
    rc = _lib().dwt2_forward_adjoint_batch(
        g.data_ptr(), g.stride(0) * g.element_size(), out.data_ptr(), out.stride(1) * es,
        out.stride(0) * es, N, H, W, TORCH_DT[out.dtype], workspace.data_ptr(), workspace.numel(),
        wid, levels, DT_F32, _stream_ptr(stream))
    if rc:
        raise Dwt2Error(rc, "dwt2_forward_adjoint_batch")
    return out


def inverse_adjoint_batch(x: torch.Tensor, wavelet="cdf97", levels: int = 1,
                          out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                          stream=None) -> torch.Tensor:
    """dwt2_inverse_adjoint_batch: W^-T on (N, H, W) float32 gradients -> (N, n) band rows."""
    _check_batch_img(x)
    N, H, W = x.shape
    wid = _wid(wavelet)
    _, nbytes = layout(H, W, levels, DT_F32)
    if out is None:
        out = torch.zeros((N, max(nbytes, 16) // 4), dtype=torch.float32, device=x.device)
    _check_batch_coeffs(out, N, nbytes)
    if workspace is None:
        workspace = new_workspace(workspace_bytes_batch(N, H, W, levels, wid, DT_F32), x.device)
    es = x.element_size()
    rc = _lib().dwt2_inverse_adjoint_batch(
        x.data_ptr(), x.stride(1) * es, x.stride(0) * es, N, H, W, TORCH_DT[x.dtype],
        out.data_ptr(), out.stride(0) * out.element_size(), workspace.data_ptr(),
        workspace.numel(), wid, levels, DT_F32, _stream_ptr(stream))
    if rc:
        raise Dwt2Error(rc, "dwt2_inverse_adjoint_batch")
    return out


def selftest_wait_timeout(which: int, workspace: torch.Tensor, stream=None) -> None:
    """dwt2_selftest_wait_timeout: one warp waits on something nothing signals (0: a barrier
    phase, 1: a counter); about 2 s later check_status(workspace) reports DWT2_ETIMEOUT."""
    rc = _lib().dwt2_selftest_wait_timeout(which, workspace.data_ptr(), workspace.numel(),
                                           _stream_ptr(stream))
    if rc:
        raise Dwt2Error(rc, "dwt2_selftest_wait_timeout")


class Plan:
    """A batched plan (dwt2_plan_create): every level of every image in one persistent launch,
    replayed from a CUDA graph by run().  Keeps the tensors it was built on alive."""

    def __init__(self, images, coeffs, wavelet, levels: int, direction: str = "forward",
                 band_dtype: int | None = None, tune_cache: str | None = None):
        self.images, self.coeffs = list(images), list(coeffs)
        n = len(self.images)
        wid = _wid(wavelet)
        img_dt = TORCH_DT[self.images[0].dtype]
        bdt = self.coeffs[0].band_dtype if band_dtype is None else band_dtype
        descs = (ImageDesc * n)()
        for k, (x, c) in enumerate(zip(self.images, self.coeffs)):
            _check_img(x)
            descs[k] = ImageDesc(x.data_ptr(), x.stride(0) * x.element_size(), x.shape[0],
                                 x.shape[1], c.buffer.data_ptr())
        nws = _lib().dwt2_plan_workspace_bytes(descs, n, wid, levels, bdt)
        if nws == 0:
            raise Dwt2Error(1, "dwt2_plan_workspace_bytes")
        self.workspace = new_workspace(nws, self.images[0].device)
        h = ctypes.c_void_p(0)
        rc = _lib().dwt2_plan_create(descs, n, wid, levels, img_dt, bdt, DIRECTIONS[direction],
                                     self.workspace.data_ptr(), nws,
                                     tune_cache.encode() if tune_cache else None, ctypes.byref(h))
        if rc:
            raise Dwt2Error(rc, "dwt2_plan_create")
        self.handle = h

    def run(self, stream=None):
        rc = _lib().dwt2_plan_execute(self.handle, _stream_ptr(stream))
        if rc:
            raise Dwt2Error(rc, "dwt2_plan_execute")

    def info(self):
        r, c, t = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _lib().dwt2_plan_info(self.handle, ctypes.byref(r), ctypes.byref(c), ctypes.byref(t))
        return {"rows_per_tile": r.value, "ctas_per_sm": c.value, "tiles": t.value}

    def close(self):
        if getattr(self, "handle", None):
            _lib().dwt2_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_forward(images, wavelet="cdf97", levels: int = 1, band_dtype=None,
                 tune_cache: str | None = None):
    """A forward plan over CUDA images of any sizes; returns (plan, [Coeffs per image])."""
    dev = images[0].device
    bdt = TORCH_DT[band_dtype] if isinstance(band_dtype, torch.dtype) else (
        band_dtype if band_dtype is not None else TORCH_DT[images[0].dtype])
    coeffs = [alloc_coeffs(x.shape[0], x.shape[1], levels, wavelet, bdt, dev) for x in images]
    return Plan(images, coeffs, wavelet, levels, "forward", bdt, tune_cache), coeffs
