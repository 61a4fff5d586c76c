"""numpy front end of the CPU oracle (dwt2_oracle.c).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's CPU-baseline leg use
it; the product path never imports it, and it imports nothing from the product package.

Every transform here runs in the C oracle: fp64 for the float wavelets, exact int64 for the
reversible CDF 5/3.  The band list follows the paper's quad order [LL, HL, LH, HH] (Sec. 2):
LL_J first, then HL_j, LH_j, HH_j for j = J..1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dwt2_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

WAVELETS = {"cdf53_int": 0, "cdf53": 1, "cdf97": 2, "dd97": 3, "dd137": 4}
SCHEMES = {"eq3": 0, "rows": 1, "cols": 2, "eq5": 3, "adapted": 4}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so (plain -O2).  OpenMP, when gcc has
    it, only shares out independent lines among threads (set_threads; one thread by default)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "dwt2_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC]
        if subprocess.call(base + ["-fopenmp"], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i = ctypes.c_void_p, ctypes.c_int
        lib.orc_set_threads.argtypes = [i]
        lib.orc_set_threads.restype = i
        lib.orc_max_levels.argtypes = [i, i]
        lib.orc_max_levels.restype = i
        lib.orc_coeff_count.argtypes = [i, i, i]
        lib.orc_coeff_count.restype = ctypes.c_int64
        lib.orc_forward.argtypes = [vp, i, i, i, i, i, i, vp]
        lib.orc_inverse.argtypes = [vp, i, i, i, i, i, vp]
        lib.orc_forward_adjoint.argtypes = [vp, i, i, i, i, vp]
        lib.orc_inverse_adjoint.argtypes = [vp, i, i, i, i, vp]
        lib.orc_nonsep_steps.argtypes = [vp, i, i, i, i, vp]
        lib.orc_adapted_steps.argtypes = [vp, i, i, i, i, vp]
        lib.orc_adapted_apply.argtypes = [vp, i, i, i, i, i]
        for f in ("orc_forward", "orc_inverse", "orc_forward_adjoint", "orc_inverse_adjoint",
                  "orc_nonsep_steps", "orc_adapted_steps", "orc_adapted_apply"):
            getattr(lib, f).restype = i
        lib.orc_set_threads(1)  # the sequential oracle unless a caller asks for more threads
        _lib = lib
    return _lib


def _wid(wavelet) -> int:
    return WAVELETS[wavelet] if isinstance(wavelet, str) else int(wavelet)


def _dtype(wavelet):
    return np.int64 if _wid(wavelet) == 0 else np.float64


def set_threads(n: int) -> int:
    """Threads for the oracle's line loops (1 = sequential, the default); the results are the
    same bits for any count.  Returns the count in effect (1 without OpenMP)."""
    return _load().orc_set_threads(int(n))


def max_levels(H: int, W: int) -> int:
    return _load().orc_max_levels(H, W)


def band_shapes(H: int, W: int, levels: int):
    """[(kind, level, h, w)] in band-list order: LL_J, then HL_j, LH_j, HH_j for j = J..1."""
    hs, ws = [H], [W]
    for _ in range(levels):
        hs.append((hs[-1] + 1) // 2)
        ws.append((ws[-1] + 1) // 2)
    out = [("LL", levels, hs[levels], ws[levels])]
    for j in range(levels, 0, -1):
        h, w = hs[j - 1], ws[j - 1]
        out += [("HL", j, (h + 1) // 2, w // 2), ("LH", j, h // 2, (w + 1) // 2),
                ("HH", j, h // 2, w // 2)]
    return out


def split_bands(flat: np.ndarray, H: int, W: int, levels: int):
    """Views of a flat band-list array as 2-D bands, in band-list order."""
    out, o = [], 0
    for _, _, h, w in band_shapes(H, W, levels):
        out.append(flat[o:o + h * w].reshape(h, w))
        o += h * w
    return out


def join_bands(bands) -> np.ndarray:
    return np.concatenate([np.ascontiguousarray(b).reshape(-1) for b in bands])


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def forward(img, wavelet, levels: int, scheme: str = "eq3", extension_form: bool = False):
    """Forward transform; returns the list of 2-D bands (int64 or float64)."""
    img = np.ascontiguousarray(img, dtype=_dtype(wavelet))
    H, W = img.shape
    lib = _load()
    n = lib.orc_coeff_count(H, W, levels)
    if n < 0:
        raise ValueError(f"invalid size/levels {H}x{W} L={levels}")
    out = np.zeros(n, dtype=_dtype(wavelet))
    rc = lib.orc_forward(_ptr(img), H, W, _wid(wavelet), levels, SCHEMES[scheme],
                         int(extension_form), _ptr(out))
    if rc:
        raise ValueError(f"orc_forward failed ({rc})")
    return split_bands(out, H, W, levels)


def inverse(bands, H: int, W: int, wavelet, levels: int, scheme: str = "eq3"):
    flat = np.ascontiguousarray(join_bands(bands), dtype=_dtype(wavelet))
    out = np.zeros((H, W), dtype=_dtype(wavelet))
    rc = _load().orc_inverse(_ptr(flat), H, W, _wid(wavelet), levels, SCHEMES[scheme],
                             _ptr(out))
    if rc:
        raise ValueError(f"orc_inverse failed ({rc})")
    return out


def forward_adjoint(g_bands, H: int, W: int, wavelet, levels: int):
    """W^T applied to a band-list gradient; returns the H x W image gradient (float64)."""
    flat = np.ascontiguousarray(join_bands(g_bands), dtype=np.float64)
    out = np.zeros((H, W), dtype=np.float64)
    rc = _load().orc_forward_adjoint(_ptr(flat), H, W, _wid(wavelet), levels, _ptr(out))
    if rc:
        raise ValueError(f"orc_forward_adjoint failed ({rc})")
    return out


def inverse_adjoint(g_img, wavelet, levels: int):
    """W^-T applied to an image gradient; returns the band-list gradient (float64)."""
    g = np.ascontiguousarray(g_img, dtype=np.float64)
    H, W = g.shape
    n = _load().orc_coeff_count(H, W, levels)
    out = np.zeros(n, dtype=np.float64)
    rc = _load().orc_inverse_adjoint(_ptr(g), H, W, _wid(wavelet), levels, _ptr(out))
    if rc:
        raise ValueError(f"orc_inverse_adjoint failed ({rc})")
    return split_bands(out, H, W, levels)


def nonsep_steps(img, wavelet, nsteps: int, adapted: bool = False):
    """The first nsteps steps of one level (no scaling): returns (a, b, c, e), the LL, HL, LH,
    HH polyphase components after those steps.  Eq. 5's fused steps (predict, update, ...), or
    with adapted=True the adapted scheme's (local predict, fused predict, local update, fused
    update, ...)."""
    img = np.ascontiguousarray(img, dtype=np.float64)
    H, W = img.shape
    ner, ndr, nec, ndc = (H + 1) // 2, H // 2, (W + 1) // 2, W // 2
    out = np.zeros(ner * nec + ner * ndc + ndr * nec + ndr * ndc)
    fn = _load().orc_adapted_steps if adapted else _load().orc_nonsep_steps
    rc = fn(_ptr(img), H, W, _wid(wavelet), nsteps, _ptr(out))
    if rc:
        raise ValueError(f"oracle step function failed ({rc})")
    shapes = [(ner, nec), (ner, ndc), (ndr, nec), (ndr, ndc)]
    res, o = [], 0
    for h, w in shapes:
        res.append(out[o:o + h * w].reshape(h, w))
        o += h * w
    return res


def adapted_apply(parts, H: int, W: int, wavelet, k0: int, k1: int):
    """Adapted steps k0 .. k1-1 applied to the polyphase components parts = (a, b, c, e) of an
    H x W level; returns the new (a, b, c, e)."""
    flat = np.concatenate([np.ascontiguousarray(p, dtype=np.float64).ravel() for p in parts])
    rc = _load().orc_adapted_apply(_ptr(flat), H, W, _wid(wavelet), k0, k1)
    if rc:
        raise ValueError(f"orc_adapted_apply failed ({rc})")
    out, o = [], 0
    for p in parts:
        out.append(flat[o:o + p.size].reshape(p.shape))
        o += p.size
    return out
