"""ctypes binding of libfastresolve.so (argument marshalling only).

Every operator runs in the library's CUDA kernels; this module checks shapes, dtypes and
devices, passes raw device pointers and the current CUDA stream, and turns error codes into
exceptions. There is no fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfastresolve.so")

FR_WTERM, FR_NTERM, FR_MFS, FR_DROP_OOB, FR_NO_PSF, FR_DETERMINISTIC = 1, 2, 4, 8, 16, 32
FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_EUNSUPPORTED, FR_ETIMEOUT = -1, -2, -3, -4, -5
ERRORS = {-1: "FR_EINVAL", -2: "FR_ENOMEM", -3: "FR_ECUDA", -4: "FR_EUNSUPPORTED", -5: "FR_ETIMEOUT"}

EXPORTS = ["fr_plan_create", "fr_degrid", "fr_grid", "fr_dirty_psf", "fr_psf_apply",
           "fr_likelihood_grad", "fr_major_cycle", "fr_plan_get_info", "fr_plan_footprint",
           "fr_plan_check", "fr_plan_destroy", "fr_strerror", "fr_last_error", "fr_launch_count",
           "fr_selftest_fft_host", "fr_psf_convolve_noalloc", "fr_noise_fit", "fr_noise_kernel",
           "fr_noise_apply_inverse", "fr_fast_likelihood_grad", "fr_psf_set_padding",
           "fr_psf_padding", "fr_degrid_weighted", "fr_fast_likelihood_grad_resid",
           "fr_selftest_wait_timeout", "fr_psf_group_scratch_bytes", "fr_psf_apply_group",
           "fr_plan_prepare"]


class FastResolveError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class PlanInfo(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nsky", ctypes.c_int32),
                ("nchan", ctypes.c_int32), ("nrow", ctypes.c_int64), ("nvis", ctypes.c_int64),
                ("grid_nu", ctypes.c_int32), ("grid_nv", ctypes.c_int32),
                ("support", ctypes.c_int32), ("beta", ctypes.c_double),
                ("wplanes_total", ctypes.c_int32), ("wplanes_max", ctypes.c_int32),
                ("dw", ctypes.c_double), ("nvis_dropped", ctypes.c_int64),
                ("work_items", ctypes.c_int64), ("flags", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load the native library (build it first with paper_2406_09144_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libfastresolve.so not found at {path}; build it with "
                           "`python -m paper_2406_09144_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, I32, I64, D, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32
    lib.fr_plan_create.argtypes = [P, I64, P, I32, P, I32, I32, D, D, D, U32, P, ctypes.POINTER(P)]
    lib.fr_degrid.argtypes = [P, P, P, P]
    lib.fr_degrid_weighted.argtypes = [P, P, P, P]
    lib.fr_fast_likelihood_grad_resid.argtypes = [P, P, P, I32, P, P, P, P]
    lib.fr_grid.argtypes = [P, P, I32, P, P]
    lib.fr_dirty_psf.argtypes = [P, P, P, P, P, P]
    lib.fr_psf_apply.argtypes = [P, P, I32, P, P]
    lib.fr_likelihood_grad.argtypes = [P, P, P, I32, I32, P, P, P]
    lib.fr_major_cycle.argtypes = [P, P, P, P, P, P, P, P]
    lib.fr_noise_fit.argtypes = [P, D, P, P]
    lib.fr_noise_kernel.argtypes = [P, P, P]
    lib.fr_noise_apply_inverse.argtypes = [P, P, I32, P, P]
    lib.fr_fast_likelihood_grad.argtypes = [P, P, P, I32, P, P, P]
    lib.fr_psf_set_padding.argtypes = [P, I32, I32, P]
    lib.fr_psf_padding.argtypes = [P, ctypes.POINTER(I32), ctypes.POINTER(I32)]
    lib.fr_plan_get_info.argtypes = [P, ctypes.POINTER(PlanInfo)]
    lib.fr_plan_footprint.argtypes = [P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
    lib.fr_plan_check.argtypes = [P, P]
    lib.fr_plan_destroy.argtypes = [P]
    lib.fr_plan_destroy.restype = None
    lib.fr_strerror.argtypes = [ctypes.c_int]
    lib.fr_strerror.restype = ctypes.c_char_p
    lib.fr_last_error.argtypes = []
    lib.fr_last_error.restype = ctypes.c_char_p
    lib.fr_launch_count.argtypes = [ctypes.c_int]
    lib.fr_launch_count.restype = ctypes.c_uint64
    lib.fr_selftest_fft_host.argtypes = [P, I32, I32, I32]
    lib.fr_selftest_wait_timeout.argtypes = [P, P]
    lib.fr_psf_group_scratch_bytes.argtypes = [P, I32, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.fr_psf_apply_group.argtypes = [P, I32, P, P, P, P, ctypes.c_size_t, P]
    lib.fr_plan_prepare.argtypes = [P, I32, P]
    lib.fr_profile_enable.argtypes = [ctypes.c_int]
    lib.fr_profile_enable.restype = None
    lib.fr_profile_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_uint64), I32]
    lib.fr_profile_read.restype = ctypes.c_int
    lib.fr_profile_category.argtypes = [I32]
    lib.fr_profile_category.restype = ctypes.c_char_p
    lib.fr_psf_convolve_noalloc.argtypes = [P, P, I32, I32, I32, P, P]
    lib.fr_psf_convolve_noalloc.restype = ctypes.c_int
    for name in ("fr_plan_create", "fr_degrid", "fr_grid", "fr_dirty_psf", "fr_psf_apply",
                 "fr_likelihood_grad", "fr_major_cycle", "fr_plan_get_info", "fr_plan_footprint",
                 "fr_plan_check", "fr_selftest_fft_host", "fr_psf_set_padding", "fr_psf_padding",
                 "fr_degrid_weighted", "fr_fast_likelihood_grad_resid", "fr_selftest_wait_timeout",
                 "fr_psf_group_scratch_bytes", "fr_psf_apply_group", "fr_plan_prepare"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def check(code: int):
    if code != 0:
        raise FastResolveError(code, load().fr_last_error().decode(errors="replace"))


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))(*[ctypes.c_void_p(int(p)) for p in ptrs])
    return arr


def psf_group_scratch_bytes(plans, batches) -> int:
    """Scratch bytes of psf_apply_group for these plans and batches."""
    hs = _ptr_array([p._h.value for p in plans])
    bs = (ctypes.c_int32 * len(batches))(*[int(b) for b in batches])
    n = ctypes.c_size_t()
    check(load().fr_psf_group_scratch_bytes(hs, len(plans), bs, ctypes.byref(n)))
    return int(n.value)


def psf_apply_group(plans, skies, outs, scratch, stream=None):
    """PSF convolutions of several plans (equal image size and PSF padding) in one launch per
    pass: skies[j], outs[j] [batch_j, nsky_j, nx, ny] float32 on the device; scratch a uint8
    device tensor of at least psf_group_scratch_bytes bytes."""
    torch = _torch()
    batches = []
    for p, s, o in zip(plans, skies, outs):
        b, shape = p._batch_shape(s)
        _dev(s, torch.float32, shape, "sky")
        _dev(o, torch.float32, shape, "out")
        batches.append(b)
    hs = _ptr_array([p._h.value for p in plans])
    bs = (ctypes.c_int32 * len(plans))(*batches)
    sp = _ptr_array([s.data_ptr() for s in skies])
    op = _ptr_array([o.data_ptr() for o in outs])
    check(load().fr_psf_apply_group(hs, len(plans), sp, bs, op, ctypes.c_void_p(scratch.data_ptr()),
                                    scratch.numel() * scratch.element_size(), _stream_ptr(stream)))


def launch_count(reset: bool = False) -> int:
    return int(load().fr_launch_count(1 if reset else 0))


PROFILE_CATEGORIES = 8


def profile_enable(on: bool = True):
    """Bracket every library launch with CUDA events (per kernel class) until disabled."""
    load().fr_profile_enable(1 if on else 0)


def profile_read() -> dict:
    """{category: (milliseconds, algorithmic bytes, launches)} since profile_enable(True)."""
    lib = load()
    n = PROFILE_CATEGORIES
    ms = (ctypes.c_double * n)()
    by = (ctypes.c_double * n)()
    nl = (ctypes.c_uint64 * n)()
    lib.fr_profile_read(ms, by, nl, n)
    return {lib.fr_profile_category(c).decode(): (ms[c], by[c], int(nl[c])) for c in range(n)}


def selftest_fft_host(x: np.ndarray, direction: int) -> np.ndarray:
    """Run the FFT passes' stage arithmetic on the CPU (no GPU): x complex [batch, n],
    n = 2^k 3^a 5^b."""
    a = np.ascontiguousarray(x, dtype=np.complex64).copy()
    batch, n = a.shape
    check(load().fr_selftest_fft_host(a.ctypes.data, n, batch, direction))
    return a


def fft_len_at_least(m: int) -> int:
    """The shortest transform length the library takes that is >= m: 2^k (32..16384),
    3 2^k (48..6144) or 5 2^k (80..5120). The oversampled grid of an n-pixel side is
    fft_len_at_least(2 n) (plan info grid_nu reports it)."""
    best = 16384
    for c, lo, hi in ((1, 32, 16384), (3, 48, 6144), (5, 80, 5120)):
        L = c * 16
        while L <= hi:
            if L >= max(m, lo) and L < best:
                best = L
            L *= 2
    return best


def padded_lengths(n: int):
    """The padded PSF transform lengths fr_psf_set_padding takes for an image side n: even
    L in (n, 2n] of the form 2^k (32..16384), 3 2^k (48..6144) or 5 2^k (80..5120)."""
    out = []
    for c, lo, hi in ((1, 32, 16384), (3, 48, 6144), (5, 80, 5120)):
        L = c * 16
        while L <= min(2 * n, hi):
            if L > n and L >= lo:
                out.append(L)
            L *= 2
    return sorted(out)


# ------------------------------------------------------------------------------- torch side
def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, shape, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A measurement-operator plan: R, R^dagger N^-1, PSF convolution, likelihood."""

    def __init__(self, uvw, freqs, nx, ny, pixsize_x, pixsize_y=None, weights=None, eps=1e-5,
                 wterm=True, nterm=True, mfs=False, drop_oob=False, no_psf=False,
                 deterministic=False, stream=None):
        lib = load()
        uvw = np.ascontiguousarray(uvw, dtype=np.float64)
        freqs = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
        if uvw.ndim != 2 or uvw.shape[1] != 3:
            raise ValueError("uvw must be [nrow, 3]")
        self.nrow, self.nchan = uvw.shape[0], freqs.shape[0]
        wptr = None
        if weights is not None:
            weights = np.ascontiguousarray(np.broadcast_to(weights, (self.nrow, self.nchan)),
                                           dtype=np.float32)
            wptr = weights.ctypes.data
        flags = ((FR_WTERM if wterm else 0) | (FR_NTERM if nterm else 0) | (FR_MFS if mfs else 0)
                 | (FR_DROP_OOB if drop_oob else 0) | (FR_NO_PSF if no_psf else 0)
                 | (FR_DETERMINISTIC if deterministic else 0))
        self.nx, self.ny = int(nx), int(ny)
        self.nsky = 1 if mfs else self.nchan
        h = ctypes.c_void_p()
        check(lib.fr_plan_create(uvw.ctypes.data, self.nrow, freqs.ctypes.data, self.nchan, wptr,
                                 self.nx, self.ny, float(pixsize_x),
                                 float(pixsize_x if pixsize_y is None else pixsize_y), float(eps),
                                 flags, _stream_ptr(stream) if _has_cuda() else None,
                                 ctypes.byref(h)))
        self._h = h

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None):
            load().fr_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = PlanInfo()
        check(load().fr_plan_get_info(self._h, ctypes.byref(i)))
        return i.as_dict()

    def footprint(self):
        r, w = ctypes.c_size_t(), ctypes.c_size_t()
        check(load().fr_plan_footprint(self._h, ctypes.byref(r), ctypes.byref(w)))
        return int(r.value), int(w.value)

    def check(self, stream=None):
        check(load().fr_plan_check(self._h, _stream_ptr(stream)))

    def prepare(self, batch=1, stream=None):
        """Allocate the per-stream workspace for calls on `stream` without computing."""
        check(load().fr_plan_prepare(self._h, int(batch), _stream_ptr(stream)))

    # ------------------------------------------------------------------ shapes
    @property
    def sky_shape(self):
        return (self.nsky, self.nx, self.ny)

    @property
    def vis_shape(self):
        return (self.nrow, self.nchan)

    # ------------------------------------------------------------------ operators
    def degrid(self, sky, out=None, stream=None, weighted=False):
        """R (Eq. rime): sky [nsky, nx, ny] float32 -> vis [nrow, nchan] complex64; with
        weighted=True N^-1 R (every visibility times its weight)."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.vis_shape, dtype=torch.complex64, device=sky.device)
        fn = load().fr_degrid_weighted if weighted else load().fr_degrid
        check(fn(self._h, _dev(sky, torch.float32, self.sky_shape, "sky"),
                 _dev(out, torch.complex64, self.vis_shape, "vis"), _stream_ptr(stream)))
        return out

    def grid(self, vis, apply_weights=True, out=None, stream=None):
        """R^dagger (N^-1) (Eq. clean): vis [nrow, nchan] complex64 -> [nsky, nx, ny] float32."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.sky_shape, dtype=torch.float32, device=vis.device)
        check(load().fr_grid(self._h, _dev(vis, torch.complex64, self.vis_shape, "vis"),
                             1 if apply_weights else 0,
                             _dev(out, torch.float32, self.sky_shape, "dirty"), _stream_ptr(stream)))
        return out

    def dirty_psf(self, vis=None, want_dirty=True, want_psf=True, device="cuda", stream=None):
        """Dirty image R^dagger N^-1 V, PSF [nsky, 2nx, 2ny] and psf_norm (sum of weights)."""
        torch = _torch()
        dirty = psf = None
        if want_dirty:
            dirty = torch.empty(self.sky_shape, dtype=torch.float32, device=device)
        if want_psf:
            psf = torch.empty((self.nsky, 2 * self.nx, 2 * self.ny), dtype=torch.float32, device=device)
        norm = np.zeros(self.nsky, dtype=np.float64)
        vptr = _dev(vis, torch.complex64, self.vis_shape, "vis") if vis is not None else None
        check(load().fr_dirty_psf(
            self._h, vptr,
            _dev(dirty, torch.float32, self.sky_shape, "dirty") if dirty is not None else None,
            _dev(psf, torch.float32, (self.nsky, 2 * self.nx, 2 * self.ny), "psf") if psf is not None else None,
            norm.ctypes.data, _stream_ptr(stream)))
        return dirty, psf, norm

    def psf_apply(self, sky, out=None, stream=None):
        """PSF convolution (Sec. 3.3.2): sky [batch, nsky, nx, ny] or [nsky, nx, ny]."""
        torch = _torch()
        batch, shape = self._batch_shape(sky)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=sky.device)
        check(load().fr_psf_apply(self._h, _dev(sky, torch.float32, shape, "sky"), batch,
                                  _dev(out, torch.float32, shape, "out"), _stream_ptr(stream)))
        return out

    def set_psf_padding(self, lx, ly, stream=None):
        """Reduced padding (Sec. 3.3.2): run the PSF convolutions on an lx x ly grid with the
        PSF truncated to |a| <= min(lx - nx, nx - 1), |b| <= min(ly - ny, ny - 1);
        lx = 2 nx, ly = 2 ny is the exact default. See padded_lengths()."""
        check(load().fr_psf_set_padding(self._h, int(lx), int(ly), _stream_ptr(stream)))

    @property
    def psf_padding(self):
        lx, ly = ctypes.c_int32(), ctypes.c_int32()
        check(load().fr_psf_padding(self._h, ctypes.byref(lx), ctypes.byref(ly)))
        return lx.value, ly.value

    def likelihood_grad(self, sky, dirty, exact=False, grad=None, want_value=True, stream=None):
        """L = 1/2 s.(A s) - s.d and grad = A s - d with A = PSF * or R^dagger N^-1 R."""
        torch = _torch()
        batch, shape = self._batch_shape(sky)
        if grad is None:
            grad = torch.empty(shape, dtype=torch.float32, device=sky.device)
        val = np.zeros(batch, dtype=np.float64)
        check(load().fr_likelihood_grad(
            self._h, _dev(sky, torch.float32, shape, "sky"), _dev(dirty, torch.float32, shape, "dirty"),
            batch, 1 if exact else 0, _dev(grad, torch.float32, shape, "grad"),
            val.ctypes.data if want_value else None, _stream_ptr(stream)))
        return (val if want_value else None), grad

    def major_cycle(self, sky, dirty, vis=None, want_resid=True, stream=None):
        """Algorithm 1 major cycle: resid = dirty - R^dagger N^-1 R sky, |resid|^2, chi^2 of vis."""
        torch = _torch()
        resid = torch.empty(self.sky_shape, dtype=torch.float32, device=sky.device) if want_resid else None
        rn = ctypes.c_double()
        chi = ctypes.c_double()
        check(load().fr_major_cycle(
            self._h, _dev(sky, torch.float32, self.sky_shape, "sky"),
            _dev(dirty, torch.float32, self.sky_shape, "dirty"),
            _dev(resid, torch.float32, self.sky_shape, "resid") if resid is not None else None,
            ctypes.byref(rn),
            _dev(vis, torch.complex64, self.vis_shape, "vis") if vis is not None else None,
            ctypes.byref(chi) if vis is not None else None, _stream_ptr(stream)))
        return resid, rn.value, (chi.value if vis is not None else None)

    def noise_fit(self, eps_noise, stream=None):
        """Fit the noise kernel K = exp(xi) + eps_noise (Sec. 3.3.3); returns 1/2 sum ln(2 pi K)
        per image (the constant ln|2 pi N'| / 2 of Eq. ham_new)."""
        logdet = np.zeros(self.nsky, dtype=np.float64)
        check(load().fr_noise_fit(self._h, float(eps_noise), logdet.ctypes.data, _stream_ptr(stream)))
        return logdet

    def noise_kernel(self, device="cuda", stream=None):
        """The fitted K [nsky, nx, ny] (numpy.fft.fft2 frequency order)."""
        torch = _torch()
        K = torch.empty((self.nsky, self.nx, self.ny), dtype=torch.float32, device=device)
        check(load().fr_noise_kernel(self._h, _dev(K, torch.float32, K.shape, "K"), _stream_ptr(stream)))
        return K

    def noise_apply_inverse(self, x, out=None, stream=None):
        """N'^-1 x = FFT^-1[K^-1 FFT(x)] per image (periodic): x [batch, nsky, nx, ny] or [nsky, nx, ny]."""
        torch = _torch()
        batch, shape = self._batch_shape(x)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=x.device)
        check(load().fr_noise_apply_inverse(self._h, _dev(x, torch.float32, shape, "x"), batch,
                                            _dev(out, torch.float32, shape, "out"), _stream_ptr(stream)))
        return out

    def fast_likelihood_grad(self, sky, dirty, grad=None, want_value=True, stream=None,
                             want_ninv_resid=False):
        """Eq. ham_new: value = 1/2 r.(N'^-1 r), grad = -PSF * (N'^-1 r), r = d - PSF * sky;
        with want_ninv_resid=True also returns N'^-1 r (the gradient with respect to d)."""
        torch = _torch()
        batch, shape = self._batch_shape(sky)
        if grad is None:
            grad = torch.empty(shape, dtype=torch.float32, device=sky.device)
        val = np.zeros(batch, dtype=np.float64)
        nr = torch.empty(shape, dtype=torch.float32, device=sky.device) if want_ninv_resid else None
        check(load().fr_fast_likelihood_grad_resid(
            self._h, _dev(sky, torch.float32, shape, "sky"), _dev(dirty, torch.float32, shape, "dirty"),
            batch, _dev(grad, torch.float32, shape, "grad"),
            _dev(nr, torch.float32, shape, "ninv_resid") if nr is not None else None,
            val.ctypes.data if want_value else None, _stream_ptr(stream)))
        if want_ninv_resid:
            return (val if want_value else None), grad, nr
        return (val if want_value else None), grad

    def _batch_shape(self, sky):
        if sky.dim() == 3:
            return 1, tuple(sky.shape)
        if sky.dim() == 4:
            return int(sky.shape[0]), tuple(sky.shape)
        raise ValueError("sky must be [nsky, nx, ny] or [batch, nsky, nx, ny]")


def _has_cuda() -> bool:
    try:
        return _torch().cuda.is_available()
    except Exception:
        return False
