"""PyTorch front end of the gbfft library.

PyTorch supplies device memory (the caching allocator) and streams; every
transform runs in libgbfft.so's CUDA kernels, reached through the C ABI with
raw device pointers.  Functions here:

  fft(x), ifft(x)           1D transforms over the last axis (Eq. E2 / Eq. E3)
  fft2_filter_ifft2(img, H) the Sec. 5 pipeline, differentiable in img and H
  fft2_filter_ifft2_padded  the same for any image size (zero padding, crop)
  fft2_spectrum(img)        the Sec. 5 spectrum display |fft2(img)|
  fft2_filter_ifft2_analytic  the pipeline with a Gaussian, Butterworth or disc filter by formula
  Plan1D, Plan2D            explicit plans (workspace owned by a torch tensor)
"""

from __future__ import annotations

import ctypes
import threading

import torch

from . import _native as nat

_P = ctypes.c_void_p


def _stream_handle(device: torch.device) -> _P:
    return _P(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: torch.Tensor) -> _P:
    return _P(t.data_ptr())


def _require_cuda(t: torch.Tensor, what: str) -> None:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor (gbfft has no CPU path)")


class _TuneArgs(ctypes.Structure):
    """gbfft_tune_args: the device buffers fft_plan_autotune runs a plan on."""

    _fields_ = [("in_", _P), ("H", _P), ("out", _P)]


class _PlanBase:
    """Owns a gbfft plan handle and its workspace tensor."""

    def __init__(self, handle: _P, device: torch.device, options: dict[int, int] | None):
        self.handle = handle
        self.device = device
        for key, value in (options or {}).items():
            nat.call("fft_plan_set_option", self.handle, int(key), int(value))
        nbytes = ctypes.c_size_t(0)
        nat.call("fft_plan_workspace_bytes", self.handle, ctypes.byref(nbytes))
        self.workspace_bytes = int(nbytes.value)
        with torch.cuda.device(device):
            # 256-byte aligned by the caching allocator
            self.workspace = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=device)
            nat.call("fft_plan_bind_workspace", self.handle, _ptr(self.workspace), self.workspace.numel(),
                     _stream_handle(device))
            # twiddle tables must be complete before another stream uses the plan
            torch.cuda.current_stream(device).synchronize()
        self.lock = threading.Lock()

    def set_option(self, key: int, value: int) -> None:
        nat.call("fft_plan_set_option", self.handle, int(key), int(value))

    def device_status(self) -> None:
        """Raise if a kernel of this plan gave up a bounded wait (synchronous)."""
        nat.call("gbfft_device_status", self.handle)

    def selftest_wait_timeout(self, polls: int = 1 << 16) -> None:
        """Launch the diagnostic block whose bounded wait runs out (sets this
        plan's device status word; see gbfft_selftest_wait_timeout)."""
        nat.call("gbfft_selftest_wait_timeout", self.handle, polls, _stream_handle(self.device))

    def get_option(self, key: int) -> int:
        v = ctypes.c_int64()
        nat.call("fft_plan_get_option", self.handle, int(key), ctypes.byref(v))
        return int(v.value)

    def check_guards(self) -> int:
        """Words changed in the workspace's guard bands (0 = none; synchronous)."""
        n = ctypes.c_int64()
        nat.call("gbfft_plan_check_guards", self.handle, ctypes.byref(n))
        return int(n.value)

    def _autotune(self, x: torch.Tensor, H: torch.Tensor | None, out: torch.Tensor) -> None:
        args = _TuneArgs(_P(x.data_ptr()), _P(H.data_ptr()) if H is not None else _P(), _P(out.data_ptr()))
        with self.lock:
            nat.call("fft_plan_autotune", self.handle, ctypes.byref(args), _stream_handle(self.device))

    def profile_read(self) -> dict[str, tuple[float, int]]:
        n = len(nat.STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        nat.call("gbfft_plan_profile_read", self.handle, ms, cnt, n)
        return {name: (ms[i], cnt[i]) for i, name in enumerate(nat.STAGES) if cnt[i]}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and nat.lib is not None:
            nat.lib.fft_plan_destroy(h)
            self.handle = None


class Plan1D(_PlanBase):
    """Batched 1D C2C plan: `batch` contiguous transforms of length n = 2^m."""

    def __init__(self, n: int, batch: int, dtype: torch.dtype, device, options=None):
        code = {torch.complex64: nat.C64, torch.complex128: nat.C128}.get(dtype)
        if code is None:
            raise TypeError(f"unsupported dtype {dtype}; use complex64 or complex128")
        h = _P()
        nat.call("fft_plan_create", int(n), int(batch), code, ctypes.byref(h))
        self.n, self.batch, self.dtype = int(n), int(batch), dtype
        super().__init__(h, torch.device(device), options)

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        return self._run("fft_forward", x, out)

    def inverse(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        return self._run("fft_inverse", x, out)

    def autotune(self, x: torch.Tensor, out: torch.Tensor | None = None) -> int:
        """Time the plan's candidate paths on x (forward transforms into out)
        and keep the fastest (cached per GPU and shape); returns
        GBFFT_OPT_ONCHIP as chosen."""
        if out is None:
            out = torch.empty_like(x)
        self._autotune(x, None, out)
        return self.get_option(nat.OPT_ONCHIP)

    def _run(self, fn: str, x: torch.Tensor, out: torch.Tensor | None) -> torch.Tensor:
        if x.dtype != self.dtype or x.numel() != self.n * self.batch or not x.is_contiguous():
            raise ValueError("input does not match the plan (dtype, size, contiguity)")
        if out is None:
            out = torch.empty_like(x)
        with self.lock:
            nat.call(fn, self.handle, _ptr(x), _ptr(out), _stream_handle(x.device))
        return out


class Plan2D(_PlanBase):
    """Sec. 5 pipeline plan for `batch` float32 images of rows x cols."""

    def __init__(self, rows: int, cols: int, batch: int, device, options=None):
        h = _P()
        nat.call("fft2_plan_create", int(rows), int(cols), int(batch), nat.C64, ctypes.byref(h))
        self.rows, self.cols, self.batch = int(rows), int(cols), int(batch)
        self.h_stride = int((options or {}).get(nat.OPT_H_BATCH_STRIDE, 0))
        super().__init__(h, torch.device(device), options)

    def filter(self, img: torch.Tensor, H: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty_like(img)
        with self.lock:
            nat.call("fft2_filter_ifft2", self.handle, _ptr(img), _ptr(H), _ptr(out), _stream_handle(img.device))
        return out

    def prepare_filter(self, H: torch.Tensor) -> None:
        """Prepare one filter for filter_prepared() calls (fft2_filter_prepare):
        the filter of a stack of images, prepared once."""
        _require_cuda(H, "H")
        with self.lock:
            nat.call("fft2_filter_prepare", self.handle, _ptr(H), _stream_handle(H.device))

    def filter_prepared(self, img: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """filter() with the filter of the last prepare_filter()
        (fft2_filter_ifft2_prepared; raises if it was discarded since)."""
        if out is None:
            out = torch.empty_like(img)
        with self.lock:
            nat.call("fft2_filter_ifft2_prepared", self.handle, _ptr(img), _ptr(out), _stream_handle(img.device))
        return out

    def autotune(self, img: torch.Tensor, H: torch.Tensor, out: torch.Tensor | None = None) -> dict[str, int]:
        """Time the plan's candidate configurations on these buffers and keep
        the fastest (cached per GPU and shape); returns the chosen options."""
        if out is None:
            out = torch.empty_like(img)
        self._autotune(img, H, out)
        return {"column_form": self.get_option(nat.OPT_COLUMN_FORM), "onchip": self.get_option(nat.OPT_ONCHIP)}

    def filter_padded(self, img: torch.Tensor, H: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Images [..., r, c] with r <= rows, c <= cols, zero-padded to the
        plan's grid, filtered with H (on the grid), cut back to r x c."""
        if out is None:
            out = torch.empty_like(img)
        with self.lock:
            nat.call("fft2_filter_ifft2_padded", self.handle, _ptr(img), int(img.shape[-2]), int(img.shape[-1]),
                     _ptr(H), _ptr(out), _stream_handle(img.device))
        return out

    def filter_analytic(self, img: torch.Tensor, kind: int, p0: float, p1: float = 0.0,
                        out: torch.Tensor | None = None) -> torch.Tensor:
        """The pipeline with an analytic filter computed in the column pass
        (nat.FILTER_GAUSSIAN: p0 = sigma; FILTER_BUTTERWORTH: p0 = order,
        p1 = cutoff in bins; FILTER_DISC: p0 = radius of Eq. filtro)."""
        if out is None:
            out = torch.empty_like(img)
        with self.lock:
            nat.call("fft2_filter_ifft2_analytic", self.handle, _ptr(img), int(kind), float(p0), float(p1), _ptr(out),
                     _stream_handle(img.device))
        return out

    def spectrum(self, img: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """|fft2| of images [..., r, c] zero-padded to the plan's grid:
        [..., rows, cols] float32 in natural frequency order."""
        if out is None:
            out = torch.empty(img.shape[:-2] + (self.rows, self.cols), dtype=torch.float32, device=img.device)
        with self.lock:
            nat.call("fft2_spectrum", self.handle, _ptr(img), int(img.shape[-2]), int(img.shape[-1]), _ptr(out),
                     _stream_handle(img.device))
        return out

    def backward(self, img, H, grad_out, grad_img=None, grad_H=None):
        with self.lock:
            nat.call("fft2_filter_ifft2_backward", self.handle, _ptr(img), _ptr(H), _ptr(grad_out),
                     _ptr(grad_img) if grad_img is not None else _P(),
                     _ptr(grad_H) if grad_H is not None else _P(), _stream_handle(img.device))
        return grad_img, grad_H


class Plan2DBatched(_PlanBase):
    """Sec. 5 pipeline over images of uneven power-of-two sizes (16..4096 per
    side), each with its own filter: the one-shape kernels once per shape
    class (default), or four persistent launches over all images
    (GBFFT_OPT_BATCH_FORM = 1); optionally replayed from a CUDA graph.
    `shapes` is a list of (rows, cols)."""

    def __init__(self, shapes, device, options=None):
        n = len(shapes)
        rows = (ctypes.c_int64 * n)(*[int(r) for r, _ in shapes])
        cols = (ctypes.c_int64 * n)(*[int(c) for _, c in shapes])
        h = _P()
        nat.call("fft2_batched_plan_create", n, rows, cols, ctypes.byref(h))
        self.shapes = [(int(r), int(c)) for r, c in shapes]
        super().__init__(h, torch.device(device), options)
        # device array of gbfft_image_ptrs {img, H, out}; its address stays fixed
        # so a captured graph keeps reading the current pointers
        self.ptrs = torch.zeros(n, 3, dtype=torch.int64, device=self.device)
        self._last_table = None  # the pointers the device array holds
        self._bound = None  # the buffers of bind(), kept alive for run()

    def _set_pointers(self, imgs, Hs, outs):
        if not (len(imgs) == len(Hs) == len(outs) == len(self.shapes)):
            raise ValueError("one image, filter and output per planned shape")
        table = []
        for (r, c), a, h, o in zip(self.shapes, imgs, Hs, outs):
            for t in (a, h, o):
                if t.dtype != torch.float32 or tuple(t.shape[-2:]) != (r, c) or not t.is_contiguous() or not t.is_cuda:
                    raise ValueError(f"expected contiguous float32 CUDA tensors of shape ({r}, {c})")
            table.append((a.data_ptr(), h.data_ptr(), o.data_ptr()))
        if table != self._last_table:  # the same buffers as last call: the array already holds them
            self.ptrs.copy_(torch.tensor(table, dtype=torch.int64), non_blocking=False)
            self._last_table = table

    def filter(self, imgs, Hs, outs=None):
        if outs is None:
            outs = [torch.empty_like(a) for a in imgs]
        with self.lock:
            self._bound = None
            self._set_pointers(imgs, Hs, outs)
            nat.call("fft2_filter_ifft2_batched", self.handle, _ptr(self.ptrs), _stream_handle(self.device))
        return outs

    def bind(self, imgs, Hs, outs):
        """Check and record the buffers once; run() then filters them again
        with no per-call checks (fixed input and output buffers, as in a
        serving loop).  The buffers must stay alive while bound."""
        with self.lock:
            self._set_pointers(imgs, Hs, outs)
            self._bound = (imgs, Hs, outs)

    def run(self):
        """The pipeline over the buffers of the last bind() (a filter() call
        in between unbinds them)."""
        if self._bound is None:
            raise RuntimeError("run() needs buffers: call bind() first")
        with self.lock:
            nat.call("fft2_filter_ifft2_batched", self.handle, _ptr(self.ptrs), _stream_handle(self.device))

    def autotune(self, imgs, Hs, outs=None):
        """Time the launch shapes on these inputs and keep the fastest."""
        if outs is None:
            outs = [torch.empty_like(a) for a in imgs]
        with self.lock:
            self._bound = None
            self._set_pointers(imgs, Hs, outs)
            nat.call("fft_plan_autotune", self.handle, _ptr(self.ptrs), _stream_handle(self.device))
        return self.get_option(nat.OPT_BLOCKS_PER_SM)

    def get_option(self, key: int) -> int:
        v = ctypes.c_int64()
        nat.call("fft_plan_get_option", self.handle, int(key), ctypes.byref(v))
        return int(v.value)


class Plan2DSlab(_PlanBase):
    """One rank's share of an image decomposed by rows over `nranks` ranks
    (include/gbfft.h, fft2_slab_*; the maps are in slab.py).  The three calls
    run this rank's kernels; the two exchanges between them are the caller's."""

    def __init__(self, rows: int, cols: int, nranks: int, rank: int, device, options=None):
        h = _P()
        nat.call("fft2_slab_plan_create", int(rows), int(cols), int(nranks), int(rank), ctypes.byref(h))
        self.rows, self.cols, self.nranks, self.rank = int(rows), int(cols), int(nranks), int(rank)
        super().__init__(h, torch.device(device), options)
        n = ctypes.c_int64()
        nat.call("fft2_slab_exchange_elems", self.handle, ctypes.byref(n))
        self.exchange_elems = int(n.value)

    def exchange_buffer(self) -> torch.Tensor:
        return torch.empty(self.exchange_elems, dtype=torch.complex64, device=self.device)

    def rows_forward(self, img: torch.Tensor, send: torch.Tensor) -> None:
        with self.lock:
            nat.call("fft2_slab_rows_forward", self.handle, _ptr(img), _ptr(send), _stream_handle(self.device))

    def columns(self, recv: torch.Tensor, H: torch.Tensor) -> None:
        with self.lock:
            nat.call("fft2_slab_columns", self.handle, _ptr(recv), _ptr(H), _stream_handle(self.device))

    def rows_inverse(self, back: torch.Tensor, out: torch.Tensor) -> None:
        with self.lock:
            nat.call("fft2_slab_rows_inverse", self.handle, _ptr(back), _ptr(out), _stream_handle(self.device))


def measure_fma_peak(fp64: bool, device=None) -> float:
    """FMA throughput of the GPU in FLOP/s (2 per FMA), double or single
    precision, measured by the library's diagnostic kernel."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    v = ctypes.c_double()
    with torch.cuda.device(dev):
        nat.call("gbfft_measure_fma_peak", 1 if fp64 else 0, ctypes.byref(v), _stream_handle(dev))
    return float(v.value)


_cache: dict[tuple, _PlanBase] = {}
_cache_lock = threading.Lock()


def _cached(key, make):
    with _cache_lock:
        p = _cache.get(key)
        if p is None:
            p = make()
            _cache[key] = p
        return p


def clear_plan_cache() -> None:
    with _cache_lock:
        _cache.clear()


def _plan1d(x: torch.Tensor) -> Plan1D:
    n = x.shape[-1]
    batch = x.numel() // n
    key = ("1d", n, batch, x.dtype, x.device)
    return _cached(key, lambda: Plan1D(n, batch, x.dtype, x.device))


def fft(x: torch.Tensor) -> torch.Tensor:
    """c = (1/N) sum_j x_j exp(-2 pi i jk/N) over the last axis (Eq. E2)."""
    _require_cuda(x, "x")
    x = x.contiguous()
    return _plan1d(x).forward(x)


def ifft(c: torch.Tensor) -> torch.Tensor:
    """f = sum_k c_k exp(+2 pi i jk/N) over the last axis, unscaled (Eq. E3)."""
    _require_cuda(c, "c")
    c = c.contiguous()
    return _plan1d(c).inverse(c)


def _plan2d(img: torch.Tensor, per_image_H: bool, backward: bool = False) -> Plan2D:
    rows, cols = img.shape[-2:]
    batch = img.numel() // (rows * cols)
    opts = {nat.OPT_H_BATCH_STRIDE: rows * cols if per_image_H else 0}
    if backward:
        opts[nat.OPT_ENABLE_BACKWARD] = 1
    key = ("2d", rows, cols, batch, per_image_H, backward, img.device)
    return _cached(key, lambda: Plan2D(rows, cols, batch, img.device, opts))


def _check_2d(img: torch.Tensor, H: torch.Tensor) -> bool:
    _require_cuda(img, "img")
    _require_cuda(H, "H")
    if img.dtype != torch.float32 or H.dtype != torch.float32:
        raise TypeError("img and H must be float32")
    if img.dim() < 2:
        raise ValueError("img must be [..., rows, cols]")
    if H.shape == img.shape[-2:]:
        return False
    if H.shape == img.shape:
        return True
    raise ValueError(f"H shape {tuple(H.shape)} must be {tuple(img.shape[-2:])} or {tuple(img.shape)}")


class _FilterFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, img, H):
        per_image = _check_2d(img, H)
        img_c, H_c = img.contiguous(), H.contiguous()
        out = _plan2d(img_c, per_image).filter(img_c, H_c)
        ctx.save_for_backward(img_c, H_c)
        ctx.per_image = per_image
        return out

    @staticmethod
    def backward(ctx, grad_out):
        img, H = ctx.saved_tensors
        g = grad_out.contiguous()
        need_img, need_H = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        plan = _plan2d(img, ctx.per_image, backward=need_H and not ctx.per_image)
        if ctx.per_image:
            if need_H:
                raise NotImplementedError("grad of a per-image filter stack is not supported; share one H")
            # the adjoint of the pipeline is the pipeline itself (real H)
            return plan.filter(g, H), None
        grad_img = torch.empty_like(img) if need_img else None
        grad_H = torch.empty_like(H) if need_H else None
        plan.backward(img, H, g, grad_img, grad_H)
        return grad_img, grad_H


def fft2_filter_ifft2_batched(imgs, Hs):
    """Sec. 5 pipeline over a list of float32 images of (possibly) different
    power-of-two shapes, each with its own filter; returns a list of outputs.
    Not differentiable; the plan is cached per list of shapes and device."""
    if len(imgs) != len(Hs) or not imgs:
        raise ValueError("need one filter per image")
    for a, h in zip(imgs, Hs):
        _check_2d(a, h)
    dev = imgs[0].device
    shapes = tuple((int(a.shape[-2]), int(a.shape[-1])) for a in imgs)
    plan = _cached(("batched", shapes, dev), lambda: Plan2DBatched(shapes, dev))
    return plan.filter([a.contiguous() for a in imgs], [h.contiguous() for h in Hs])


def _next_pow2(n: int) -> int:
    return 1 << max(0, int(n) - 1).bit_length()


def fft2_filter_ifft2_padded(img: torch.Tensor, H: torch.Tensor) -> torch.Tensor:
    """Sec. 5 application path for any image size: float32 images
    [..., r, c] are zero-padded (after the last row and column) to the filter's
    grid H [R, C] (powers of two, R >= r, C >= c; or one filter per image,
    [..., R, C]), filtered, and cut back to r x c.  Not differentiable."""
    _require_cuda(img, "img")
    _require_cuda(H, "H")
    if img.dtype != torch.float32 or H.dtype != torch.float32 or img.dim() < 2:
        raise TypeError("img and H must be float32, img [..., rows, cols]")
    R, C = int(H.shape[-2]), int(H.shape[-1])
    per_image = H.dim() > 2
    if per_image and H.shape[:-2] != img.shape[:-2]:
        raise ValueError("per-image filters must match the batch dimensions of img")
    r, c = int(img.shape[-2]), int(img.shape[-1])
    batch = img.numel() // (r * c)
    opts = {nat.OPT_H_BATCH_STRIDE: R * C if per_image else 0}
    plan = _cached(("2dpad", R, C, batch, per_image, img.device), lambda: Plan2D(R, C, batch, img.device, opts))
    return plan.filter_padded(img.contiguous(), H.contiguous())


def fft2_filter_ifft2_analytic(img: torch.Tensor, kind: int, p0: float, p1: float = 0.0) -> torch.Tensor:
    """Sec. 5 pipeline on float32 images [..., rows, cols] with a filter given
    by formula (Gaussian, Butterworth or the disc of Eq. filtro; see
    Plan2D.filter_analytic), computed in the column pass.  Not differentiable."""
    _require_cuda(img, "img")
    if img.dtype != torch.float32 or img.dim() < 2:
        raise TypeError("img must be float32 [..., rows, cols]")
    rows, cols = int(img.shape[-2]), int(img.shape[-1])
    batch = img.numel() // (rows * cols)
    plan = _cached(("2dan", rows, cols, batch, img.device), lambda: Plan2D(rows, cols, batch, img.device))
    return plan.filter_analytic(img.contiguous(), kind, p0, p1)


def fft2_spectrum(img: torch.Tensor, rows: int | None = None, cols: int | None = None,
                  eq5: bool = False) -> torch.Tensor:
    """Spectrum display of Sec. 5: sqrt(Re^2 + Im^2) of the 2D transform of
    float32 images [..., r, c] zero-padded to rows x cols (default: the next
    powers of two), natural frequency order; per-axis scale (the DFT divided by
    rows * cols), or Eq. 5's (divided by rows) with eq5=True."""
    _require_cuda(img, "img")
    if img.dtype != torch.float32 or img.dim() < 2:
        raise TypeError("img must be float32 [..., rows, cols]")
    r, c = int(img.shape[-2]), int(img.shape[-1])
    R = int(rows) if rows is not None else _next_pow2(r)
    C = int(cols) if cols is not None else _next_pow2(c)
    batch = img.numel() // (r * c)
    opts = {nat.OPT_SCALE_CONVENTION: 1 if eq5 else 0}
    plan = _cached(("2dspec", R, C, batch, bool(eq5), img.device), lambda: Plan2D(R, C, batch, img.device, opts))
    return plan.spectrum(img.contiguous())


def fft2_filter_ifft2(img: torch.Tensor, H: torch.Tensor) -> torch.Tensor:
    """Sec. 5: Re(ifft2(H * fft2(img))) for float32 images [..., rows, cols].

    H is a real float32 filter [rows, cols] (shared) or one per image (same
    shape as img), in natural (unshifted) DFT order.  Differentiable in img
    and (for a shared H) in H.
    """
    return _FilterFn.apply(img, H)


def fft2_filter_ifft2_sharded(img: torch.Tensor, H: torch.Tensor, group=None, nranks: int | None = None,
                              out: torch.Tensor | None = None) -> torch.Tensor:
    """Sec. 5 pipeline on one float32 image [rows, cols] decomposed by rows.

    With a torch.distributed `group` (one rank per GPU, NCCL): every rank
    passes the whole-image buffers `img` and `out` (only its own rows, see
    slab.slab_rows, are read and written; the other rows of `out` are left
    as they are) and the whole filter H; the two exchanges are
    all_to_all_single calls of equal chunks.  Without a group, `nranks` ranks
    are emulated on img's device, one after the other, with the exchanges
    done as local copies; then every row of `out` is written.  Equals
    fft2_filter_ifft2(img, H).  Not differentiable."""
    _check_2d(img, H)
    if img.dim() != 2 or H.shape != img.shape:
        raise ValueError("one image [rows, cols] and one filter of the same shape")
    rows, cols = int(img.shape[0]), int(img.shape[1])
    img, H = img.contiguous(), H.contiguous()
    if out is None:
        out = torch.empty_like(img)
    dev = img.device
    if group is not None:
        import torch.distributed as dist

        from . import slab

        R, r = dist.get_world_size(group), dist.get_rank(group)
        plan = _cached(("slab", rows, cols, R, r, dev), lambda: Plan2DSlab(rows, cols, R, r, dev))
        send, recv = plan.exchange_buffer(), plan.exchange_buffer()
        plan.rows_forward(img, send)
        slab.exchange(send, recv, group)
        plan.columns(recv, H)
        slab.exchange(recv, send, group)
        plan.rows_inverse(send, out)
        return out
    R = int(nranks or 1)
    plans = [_cached(("slab", rows, cols, R, r, dev), lambda r=r: Plan2DSlab(rows, cols, R, r, dev))
             for r in range(R)]
    n = plans[0].exchange_elems
    sends = torch.empty(R, R, n // R, dtype=torch.complex64, device=dev)  # [rank][chunk]
    for r, p in enumerate(plans):
        p.rows_forward(img, sends[r])
    recvs = sends.transpose(0, 1).contiguous()  # rank q receives chunk q of every rank, in rank order
    for q, p in enumerate(plans):
        p.columns(recvs[q], H)
    backs = recvs.transpose(0, 1).contiguous()  # and sends chunk r back to rank r
    for r, p in enumerate(plans):
        p.rows_inverse(backs[r], out)
    return out
