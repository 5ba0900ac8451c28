"""ctypes binding over the C ABI in include/sfft.h, include/rb.h and include/phot.h.

Argument marshalling only: every step of the subtraction runs in the CUDA
kernels of libsfft_gb300.so.  PyTorch provides device memory and the stream.
There is no CPU fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsfft_gb300.so")

SFFT_OK, SFFT_ERR_ARG, SFFT_ERR_CUDA, SFFT_ERR_NOMEM = 0, 1, 2, 3
SFFT_ERR_SINGULAR, SFFT_ERR_NONFINITE, SFFT_ERR_TIMEOUT, SFFT_ERR_UNSUPPORTED = 4, 5, 6, 7
PREC = {"fp64": 0, "mixed": 1}
FLAG_GRAPH = 1
FLAG_CONST_RATIO = 2
FLAG_FMA_CONTRACT = 4
FLAG_MMA_SYNC_CONTRACT = 8
FLAG_PAIR_LANE_CONTRACT = 16


class Desc(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("L", C.c_int32), ("DK", C.c_int32), ("DB", C.c_int32),
                ("batch", C.c_int32), ("prec", C.c_int32), ("autotune", C.c_int32), ("d_batch", C.c_int32),
                ("rows_per_cta", C.c_int32), ("lag_parts", C.c_int32), ("flags", C.c_uint32),
                ("ccd_group", C.c_int32)]


VP, I32, I64, SZ, DBL = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.c_double

# name -> (restype, argtypes); every symbol declared in include/*.h
SIGNATURES = {
    "sfft_plan": (I32, [C.POINTER(Desc), VP, C.POINTER(VP)]),
    "sfft_plan_destroy": (None, [VP]),
    "sfft_plan_set_stream": (I32, [VP, VP]),
    "sfft_num_unknowns": (I64, [VP]),
    "sfft_workspace_bytes": (SZ, [VP]),
    "sfft_plan_engine": (I32, [VP]),
    "sfft_plan_tiles": (I32, [VP, C.POINTER(I32)]),
    "sfft_plan_ccd_group": (I32, [VP]),
    "sfft_plan_set_wait_limit": (I32, [VP, I32]),
    "sfft_debug_live_allocations": (I64, []),
    "sfft_probe_fma_peak": (I32, [I32, C.POINTER(C.c_double), VP]),
    "sfft_probe_umma_cycles": (I32, [I32, C.POINTER(C.c_double), VP]),
    "sfft_debug_contract_waits": (I32, [C.POINTER(C.c_uint64), I32]),
    "sfft_build_normal": (I32, [VP, VP, VP, VP, VP, VP, VP, VP]),
    "sfft_solve": (I32, [VP, VP, VP, VP, I32, VP, VP, VP, VP, VP]),
    "sfft_apply": (I32, [VP, VP, VP, VP, VP, VP, VP]),
    "sfft_subtract": (I32, [VP, VP, VP, VP, VP, I32, VP, VP, VP, VP, VP, VP]),
    "sfft_kernel_at": (I32, [VP, VP, DBL, DBL, VP]),
    "sfft_apply_noalloc": (I32, [I32, I32, I32, I32, I32, I32, I32, VP, VP, VP, VP, VP, VP]),
    "sfft_profile_enable": (I32, [VP, I32]),
    "sfft_profile_read": (I32, [VP, C.POINTER(C.c_double), C.POINTER(I64), I32]),
    "sfft_status_str": (C.c_char_p, [I32]),
    "sfft_last_error": (C.c_char_p, []),
    # classifier and detector (include/rb.h)
    "rb_create": (I32, [VP, C.POINTER(VP)]),
    "rb_destroy": (I32, [VP]),
    "rb_set_weights": (I32, [VP, VP, SZ]),
    "rb_get_weights": (I32, [VP, VP, SZ]),
    "rb_get_grads": (I32, [VP, VP, SZ]),
    "rb_get_state": (I32, [VP, VP, SZ, C.POINTER(I64)]),
    "rb_set_state": (I32, [VP, VP, SZ, I64]),
    "rb_logits": (I32, [VP, VP, I64, VP, VP]),
    "rb_score": (I32, [VP, VP, I64, VP, VP]),
    "rb_conv_layer": (I32, [VP, I32, VP, I64, I64, VP, VP]),
    "rb_get_error": (I32, [VP, C.POINTER(I32)]),
    "rb_debug_conv_waits": (I32, [I32, C.POINTER(C.c_uint64), I32]),
    "rb_backward": (I32, [VP, VP, VP, I64, VP, VP]),
    "rb_train_step": (I32, [VP, VP, VP, I64, C.c_float, VP, VP]),
    "rbri_create": (I32, [VP, C.POINTER(VP)]),
    "rbri_destroy": (I32, [VP]),
    "rbri_set_weights": (I32, [VP, VP, SZ]),
    "rbri_get_weights": (I32, [VP, VP, SZ]),
    "rbri_get_grads": (I32, [VP, VP, SZ]),
    "rbri_get_state": (I32, [VP, VP, SZ, C.POINTER(I64)]),
    "rbri_set_state": (I32, [VP, VP, SZ, I64]),
    "rbri_logits": (I32, [VP, VP, I64, VP, VP]),
    "rbri_score": (I32, [VP, VP, I64, VP, VP]),
    "rbri_backward": (I32, [VP, VP, VP, I64, VP, VP]),
    "rbri_train_step": (I32, [VP, VP, VP, I64, C.c_float, VP, VP]),
    "rb_detect_workspace_bytes": (SZ, [I32, I32, I32, I32]),
    "rb_detect": (I32, [I32, I32, I32, VP, VP, VP, VP, C.c_float, C.c_float, I32, I32, VP, VP, VP, VP, VP, VP]),
    "rb_shape_cuts": (I32, [VP, VP, I64, C.c_float, C.c_float, VP, VP]),
    "rb_shape_cuts_adaptive": (I32, [VP, VP, I64, C.c_float, C.c_float, VP, VP]),
    # differential photometry and multi-template combination (include/phot.h)
    "phot_aperture_flux": (I32, [I32, I32, I32, VP, VP, VP, I32, DBL, VP, VP, VP]),
    "phot_limiting_workspace_bytes": (SZ, [I32, I32]),
    "phot_limiting_mag": (I32, [I32, I32, I32, VP, VP, VP, I32, DBL, DBL, VP, VP, VP, VP, VP]),
    "phot_median_combine": (I32, [I32, I32, I32, VP, VP, VP, VP, VP]),
}

RB_STAMP = 31
RB_NPARAM = 130305
RBRI_NPARAM = 185729

_LIB = None


class SfftError(RuntimeError):
    pass


def load(path=LIB_PATH):
    """Load the shared library (once).  Raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise SfftError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(st, what):
    if st != SFFT_OK:
        lib = load()
        msg = lib.sfft_status_str(st).decode()
        err = lib.sfft_last_error().decode()
        raise SfftError(f"{what}: {msg} ({st}) {err}")


def _device(device):
    """A CUDA device with an explicit index (the current device when unspecified)."""
    import torch
    d = torch.device(device) if device is not None else torch.device("cuda")
    return d if d.index is not None else torch.device(d.type, torch.cuda.current_device())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def probe_umma_cycles(n, stream=None):
    """Clock cycles per tcgen05 MMA (BF16, M = 128, K = 16, N = n) with both
    operands in shared memory (include/sfft.h sfft_probe_umma_cycles)."""
    import torch
    lib = load()
    s = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double()
    _check(lib.sfft_probe_umma_cycles(int(n), C.byref(out), VP(s.cuda_stream)), "sfft_probe_umma_cycles")
    return float(out.value)


def probe_fma_peak(fp64=False, stream=None):
    """Measured FMA peak of the current GPU in TFLOP/s (FP32 or FP64)."""
    import torch
    lib = load()
    s = stream if stream is not None else torch.cuda.current_stream()
    v = C.c_double()
    _check(lib.sfft_probe_fma_peak(1 if fp64 else 0, C.byref(v), VP(s.cuda_stream)), "sfft_probe_fma_peak")
    return float(v.value)


def apply_noalloc(R, S, theta, sky, D, L, DK, DB, prec="mixed", stream=None):
    """Difference image through the allocation-free entry point: no plan and no
    workspace; R, S, D are [batch][H][W] float32, theta [batch][N] and sky
    [batch][2] float64, all on the current device.  Writes D in place."""
    import torch
    lib = load()
    B, H, W = D.shape
    s = stream if stream is not None else torch.cuda.current_stream(D.device)
    st = lib.sfft_apply_noalloc(H, W, L, DK, DB, B, PREC[prec], _ptr(R), _ptr(S), _ptr(theta), _ptr(sky), _ptr(D),
                                VP(s.cuda_stream))
    _check(st, "sfft_apply_noalloc")
    return D


class Plan:
    """A subtraction plan plus its workspace (a torch uint8 device tensor).
    const_ratio=True holds the kernel sum constant over the chip
    (SFFT_FLAG_CONST_RATIO); theta keeps the full N-term layout.
    fma_contract=True runs the mixed path's KK contraction on the FP32 FMA
    pipes instead of the tensor cores (SFFT_FLAG_FMA_CONTRACT);
    mma_sync_contract=True keeps it on the tensor cores through warp-level
    mma.sync instead of tcgen05 (SFFT_FLAG_MMA_SYNC_CONTRACT);
    pair_lane_contract=True runs the tcgen05 contraction with one tensor-memory
    lane per (difference, u_y) pair (SFFT_FLAG_PAIR_LANE_CONTRACT).
    ccd_group: CCDs whose product spectra are held at once (0: the plan's choice)."""

    def __init__(self, H, W, L, DK, DB, batch=1, prec="mixed", d_batch=0, rows_per_cta=0, autotune=0,
                 graph=False, stream=None, device=None, lag_parts=0, const_ratio=False, fma_contract=False,
                 mma_sync_contract=False, pair_lane_contract=False, ccd_group=0):
        import torch
        self._torch = torch
        lib = load()
        self.lib = lib
        self.device = _device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.desc = Desc(H, W, L, DK, DB, batch, PREC[prec], autotune, d_batch, rows_per_cta, lag_parts,
                         (FLAG_GRAPH if graph else 0) | (FLAG_CONST_RATIO if const_ratio else 0) |
                         (FLAG_FMA_CONTRACT if fma_contract else 0) |
                         (FLAG_MMA_SYNC_CONTRACT if mma_sync_contract else 0) |
                         (FLAG_PAIR_LANE_CONTRACT if pair_lane_contract else 0), int(ccd_group))
        h = VP()
        with torch.cuda.device(self.device):
            _check(lib.sfft_plan(C.byref(self.desc), VP(self.stream.cuda_stream), C.byref(h)), "sfft_plan")
        self.h = h
        self.H, self.W, self.L, self.DK, self.DB, self.batch = H, W, L, DK, DB, batch
        self.const_ratio = bool(const_ratio)
        self.N = int(lib.sfft_num_unknowns(h))
        self.ws_bytes = int(lib.sfft_workspace_bytes(h))
        self.engine = self.ENGINES[int(lib.sfft_plan_engine(h))]
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_view = self.ws[off:off + self.ws_bytes]
        t = (I32 * 3)()
        _check(lib.sfft_plan_tiles(h, t), "sfft_plan_tiles")
        self.tiles = tuple(int(v) for v in t)
        self.ccd_group = int(lib.sfft_plan_ccd_group(h))

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.sfft_plan_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def set_wait_limit(self, tries):
        """Polls before the factorisation's grid-barrier wait gives up (< 0: the default, about a second)."""
        _check(self.lib.sfft_plan_set_wait_limit(self.h, int(tries)), "sfft_plan_set_wait_limit")

    def set_stream(self, stream):
        self.stream = stream
        _check(self.lib.sfft_plan_set_stream(self.h, VP(stream.cuda_stream)), "sfft_plan_set_stream")

    # -- helpers
    def _f64(self, *shape):
        return self._torch.empty(*shape, dtype=self._torch.float64, device=self.device)

    def _check_img(self, x, dtype):
        t = self._torch
        if x is None:
            return None
        if x.device != self.device or x.dtype != dtype or not x.is_contiguous():
            raise ValueError(f"expected a contiguous {dtype} tensor on {self.device}")
        if x.numel() != self.batch * self.H * self.W:
            raise ValueError("image shape does not match the plan")
        return x

    # -- entry points
    def build_normal(self, R, S, bad=None, sky=None, A=None, b=None):
        t = self._torch
        R = self._check_img(R, t.float32)
        S = self._check_img(S, t.float32)
        bad = self._check_img(bad, t.uint8)
        A = A if A is not None else self._f64(self.batch, self.N, self.N)
        b = b if b is not None else self._f64(self.batch, self.N)
        st = self.lib.sfft_build_normal(self.h, _ptr(R), _ptr(S), _ptr(bad), _ptr(sky), _ptr(A), _ptr(b),
                                        _ptr(self.ws_view))
        _check(st, "sfft_build_normal")
        return A, b

    def solve(self, A, b, R=None, S=None, bad=None, refine=1, theta=None, info=None):
        t = self._torch
        theta = theta if theta is not None else self._f64(self.batch, self.N)
        info = info if info is not None else t.empty(self.batch, dtype=t.int32, device=self.device)
        st = self.lib.sfft_solve(self.h, _ptr(A), _ptr(b), _ptr(theta), int(refine), _ptr(R), _ptr(S), _ptr(bad),
                                 _ptr(info), _ptr(self.ws_view))
        _check(st, "sfft_solve")
        return theta, info

    def apply(self, R, S, theta, sky=None, D=None):
        t = self._torch
        D = D if D is not None else t.empty(self.batch, self.H, self.W, dtype=t.float32, device=self.device)
        st = self.lib.sfft_apply(self.h, _ptr(R), _ptr(S), _ptr(theta), _ptr(sky), _ptr(D), _ptr(self.ws_view))
        _check(st, "sfft_apply")
        return D

    def subtract(self, R, S, bad=None, sky=None, refine=1, out=None):
        """build_normal + solve + apply; `out` may carry preallocated A, b, theta, info, D."""
        t = self._torch
        R = self._check_img(R, t.float32)
        S = self._check_img(S, t.float32)
        bad = self._check_img(bad, t.uint8)
        o = dict(out) if out else {}
        o.setdefault("A", self._f64(self.batch, self.N, self.N))
        o.setdefault("b", self._f64(self.batch, self.N))
        o.setdefault("theta", self._f64(self.batch, self.N))
        o.setdefault("info", t.empty(self.batch, dtype=t.int32, device=self.device))
        o.setdefault("D", t.empty(self.batch, self.H, self.W, dtype=t.float32, device=self.device))
        st = self.lib.sfft_subtract(self.h, _ptr(R), _ptr(S), _ptr(bad), _ptr(sky), int(refine), _ptr(o["A"]),
                                    _ptr(o["b"]), _ptr(o["theta"]), _ptr(o["info"]), _ptr(o["D"]),
                                    _ptr(self.ws_view))
        _check(st, "sfft_subtract")
        return o

    PROF_PHASES = ("prep", "fft_weights", "fft_prod", "contract_kk", "contract_rk", "scatter", "solve", "apply",
                   "lag_dft")
    ENGINES = ("fp64_fma", "fp32_fma", "mma_sync", "tcgen05_pair_lane", "tcgen05_difference_lane")

    def profile(self, enable=True):
        _check(self.lib.sfft_profile_enable(self.h, 1 if enable else 0), "sfft_profile_enable")

    def profile_read(self, reset=True):
        """{phase: (milliseconds, kernel launches)} accumulated since the last reset."""
        ms = (C.c_double * len(self.PROF_PHASES))()
        n = (I64 * len(self.PROF_PHASES))()
        _check(self.lib.sfft_profile_read(self.h, ms, n, 1 if reset else 0), "sfft_profile_read")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.PROF_PHASES)}

    def kernel_at(self, theta, x, y):
        K = self._f64(self.batch, self.L * self.L)
        _check(self.lib.sfft_kernel_at(self.h, _ptr(theta), float(x), float(y), _ptr(K)), "sfft_kernel_at")
        return K.view(self.batch, self.L, self.L)


def _stream(t, stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(t.device)
    return VP(s.cuda_stream)


def _need(t, dtype, what):
    if t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous {dtype} CUDA tensor")
    return t


class RBModel:
    """The stamp classifier: FP32 master weights and Adam state on the device,
    BF16 tensor-core forward/backward.  Weight vectors use the layout of
    include/rb.h (w1 b1 ... w5 b5, RB_NPARAM floats)."""

    PREFIX = "rb"
    NPARAM = RB_NPARAM

    def __init__(self, max_batch=1024, seed=0):
        import numpy as np
        self._np = np
        self.lib = load()
        desc = (I32 * 2)(int(max_batch), int(seed))
        h = VP()
        _check(self._fn("create")(desc, C.byref(h)), f"{self.PREFIX}_create")
        self.h = h
        self.max_batch = int(max_batch)

    def _fn(self, name):
        return getattr(self.lib, f"{self.PREFIX}_{name}")

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self._fn("destroy")(self.h)
                self.h = None
        except Exception:
            pass

    def _vec(self, name):
        out = self._np.empty(self.NPARAM, dtype=self._np.float32)
        _check(self._fn(name)(self.h, out.ctypes.data_as(VP), out.nbytes), f"{self.PREFIX}_{name}")
        return out

    def set_weights(self, w):
        w = self._np.ascontiguousarray(w, dtype=self._np.float32)
        if w.size != self.NPARAM:
            raise ValueError(f"expected {self.NPARAM} weights")
        _check(self._fn("set_weights")(self.h, w.ctypes.data_as(VP), w.nbytes), f"{self.PREFIX}_set_weights")

    def get_weights(self):
        return self._vec("get_weights")

    def get_grads(self):
        return self._vec("get_grads")

    def get_state(self):
        """(weights, adam_m, adam_v) as one array of 3 * NPARAM floats, and the step count."""
        out = self._np.empty(3 * self.NPARAM, dtype=self._np.float32)
        step = I64()
        _check(self._fn("get_state")(self.h, out.ctypes.data_as(VP), out.nbytes, C.byref(step)),
               f"{self.PREFIX}_get_state")
        return out, int(step.value)

    def set_state(self, state, step):
        s = self._np.ascontiguousarray(state, dtype=self._np.float32)
        _check(self._fn("set_state")(self.h, s.ctypes.data_as(VP), s.nbytes, int(step)), f"{self.PREFIX}_set_state")

    def logits(self, stamps, out=None, stream=None):
        import torch
        _need(stamps, torch.float32, "stamps")
        n = stamps.shape[0]
        out = out if out is not None else torch.empty(n, dtype=torch.float32, device=stamps.device)
        _check(self._fn("logits")(self.h, _ptr(stamps), n, _ptr(out), _stream(stamps, stream)),
               f"{self.PREFIX}_logits")
        return out

    def score(self, stamps, out=None, stream=None):
        import torch
        _need(stamps, torch.float32, "stamps")
        n = stamps.shape[0]
        out = out if out is not None else torch.empty(n, dtype=torch.float32, device=stamps.device)
        _check(self._fn("score")(self.h, _ptr(stamps), n, _ptr(out), _stream(stamps, stream)), f"{self.PREFIX}_score")
        return out

    def conv_layer(self, layer, inp, n, n_alloc, out, stream=None):
        """One fused inference convolution (include/rb.h rb_conv_layer) on
        BF16 CUDA tensors: layer 1 reads NHWC stamps, layers 2 and 3 read
        channel-block planes of n_alloc stamps; writes `out` in place."""
        import torch
        if self.PREFIX != "rb":
            raise NotImplementedError("conv_layer: the three-convolution classifier only")
        _need(inp, torch.bfloat16, "inp")
        _need(out, torch.bfloat16, "out")
        _check(self._fn("conv_layer")(self.h, int(layer), _ptr(inp), int(n), int(n_alloc), _ptr(out),
                                      _stream(inp, stream)), "rb_conv_layer")
        return out

    def error_flags(self):
        """Sticky error flags of the model's tensor-core kernels (synchronous)."""
        if self.PREFIX != "rb":
            raise NotImplementedError("error_flags: the three-convolution classifier only")
        v = I32()
        _check(self._fn("get_error")(self.h, C.byref(v)), "rb_get_error")
        return int(v.value)

    def backward(self, stamps, labels, loss=None, stream=None):
        import torch
        _need(stamps, torch.float32, "stamps")
        _need(labels, torch.float32, "labels")
        loss = loss if loss is not None else torch.empty(1, dtype=torch.float32, device=stamps.device)
        _check(self._fn("backward")(self.h, _ptr(stamps), _ptr(labels), stamps.shape[0], _ptr(loss),
                                    _stream(stamps, stream)), f"{self.PREFIX}_backward")
        return loss

    def train_step(self, stamps, labels, lr, loss=None, stream=None):
        import torch
        _need(stamps, torch.float32, "stamps")
        _need(labels, torch.float32, "labels")
        loss = loss if loss is not None else torch.empty(1, dtype=torch.float32, device=stamps.device)
        _check(self._fn("train_step")(self.h, _ptr(stamps), _ptr(labels), stamps.shape[0], float(lr), _ptr(loss),
                                      _stream(stamps, stream)), f"{self.PREFIX}_train_step")
        return loss


class RIModel(RBModel):
    """The paper's rotation-invariant residual classifier (include/rb.h rbri_*):
    the same interface as RBModel, RBRI_NPARAM weights in the order w1 b1 wa ba
    wb bb w2 b2 wc bc wd bd w4 b4 w5 b5; at most 2048 stamps per internal batch."""

    PREFIX = "rbri"
    NPARAM = RBRI_NPARAM

    def __init__(self, max_batch=512, seed=0):
        super().__init__(max_batch=max_batch, seed=seed)


class Detector:
    """Matched-filter candidate detection with a reusable workspace.  After a
    call, `snr_map` views the [batch][H][W] SNR image left in the workspace."""

    def __init__(self, H, W, batch=1, max_cand=4096, device=None):
        import torch
        self.lib = load()
        self.H, self.W, self.batch, self.max_cand = H, W, batch, max_cand
        self.device = _device(device)
        nb = int(self.lib.rb_detect_workspace_bytes(H, W, batch, max_cand))
        if nb == 0:
            raise SfftError("rb_detect_workspace_bytes: invalid sizes")
        self.ws = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_view = self.ws[off:off + nb]
        self.xy = torch.empty(batch, max_cand, 2, dtype=torch.int32, device=self.device)
        self.snr = torch.empty(batch, max_cand, dtype=torch.float32, device=self.device)
        self.count = torch.empty(batch, dtype=torch.int32, device=self.device)
        self.stamps = torch.empty(batch, max_cand, 3, RB_STAMP, RB_STAMP, dtype=torch.float32, device=self.device)
        self.snr_map = self.ws_view[:batch * H * W * 4].view(torch.float32).view(batch, H, W)

    def __call__(self, D, S, R, bad=None, psf_sigma=1.0, thresh=5.0, guard=0, stream=None):
        import torch
        for t, name in ((D, "D"), (S, "S"), (R, "R")):
            _need(t, torch.float32, name)
            if t.numel() != self.batch * self.H * self.W:
                raise ValueError(f"{name}: shape does not match the detector")
        if bad is not None:
            _need(bad, torch.uint8, "bad")
        st = self.lib.rb_detect(self.H, self.W, self.batch, _ptr(D), _ptr(S), _ptr(R), _ptr(bad), float(psf_sigma),
                                float(thresh), int(guard), self.max_cand, _ptr(self.xy), _ptr(self.snr), _ptr(self.count),
                                _ptr(self.stamps), _ptr(self.ws_view), _stream(D, stream))
        _check(st, "rb_detect")
        return self.xy, self.snr, self.count, self.stamps


def shape_cuts(stamps, snr, psf_fwhm, snr_min=5.0, out=None, stream=None, adaptive=False):
    """Plain SNR/shape cuts on [n][3][31][31] stamps: int32 pass flags.
    adaptive=True takes the size and axis ratio from Gaussian-weighted adaptive
    moments (rb_shape_cuts_adaptive) instead of the positive 9 x 9's moments."""
    import torch
    _need(stamps, torch.float32, "stamps")
    _need(snr, torch.float32, "snr")
    n = stamps.shape[0]
    out = out if out is not None else torch.empty(n, dtype=torch.int32, device=stamps.device)
    fn = load().rb_shape_cuts_adaptive if adaptive else load().rb_shape_cuts
    _check(fn(_ptr(stamps), _ptr(snr), n, float(psf_fwhm), float(snr_min), _ptr(out), _stream(stamps, stream)),
           "rb_shape_cuts_adaptive" if adaptive else "rb_shape_cuts")
    return out


# ---------------------------------------------------------------- differential photometry
def aperture_flux(D, pos, radius, bad=None, stream=None):
    """Forced aperture fluxes on D [batch][H][W] (float32) at pos [batch][n][2]
    (float64 x, y): returns (flux float64 [batch][n], flag int32 [batch][n])."""
    import torch
    _need(D, torch.float32, "D")
    _need(pos, torch.float64, "pos")
    B, H, W = D.shape
    n = pos.shape[1]
    if bad is not None:
        _need(bad, torch.uint8, "bad")
    flux = torch.empty(B, n, dtype=torch.float64, device=D.device)
    flag = torch.empty(B, n, dtype=torch.int32, device=D.device)
    _check(load().phot_aperture_flux(H, W, B, _ptr(D), _ptr(bad), _ptr(pos), n, float(radius), _ptr(flux),
                                     _ptr(flag), _stream(D, stream)), "phot_aperture_flux")
    return flux, flag


def random_positions(batch, H, W, n=1024, seed=0, margin=16.0, device="cuda"):
    """The Monte Carlo's background positions, drawn on the host from a seeded
    generator (uniform over the image, `margin` px from the edges)."""
    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    xy = np.empty((batch, n, 2))
    xy[..., 0] = rng.uniform(margin, W - 1 - margin, (batch, n))
    xy[..., 1] = rng.uniform(margin, H - 1 - margin, (batch, n))
    return torch.from_numpy(xy).to(device)


def limiting_mag(D, radius, zp, pos=None, bad=None, n=1024, seed=0, stream=None):
    """Per-CCD limiting magnitude from aperture fluxes at random positions:
    returns (sigma, mlim, ngood), each a [batch] tensor."""
    import torch
    _need(D, torch.float32, "D")
    B, H, W = D.shape
    if pos is None:
        pos = random_positions(B, H, W, n, seed, device=D.device)
    _need(pos, torch.float64, "pos")
    n = pos.shape[1]
    lib = load()
    nb = int(lib.phot_limiting_workspace_bytes(B, n))
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=D.device)
    off = (-ws.data_ptr()) % 256
    sigma = torch.empty(B, dtype=torch.float64, device=D.device)
    mlim = torch.empty(B, dtype=torch.float64, device=D.device)
    ngood = torch.empty(B, dtype=torch.int32, device=D.device)
    if bad is not None:
        _need(bad, torch.uint8, "bad")
    _check(lib.phot_limiting_mag(H, W, B, _ptr(D), _ptr(bad), _ptr(pos), n, float(radius), float(zp), _ptr(sigma),
                                 _ptr(mlim), _ptr(ngood), VP(ws.data_ptr() + off), _stream(D, stream)),
           "phot_limiting_mag")
    return sigma, mlim, ngood


def median_combine(D, scale, bad=None, out=None, stream=None):
    """Median over templates of scale[t] D[t] ([ntemp][H][W] float32) at good pixels."""
    import torch
    _need(D, torch.float32, "D")
    _need(scale, torch.float32, "scale")
    T, H, W = D.shape
    if bad is not None:
        _need(bad, torch.uint8, "bad")
    out = out if out is not None else torch.empty(H, W, dtype=torch.float32, device=D.device)
    _check(load().phot_median_combine(H, W, T, _ptr(D), _ptr(scale), _ptr(bad), _ptr(out), _stream(D, stream)),
           "phot_median_combine")
    return out


def multi_template_difference(plan, R, S, bad=None, scale=None, refine=1):
    """Difference one science image against N_TEMP templates and median-combine
    the differences: R [T][H][W] templates, S [H][W] science (float32, on the
    plan's device), bad [T][H][W] or None, scale [T] zero-point factors
    (float32; ones when None).  The plan's batch must be T.  Returns the
    combined difference [H][W] and the per-template outputs of Plan.subtract."""
    import torch
    T = R.shape[0]
    if plan.batch != T:
        raise ValueError("the plan's batch must equal the number of templates")
    Sx = S.reshape(1, *S.shape).expand(T, -1, -1).contiguous()
    out = plan.subtract(R, Sx, bad, None, refine=refine)
    if scale is None:
        scale = torch.ones(T, dtype=torch.float32, device=R.device)
    comb = median_combine(out["D"], scale, bad)
    return comb, out
