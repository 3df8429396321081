"""Thin ctypes binding of libwd.so (argument marshalling only).

Every function forwards to the C entry point of the same name declared in
``include/wd.h``; torch tensors are passed as raw device or host pointers and
streams as ``torch.cuda.Stream.cuda_stream``. There is no fallback: if the
compiled library is missing, loading raises.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwd.so")

# enums of wd.h
WD_OK, WD_ERR_INVALID_ARG, WD_ERR_CUDA, WD_ERR_NOT_SU3 = 0, 1, 2, 3
WD_ERR_NOT_CONVERGED, WD_ERR_BREAKDOWN, WD_ERR_NONFINITE, WD_ERR_TIMEOUT, WD_ERR_NO_GAUGE = 4, 5, 6, 7, 8
WD_FP64, WD_FP32, WD_FP16, WD_BF16 = 0, 1, 2, 3
WD_OP_HOP_EO, WD_OP_HOP_OE, WD_OP_EO_A, WD_OP_FULL = 0, 1, 2, 3
WD_HOST, WD_DEVICE = 0, 1
WD_FP64_BICGSTAB, WD_MIXED_FP32, WD_MIXED_FP16_PLAIN, WD_MIXED_FP16, WD_MIXED_BF16 = 0, 1, 2, 3, 4

PREC = {"fp64": WD_FP64, "fp32": WD_FP32, "fp16": WD_FP16, "bf16": WD_BF16}
SCHEME = {"fp64": WD_FP64_BICGSTAB, "mixed_fp32": WD_MIXED_FP32, "mixed_fp16_plain": WD_MIXED_FP16_PLAIN,
          "mixed_fp16": WD_MIXED_FP16, "mixed_bf16": WD_MIXED_BF16}

# Exported symbols (the declarations of include/wd.h).
SYMBOLS = ["wd_create", "wd_destroy", "wd_set_gauge", "wd_gauge_unitarity", "wd_set_clover", "wd_set_arith",
           "wd_get_arith", "wd_vector_bytes", "wd_pack",
           "wd_unpack", "wd_apply", "wd_apply_eo_noalloc", "wd_tune", "wd_solve_params_default", "wd_solve",
           "wd_solve_batch",
           "wd_precond_set",
           "wd_precond_get", "wd_precond_apply", "wd_precond_grad", "wd_precond_train_step", "wd_status_string",
           "wd_last_error", "wd_dd_set_partition", "wd_dd_face_bytes", "wd_dd_pack", "wd_dd_hop_interior",
           "wd_dd_hop_faces", "wd_vec_dot", "wd_vec_axpby", "wd_set_wait_limit", "wd_apply_batch",
           "wd_set_rhs_per_thread", "wd_fma_probe", "wd_timeline_set", "wd_precond_load", "wd_precond_train"]
WD_MIXED_FP16_LEARNED = 5
SCHEME["mixed_fp16_learned"] = WD_MIXED_FP16_LEARNED
PRECOND_FLOATS = 6912


class TuneResult(C.Structure):
    _fields_ = [("variant", C.c_int), ("block", C.c_int), ("us", C.c_double), ("default_us", C.c_double),
                ("candidates", C.c_int), ("variant_reducing", C.c_int), ("block_reducing", C.c_int),
                ("us_reducing", C.c_double), ("rhs_per_thread", C.c_int), ("rhs_links_smem", C.c_int),
                ("us16", C.c_double), ("rhs_per_thread_reducing", C.c_int), ("rhs_links_smem_reducing", C.c_int),
                ("us16_reducing", C.c_double), ("candidates16", C.c_int), ("sites_per_thread", C.c_int)]


class SolveParams(C.Structure):
    _fields_ = [("s", C.c_double), ("sigma", C.c_double), ("sigma_lambda", C.c_double),
                ("inner_eps", C.c_double), ("omega0", C.c_double), ("recalc_gamma", C.c_int),
                ("rescale_x", C.c_int), ("use_shat", C.c_int), ("x_is_guess", C.c_int), ("max_outer", C.c_int),
                ("max_inner", C.c_int), ("recon", C.c_int), ("ftz", C.c_int), ("iters_per_sync", C.c_int),
                ("history", C.POINTER(C.c_double)), ("history_cap", C.c_int), ("fused_rescale", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iterations", C.c_int), ("inner_iterations", C.c_int),
                ("inner_matvecs", C.c_int), ("outer_matvecs", C.c_int), ("true_residual", C.c_double),
                ("outer_residual", C.c_double), ("elapsed_ms", C.c_double),
                ("first_inner_nonzeros", C.c_longlong), ("kernel_launches", C.c_longlong),
                ("history_len", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def use_library(path: str) -> None:
    """Load the library from `path` instead of libwd.so (before the first call
    into it; the timeline build, for instance)."""
    global LIB_PATH
    if _lib is not None and path != LIB_PATH:
        raise RuntimeError("the library is already loaded from " + LIB_PATH)
    LIB_PATH = path


def lib():
    """Load libwd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_2602_14450_gb300.build")
        L = C.CDLL(LIB_PATH)
        vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
        L.wd_create.argtypes = [C.POINTER(C.c_int), d, C.POINTER(C.c_int), C.POINTER(vp)]
        L.wd_destroy.argtypes = [vp]
        L.wd_set_gauge.argtypes = [vp, vp, i]
        L.wd_gauge_unitarity.argtypes = [vp, C.POINTER(d), C.POINTER(d)]
        L.wd_set_clover.argtypes = [vp, d]
        L.wd_set_arith.argtypes = [vp, i]
        L.wd_get_arith.argtypes = [vp]
        L.wd_set_wait_limit.argtypes = [vp, C.c_longlong]
        L.wd_timeline_set.argtypes = [vp, vp]
        L.wd_vector_bytes.argtypes = [vp, i]
        L.wd_vector_bytes.restype = sz
        L.wd_pack.argtypes = [vp, i, i, vp, vp, vp]
        L.wd_unpack.argtypes = [vp, i, i, vp, vp, vp]
        L.wd_apply.argtypes = [vp, i, i, i, vp, vp, vp]
        L.wd_apply_eo_noalloc.argtypes = [vp, i, i, vp, vp, vp]
        L.wd_apply_batch.argtypes = [vp, i, i, i, i, vp, vp, vp]
        L.wd_set_rhs_per_thread.argtypes = [vp, i, i, i, i]
        L.wd_tune.argtypes = [vp, i, i, i, vp, C.POINTER(TuneResult)]
        L.wd_solve_params_default.argtypes = [i, C.POINTER(SolveParams)]
        L.wd_solve.argtypes = [vp, vp, vp, d, i, C.POINTER(SolveParams), C.POINTER(SolveStats), vp]
        L.wd_solve_batch.argtypes = [i, C.POINTER(vp), C.POINTER(C.c_int), C.POINTER(vp), C.POINTER(vp), d, i,
                                     C.POINTER(SolveParams), C.POINTER(SolveStats), vp]
        L.wd_precond_set.argtypes = [vp, vp, i]
        L.wd_precond_get.argtypes = [vp, vp, i]
        L.wd_precond_apply.argtypes = [vp, i, vp, vp, vp]
        L.wd_precond_grad.argtypes = [vp, i, vp, vp, d, vp, C.POINTER(d), vp]
        L.wd_precond_train_step.argtypes = [vp, i, vp, vp, d, d, C.POINTER(d), vp]
        L.wd_precond_load.argtypes = [vp, vp, sz]
        L.wd_precond_train.argtypes = [vp, i, i, vp, vp, d, d, C.POINTER(d), vp]
        L.wd_dd_set_partition.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.wd_dd_face_bytes.argtypes = [vp, i, i]
        L.wd_dd_face_bytes.restype = sz
        L.wd_dd_pack.argtypes = [vp, i, i, vp, C.POINTER(vp), vp]
        L.wd_dd_hop_interior.argtypes = [vp, i, i, i, vp, vp, d, d, vp, vp]
        L.wd_dd_hop_faces.argtypes = [vp, i, i, C.POINTER(vp), d, vp, vp]
        L.wd_vec_dot.argtypes = [vp, i, vp, vp, C.POINTER(d), vp]
        L.wd_vec_axpby.argtypes = [vp, i, C.POINTER(d), vp, C.POINTER(d), vp, vp]
        L.wd_fma_probe.argtypes = [i, C.c_longlong, vp, vp, C.POINTER(d)]
        L.wd_status_string.argtypes = [i]
        L.wd_status_string.restype = C.c_char_p
        L.wd_last_error.argtypes = [vp]
        L.wd_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def fma_peak(bits, iters=1 << 14, stream=None):
    """Measured FMA throughput of the FP64 (64), FP32 (32) or packed FP16 (16) pipe in
    TFLOP/s: wd_fma_probe timed with CUDA events (one warm-up launch, then three)."""
    import torch
    sink = torch.zeros(4096, dtype=torch.float32, device="cuda")
    st = _stream(stream)
    fl = C.c_double()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    rc = lib().wd_fma_probe(int(bits), int(iters), _ptr(sink), st, C.byref(fl))
    if rc:
        raise WDError(rc, "wd_fma_probe")
    s = torch.cuda.current_stream() if stream is None else stream
    ev[0].record(s)
    for _ in range(3):
        lib().wd_fma_probe(int(bits), int(iters), _ptr(sink), st, C.byref(fl))
    ev[1].record(s)
    ev[1].synchronize()
    return 3 * fl.value / (ev[0].elapsed_time(ev[1]) * 1e-3) / 1e12


class WDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{lib().wd_status_string(code).decode()}: {msg}")
        self.code = code


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def default_params(scheme) -> SolveParams:
    p = SolveParams()
    rc = lib().wd_solve_params_default(SCHEME.get(scheme, scheme), C.byref(p))
    if rc:
        raise WDError(rc, "wd_solve_params_default")
    return p


class Lattice:
    """One wd_handle: lattice geometry, kappa, boundary phases and gauge field."""

    def __init__(self, dims, kappa, bc=(1, 1, 1, -1)):
        self.dims = tuple(int(d) for d in dims)
        self.kappa = float(kappa)
        d = (C.c_int * 4)(*self.dims)
        b = (C.c_int * 4)(*bc)
        h = C.c_void_p()
        rc = lib().wd_create(d, self.kappa, b, C.byref(h))
        if rc:
            raise WDError(rc, f"wd_create{self.dims}")
        self.h = h

    def _check(self, rc, what):
        if rc not in (WD_OK,):
            raise WDError(rc, f"{what}: {lib().wd_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            lib().wd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_gauge(self, u):
        """u: float64 tensor in the host layout [4, V, 3, 3, 2] (CPU or CUDA)."""
        where = WD_DEVICE if u.is_cuda else WD_HOST
        self._check(lib().wd_set_gauge(self.h, _ptr(u.contiguous()), where), "wd_set_gauge")

    def set_clover(self, csw):
        """wd_set_clover: add the clover term with coefficient csw (0 removes it)."""
        self._check(lib().wd_set_clover(self.h, float(csw)), "wd_set_clover")

    def set_arith(self, bits):
        """wd_set_arith: arithmetic of the FP16-storage hopping term, 32 (FP32) or 16 (FP16, half2)."""
        self._check(lib().wd_set_arith(self.h, int(bits)), "wd_set_arith")

    def set_wait_limit(self, rounds):
        """wd_set_wait_limit: rounds of every bounded device wait (< 0: the default)."""
        self._check(lib().wd_set_wait_limit(self.h, int(rounds)), "wd_set_wait_limit")

    @property
    def arith(self):
        """wd_get_arith: 32 or 16."""
        return int(lib().wd_get_arith(self.h))

    def unitarity(self):
        a, b = C.c_double(), C.c_double()
        self._check(lib().wd_gauge_unitarity(self.h, C.byref(a), C.byref(b)), "wd_gauge_unitarity")
        return a.value, b.value

    def vector_bytes(self, prec):
        return int(lib().wd_vector_bytes(self.h, PREC.get(prec, prec)))

    def pack(self, prec, parity, lex, packed, stream=None):
        self._check(lib().wd_pack(self.h, PREC.get(prec, prec), parity, _ptr(lex), _ptr(packed), _stream(stream)),
                    "wd_pack")

    def unpack(self, prec, parity, packed, lex, stream=None):
        self._check(lib().wd_unpack(self.h, PREC.get(prec, prec), parity, _ptr(packed), _ptr(lex), _stream(stream)),
                    "wd_unpack")

    def apply(self, prec, recon, op, x, y, stream=None):
        self._check(lib().wd_apply(self.h, PREC.get(prec, prec), recon, op, _ptr(x), _ptr(y), _stream(stream)),
                    "wd_apply")

    def apply_batch(self, prec, recon, op, nrhs, x, y, stream=None):
        """wd_apply_batch: the operator on nrhs packed vectors stored back to back."""
        self._check(lib().wd_apply_batch(self.h, PREC.get(prec, prec), recon, op, int(nrhs), _ptr(x), _ptr(y),
                                         _stream(stream)), "wd_apply_batch")

    def set_rhs_per_thread(self, recon, k_plain, k_reducing=None, links_smem=0):
        """wd_set_rhs_per_thread: right-hand sides per thread of the FP16-arithmetic hop."""
        k_reducing = k_plain if k_reducing is None else k_reducing
        self._check(lib().wd_set_rhs_per_thread(self.h, int(recon), int(k_plain), int(k_reducing), int(links_smem)),
                    "wd_set_rhs_per_thread")

    # --- domain decomposition ---------------------------------------------
    def dd_set_partition(self, grid, coords):
        """wd_dd_set_partition: this handle is the sub-lattice at `coords` of the process grid `grid`."""
        self._check(lib().wd_dd_set_partition(self.h, (C.c_int * 4)(*grid), (C.c_int * 4)(*coords)),
                    "wd_dd_set_partition")

    def dd_face_bytes(self, prec, mu):
        return int(lib().wd_dd_face_bytes(self.h, PREC.get(prec, prec), int(mu)))

    @staticmethod
    def _faces(bufs):
        return (C.c_void_p * 8)(*[None if b is None else b.data_ptr() for b in bufs])

    def dd_pack(self, prec, parity, x, send, stream=None):
        self._check(lib().wd_dd_pack(self.h, PREC.get(prec, prec), int(parity), _ptr(x), self._faces(send),
                                     _stream(stream)), "wd_dd_pack")

    def dd_hop_interior(self, prec, recon, parity, x, y, a, b, out, stream=None):
        self._check(lib().wd_dd_hop_interior(self.h, PREC.get(prec, prec), int(recon), int(parity), _ptr(x),
                                             None if y is None else _ptr(y), float(a), float(b), _ptr(out),
                                             _stream(stream)), "wd_dd_hop_interior")

    def dd_hop_faces(self, prec, parity, recv, a, out, stream=None):
        self._check(lib().wd_dd_hop_faces(self.h, PREC.get(prec, prec), int(parity), self._faces(recv), float(a),
                                          _ptr(out), _stream(stream)), "wd_dd_hop_faces")

    def vec_dot(self, prec, a, b, stream=None) -> complex:
        """wd_vec_dot: FP64 sum_i conj(a_i) b_i over one packed parity vector."""
        out = (C.c_double * 2)()
        self._check(lib().wd_vec_dot(self.h, PREC.get(prec, prec), _ptr(a), _ptr(b), out, _stream(stream)),
                    "wd_vec_dot")
        return complex(out[0], out[1])

    def vec_axpby(self, prec, a, x, b, y, stream=None):
        """wd_vec_axpby: y = a x + b y (a, b complex)."""
        a, b = complex(a), complex(b)
        self._check(lib().wd_vec_axpby(self.h, PREC.get(prec, prec), (C.c_double * 2)(a.real, a.imag), _ptr(x),
                                       (C.c_double * 2)(b.real, b.imag), _ptr(y), _stream(stream)), "wd_vec_axpby")

    # --- learned right preconditioner -------------------------------------
    def tune(self, prec, recon, nrhs=1, stream=None):
        """wd_tune: pick the fastest hop kernel variant and block size for (prec, recon) on this lattice."""
        r = TuneResult()
        self._check(lib().wd_tune(self.h, PREC.get(prec, prec), int(recon), int(nrhs), _stream(stream), C.byref(r)),
                    "wd_tune")
        return {k: getattr(r, k) for k, _ in TuneResult._fields_}

    def precond_set(self, w):
        """w: float32 tensor of PRECOND_FLOATS weights (flat layout of wd.h), CPU or CUDA."""
        w = w.to(dtype=__import__("torch").float32).contiguous()
        self._check(lib().wd_precond_set(self.h, _ptr(w), WD_DEVICE if w.is_cuda else WD_HOST), "wd_precond_set")

    def precond_get(self):
        import torch
        w = torch.empty(PRECOND_FLOATS, dtype=torch.float32)
        self._check(lib().wd_precond_get(self.h, _ptr(w), WD_HOST), "wd_precond_get")
        return w

    def precond_apply(self, prec, x, y, stream=None):
        self._check(lib().wd_precond_apply(self.h, PREC.get(prec, prec), _ptr(x), _ptr(y), _stream(stream)),
                    "wd_precond_apply")

    def precond_grad(self, v, y, mu, stream=None):
        """(loss, gradient) for n samples: v, y float32 device tensors [n, packed even vector]."""
        import torch
        g = torch.empty(PRECOND_FLOATS, dtype=torch.float32, device="cuda")
        loss = C.c_double()
        self._check(lib().wd_precond_grad(self.h, int(v.shape[0]), _ptr(v), _ptr(y), float(mu), _ptr(g),
                                          C.byref(loss), _stream(stream)), "wd_precond_grad")
        return loss.value, g

    def precond_train_step(self, v, y, mu, lr, stream=None):
        loss = C.c_double()
        self._check(lib().wd_precond_train_step(self.h, int(v.shape[0]), _ptr(v), _ptr(y), float(mu), float(lr),
                                                C.byref(loss), _stream(stream)), "wd_precond_train_step")
        return loss.value

    def precond_load(self, w_bf16):
        """w_bf16: PRECOND_FLOATS BF16 weights (torch.bfloat16 or their int16 bit patterns), CPU."""
        import torch
        w = w_bf16.contiguous().view(torch.int16).cpu()
        self._check(lib().wd_precond_load(self.h, _ptr(w), w.numel()), "wd_precond_load")

    def precond_train(self, steps, v, y, mu, lr, stream=None):
        loss = C.c_double()
        self._check(lib().wd_precond_train(self.h, int(steps), int(v.shape[0]), _ptr(v), _ptr(y), float(mu),
                                           float(lr), C.byref(loss), _stream(stream)), "wd_precond_train")
        return loss.value

    def solve_rhs(self, b, x, tol=1e-10, scheme="mixed_fp16", params=None, stream=None, check=True):
        """Several right-hand sides of this lattice in one batched solve; b, x: [nrhs, ...] float64."""
        return solve_batch([self], [b], [x], tol, scheme, params, stream, check)

    def solve(self, b, x, tol=1e-10, scheme="mixed_fp16", params=None, stream=None, check=True):
        """Solve D_W x = b; b, x float64 full-lattice tensors (host layout), CPU or CUDA."""
        sc = SCHEME.get(scheme, scheme)
        prm = params if params is not None else default_params(sc)
        st = SolveStats()
        rc = lib().wd_solve(self.h, _ptr(b), _ptr(x), float(tol), sc, C.byref(prm), C.byref(st), _stream(stream))
        if check:
            self._check(rc, "wd_solve")
        return st


def solve_with_history(lat, b, x, tol=1e-10, scheme="mixed_fp16", params=None, stream=None, cap=100000):
    """wd_solve with the convergence history: returns (stats, rows) with rows a list of
    (kind, matvecs, residual, nonzeros); kind 1 = refinement trip, 0 = inner iteration."""
    sc = SCHEME.get(scheme, scheme)
    prm = params if params is not None else default_params(sc)
    buf = (C.c_double * (4 * cap))()
    prm.history = C.cast(buf, C.POINTER(C.c_double))
    prm.history_cap = cap
    st = lat.solve(b, x, tol, scheme, prm, stream, check=False)
    rows = [tuple(buf[4 * i: 4 * i + 4]) for i in range(st.history_len)]
    prm.history = None
    prm.history_cap = 0
    return st, rows


def solve_batch(lattices, bs, xs, tol=1e-10, scheme="mixed_fp16", params=None, stream=None, check=True):
    """wd_solve_batch: lattice i solves bs[i] ([nrhs_i, ...] float64, device) into xs[i].

    Returns the list of per-right-hand-side SolveStats (lattice-major order).
    """
    n = len(lattices)
    sc = SCHEME.get(scheme, scheme)
    prm = params if params is not None else default_params(sc)
    nr = [int(b.shape[0]) for b in bs]
    hs = (C.c_void_p * n)(*[lat.h for lat in lattices])
    nrhs = (C.c_int * n)(*nr)
    bp = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    stats = (SolveStats * max(1, sum(nr)))()
    rc = lib().wd_solve_batch(n, hs, nrhs, bp, xp, float(tol), sc, C.byref(prm), stats, _stream(stream))
    if check and rc != WD_OK:
        raise WDError(rc, f"wd_solve_batch: {lib().wd_last_error(lattices[0].h).decode()}")
    return list(stats)[:sum(nr)]
