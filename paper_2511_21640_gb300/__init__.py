"""Python binding of the GB300 relativistic CD-ADC library (libadc_gb300.so).

Argument marshalling only: every arithmetic step runs in the library's CUDA
kernels. Inputs may be numpy arrays (host) or torch tensors (host or CUDA);
complex arrays must be complex128 and C-contiguous. There is no CPU fallback:
importing this package fails when the compiled library is missing.

The C ABI is declared in ``include/adc_gb300.h``; the names here mirror it:
``Context(...)`` wraps ``adc_init``/``adc_free``, ``Context.sigma`` wraps
``adc_sigma``, ``Context.davidson`` wraps ``adc_davidson``,
``Context.fns_density`` wraps ``adc_fns_density``; ``ssfns`` wraps ``adc_ssfns``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libadc_gb300.so")

ADC_IP, ADC_EA, ADC_EE = 0, 1, 2
ADC_PREC_FP64, ADC_PREC_BF16X3, ADC_PREC_BF16X6, ADC_PREC_SLICED, ADC_PREC_SLICED24 = 0, 1, 2, 3, 4
KINDS = {"IP": ADC_IP, "EA": ADC_EA, "EE": ADC_EE}
PRECISIONS = {"fp64": ADC_PREC_FP64, "bf16x3": ADC_PREC_BF16X3, "bf16x6": ADC_PREC_BF16X6,
              "sliced": ADC_PREC_SLICED, "sliced24": ADC_PREC_SLICED24}
ERRORS = {0: "ADC_OK", -1: "ADC_ERR_ARG", -2: "ADC_ERR_OOM", -3: "ADC_ERR_CUDA", -4: "ADC_ERR_NOCONV",
          -5: "ADC_ERR_TIMEOUT", -6: "ADC_ERR_UNSUPPORTED", -7: "ADC_ERR_STATE", -8: "ADC_ERR_NUMERIC"}


class AdcError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"{ERRORS.get(code, code)}: {message}")
        self.code = code


class adc_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("stream", ctypes.c_void_p), ("block", ctypes.c_int),
                ("max_subspace", ctypes.c_int), ("herm_tol", ctypes.c_double),
                ("mem_limit", ctypes.c_int64), ("verbose", ctypes.c_int), ("dd_order", ctypes.c_int),
                ("refine", ctypes.c_int), ("setup", ctypes.c_int), ("ee_vvvv", ctypes.c_int),
                ("correction", ctypes.c_int), ("ladder", ctypes.c_int), ("profile", ctypes.c_int),
                ("grouped_sigma", ctypes.c_int)]


class adc_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("iterations_fp64", ctypes.c_int),
                ("sigma_calls", ctypes.c_int), ("sigma_calls_fp64", ctypes.c_int),
                ("time_total_s", ctypes.c_double), ("time_sigma_s", ctypes.c_double),
                ("max_residual", ctypes.c_double), ("sigma_calls_mid", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class adc_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class adc_ssfns_root(ctypes.Structure):
    _fields_ = [("omega_corrected", ctypes.c_double), ("omega_fns", ctypes.c_double),
                ("omega2_canonical", ctypes.c_double), ("omega2_fns", ctypes.c_double),
                ("err64", ctypes.c_double), ("n_keep", ctypes.c_int64), ("status", ctypes.c_int),
                ("pad_", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class adc_batch_info(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_int64), ("graph_launches", ctypes.c_int64),
                ("graphs_captured", ctypes.c_int64), ("direct_launches", ctypes.c_int64),
                ("sigma_vectors", ctypes.c_int64), ("batch_ms", ctypes.c_double), ("tc_flops", ctypes.c_double),
                ("tuned_shapes", ctypes.c_int64), ("waves", ctypes.c_int64), ("init_s", ctypes.c_double),
                ("solve_s", ctypes.c_double), ("grouped_launches", ctypes.c_int64), ("grouped_ms", ctypes.c_double),
                ("grouped_flops", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class adc_problem(ctypes.Structure):
    _fields_ = [("B", ctypes.c_void_p), ("naux", ctypes.c_int64), ("eps_occ", ctypes.c_void_p),
                ("nocc", ctypes.c_int64), ("eps_vir", ctypes.c_void_p), ("nvir", ctypes.c_int64),
                ("kind", ctypes.c_int), ("order", ctypes.c_int), ("x", ctypes.c_double)]


class adc_batch_opts(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_int64), ("init_lanes", ctypes.c_int), ("verbose", ctypes.c_int),
                ("setup", ctypes.c_int), ("refine", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(or python paper_2511_21640_gb300/build.py)")
    L = ctypes.CDLL(LIB_PATH)
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "adc_opts_default": (I, [ctypes.POINTER(adc_opts)]),
        "adc_init": (I, [ctypes.POINTER(P), P, I64, P, I64, P, I64, I, I, D, ctypes.POINTER(adc_opts)]),
        "adc_dims": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "adc_sigma": (I, [P, P, P, I64, I]),
        "adc_sigma_noalloc": (I, [P, P, P, I64]),
        "adc_sigma_share": (I, [P, P, P, I64, I64, I64, I]),
        "adc_diagonal": (I, [P, P]),
        "adc_main_block": (I, [P, P]),
        "adc_davidson": (I, [P, I, D, I, I, P, I64, P, P, P, ctypes.POINTER(adc_stats)]),
        "adc_fns_density": (I, [P, P, P, P, D, ctypes.POINTER(I64), P, P]),
        "adc_sync": (I, [P]),
        "adc_fns_transform": (I, [P, P, I64, I64, P]),
        "adc_free": (None, [P]),
        "adc_profile_enable": (I, [P, I]),
        "adc_profile_read": (I, [P, ctypes.POINTER(adc_kernel_stat), I, ctypes.POINTER(I)]),
        "adc_launch_count": (I64, []),
        "adc_strerror": (ctypes.c_char_p, [I]),
        "adc_last_error": (ctypes.c_char_p, [P]),
        "adc_diag_gemm": (I, [I, I64, I64, I64, ctypes.c_uint64, I, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "adc_diag_blockops": (I, [I, I64, I64, I64, ctypes.c_uint64, I, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "adc_diag_fp64_peak": (I, [I, I64, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "adc_diag_set_wait_ns": (I, [ctypes.c_uint64]),
        "adc_diag_set_setup_chunk": (I, [ctypes.c_int64]),
        "adc_diag_set_sliced_cap": (I, [ctypes.c_int64]),
        "adc_diag_eigh": (I, [I, P, I, P, P, ctypes.POINTER(D), ctypes.POINTER(I)]),
        "adc_sigma_adjoint": (I, [P, P, P, I64, P, P, P, ctypes.POINTER(D)]),
        "adc_state_density": (I, [P, P, P]),
        "adc_transition_density": (I, [P, P, I64, P]),
        "adc_excited_density": (I, [P, P, I64, P]),
        "adc_spectroscopic_amplitudes": (I, [P, P, I64, P]),
        "adc_state_pair_density": (I, [P, P, P, I64, P]),
        "adc_memory": (I, [P, P, P]),
        "adc_setup_routes": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "adc_ladder_mode": (I, [P, ctypes.POINTER(I)]),
        "adc_cholesky": (I, [P, I64, D, I64, P, P, ctypes.POINTER(I64)]),
        "adc_cholesky_mo": (I, [P, I64, I64, P, I64, P]),
        "adc_ssfns_density": (I, [P, P, D, P, P, ctypes.POINTER(I64), P, P]),
        "adc_fns_vector": (I, [P, P, P, I64, I64, P]),
        "adc_davidson_follow": (I, [P, P, D, I, I, ctypes.POINTER(D), P, ctypes.POINTER(D), P]),
        "adc_ssfns": (I, [P, I64, P, I64, P, I64, I, I, D, I, D, D, I, I, P, P]),
        "adc_batch_create": (I, [ctypes.POINTER(P), P, I]),
        "adc_batch_sigma": (I, [P, P, P, P, I]),
        "adc_batch_davidson": (I, [P, I, D, I, I, P, P, P, P]),
        "adc_batch_use_graphs": (I, [P, I]),
        "adc_batch_info_get": (I, [P, ctypes.POINTER(adc_batch_info)]),
        "adc_batch_free": (None, [P]),
        "adc_batch_last_error": (ctypes.c_char_p, [P]),
        "adc_batch_plan": (I, [I, P, I, I64, P, P, P, P]),
        "adc_batch_solve": (I, [I, P, I, D, I, I, ctypes.POINTER(adc_batch_opts), P, P, P,
                                ctypes.POINTER(adc_batch_info)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _check(rc, ctx=None):
    if rc != 0:
        msg = lib.adc_last_error(ctx)
        raise AdcError(rc, msg.decode() if msg else "")


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """Raw pointer of a C-contiguous array of the given numpy dtype."""
    if a is None:
        return None
    if _is_torch(a):
        import torch
        want = {np.complex128: torch.complex128, np.float64: torch.float64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    return ctypes.c_void_p(a.ctypes.data)


def _on_cuda(*arrays):
    return any(a is not None and _is_torch(a) and a.is_cuda for a in arrays)


def _torch_sync():
    import torch
    torch.cuda.current_stream().synchronize()


def _empty_like_kind(ref, shape, dtype):
    if ref is not None and _is_torch(ref):
        import torch
        tdt = {np.complex128: torch.complex128, np.float64: torch.float64}[dtype]
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.empty(shape, dtype=dtype)


class Context:
    """One ADC problem on the GPU (``adc_init``)."""

    def __init__(self, B, eps_occ, eps_vir, kind="IP", order=3, x=1.0, precision="fp64", stream=None,
                 block=0, max_subspace=0, herm_tol=1e-12, mem_limit=0, verbose=False, dd_order=1,
                 refine="fp64", setup="fp64", vvvv="auto", correction="davidson", ladder="auto",
                 profile=False, grouped_sigma=True):
        o = adc_opts()
        lib.adc_opts_default(ctypes.byref(o))
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if isinstance(stream, str) and stream == "torch":
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self._shared_stream = stream is not None
        o.stream = stream
        o.block = block
        o.max_subspace = max_subspace
        o.herm_tol = herm_tol
        o.mem_limit = mem_limit
        o.verbose = 1 if verbose else 0
        o.dd_order = int(dd_order)
        o.refine = PRECISIONS[refine] if isinstance(refine, str) else int(refine)
        o.setup = PRECISIONS[setup] if isinstance(setup, str) else int(setup)
        o.ee_vvvv = {"auto": 0, "chunked": 1, "dense": -1}[vvvv]
        o.correction = {"davidson": 0, "olsen": 1}[correction]
        o.ladder = {"auto": 0, "direct": 1, "stored": -1}[ladder]
        o.profile = 1 if profile else 0
        o.grouped_sigma = 0 if grouped_sigma else -1
        naux, nmo, nmo2 = B.shape
        nocc, nvir = eps_occ.shape[0], eps_vir.shape[0]
        if nmo != nmo2 or nmo != nocc + nvir:
            raise ValueError("B must be [naux][nmo][nmo] with nmo = nocc + nvir")
        self._h = ctypes.c_void_p()
        self.kind = kind
        self.nocc, self.nvir, self.naux = nocc, nvir, naux
        if _on_cuda(B, eps_occ, eps_vir) and not self._shared_stream:
            _torch_sync()
        rc = lib.adc_init(ctypes.byref(self._h), _ptr(B, np.complex128), naux, _ptr(eps_occ, np.float64), nocc,
                          _ptr(eps_vir, np.float64), nvir, KINDS[kind] if isinstance(kind, str) else kind,
                          order, float(x), ctypes.byref(o))
        _check(rc)
        n1, n2 = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.adc_dims(self._h, ctypes.byref(n1), ctypes.byref(n2)), self._h)
        self.n1, self.n2 = n1.value, n2.value
        self.N = self.n1 + self.n2

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.adc_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sigma(self, X, precision="fp64", out=None):
        """S = M X for X of shape [k][N] (``adc_sigma``)."""
        k = X.shape[0] if X.ndim == 2 else 1
        if X.shape[-1] != self.N:
            raise ValueError("last dimension of X must be N")
        S = out if out is not None else _empty_like_kind(X, tuple(X.shape), np.complex128)
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        dev = _on_cuda(X, S)
        if dev and not self._shared_stream:
            _torch_sync()  # X was written on torch's stream
        _check(lib.adc_sigma(self._h, _ptr(X, np.complex128), _ptr(S, np.complex128), k, p), self._h)
        if dev and not self._shared_stream:
            _check(lib.adc_sync(self._h), self._h)  # S is read on torch's stream
        return S

    def sigma_share(self, X, i0, i1, with_main):
        """One rank's share of S = M X for an EA problem split by the satellites'
        occupied index (``adc_sigma_share``): X [k][N] whole, returns [k][n1 + (i1 - i0) Pv]
        (partial 1p rows, then the share's satellite rows)."""
        X2 = X if X.ndim == 2 else X.reshape(1, -1)
        k = X2.shape[0]
        if X2.shape[1] != self.N:
            raise ValueError("last dimension of X must be N")
        pv = self.nvir * (self.nvir - 1) // 2
        S = _empty_like_kind(X2, (k, self.n1 + (int(i1) - int(i0)) * pv), np.complex128)
        dev = _on_cuda(X2, S)
        if dev and not self._shared_stream:
            _torch_sync()
        _check(lib.adc_sigma_share(self._h, _ptr(X2, np.complex128), _ptr(S, np.complex128), k, int(i0), int(i1),
                                   1 if with_main else 0), self._h)
        if dev and not self._shared_stream:
            _check(lib.adc_sync(self._h), self._h)
        return S

    def fns_transform(self, U, n_keep=None):
        """Cholesky vectors in the truncated natural-spinor basis (``adc_fns_transform``)."""
        U = np.ascontiguousarray(U, dtype=np.complex128) if not _is_torch(U) else U
        nk = U.shape[1] if n_keep is None else int(n_keep)
        n2 = self.nocc + nk
        Bo = _empty_like_kind(U, (self.naux, n2, n2), np.complex128)
        dev = _on_cuda(U, Bo)
        if dev and not self._shared_stream:
            _torch_sync()
        _check(lib.adc_fns_transform(self._h, _ptr(U, np.complex128), U.shape[1], nk, _ptr(Bo, np.complex128)),
               self._h)
        return Bo

    def sync(self):
        _check(lib.adc_sync(self._h), self._h)

    def profile(self, on=True):
        """Start (clear) or stop per-kernel CUDA-event timing (``adc_profile_enable``)."""
        _check(lib.adc_profile_enable(self._h, 1 if on else 0), self._h)

    def profile_read(self):
        """Per kernel and sigma term: launches, total device ms, algorithmic flops."""
        buf = (adc_kernel_stat * 512)()
        n = ctypes.c_int()
        _check(lib.adc_profile_read(self._h, buf, 512, ctypes.byref(n)), self._h)
        return {buf[i].name.decode(): {"launches": buf[i].launches, "total_ms": buf[i].total_ms,
                                       "flops": buf[i].flops, "bytes": buf[i].bytes} for i in range(n.value)}

    def diagonal(self):
        d = np.empty(self.N, dtype=np.float64)
        _check(lib.adc_diagonal(self._h, _ptr(d, np.float64)), self._h)
        return d

    def main_block(self):
        m = np.empty((self.n1, self.n1), dtype=np.complex128)
        _check(lib.adc_main_block(self._h, _ptr(m, np.complex128)), self._h)
        return m

    def davidson(self, nroots, tol=1e-8, max_iter=200, precision="fp64", guess=None, want_vectors=True,
                 raise_on_noconv=True):
        """Lowest roots (``adc_davidson``): returns (omega, Y or None, err64, stats dict, rc)."""
        omega = np.empty(nroots, dtype=np.float64)
        err = np.empty(nroots, dtype=np.float64)
        Y = np.empty((nroots, self.N), dtype=np.complex128) if want_vectors else None
        st = adc_stats()
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        ng = 0 if guess is None else guess.shape[0]
        rc = lib.adc_davidson(self._h, nroots, float(tol), int(max_iter), p, _ptr(guess, np.complex128), ng,
                              _ptr(omega, np.float64), _ptr(Y, np.complex128) if Y is not None else None,
                              _ptr(err, np.float64), ctypes.byref(st))
        if rc != 0 and not (rc == -4 and not raise_on_noconv):
            _check(rc, self._h)
        return omega, Y, err, st.as_dict(), rc

    def sigma_adjoint(self, Y, gomega):
        """Gradients of sum_r gomega[r] y_r^H M y_r (``adc_sigma_adjoint``): (gB, geps_occ, geps_vir, gx).

        Y: [nroots][N] eigenvectors (numpy or torch); outputs are numpy arrays,
        or CUDA tensors when Y is a CUDA tensor."""
        g = np.ascontiguousarray(np.asarray(gomega, dtype=np.float64).reshape(-1))
        k = Y.shape[0] if Y.ndim == 2 else 1
        if g.shape[0] != k:
            raise ValueError("one weight per vector")
        nmo = self.nocc + self.nvir
        gB = _empty_like_kind(Y, (self.naux, nmo, nmo), np.complex128)
        geo = _empty_like_kind(Y, (self.nocc,), np.float64)
        gev = _empty_like_kind(Y, (self.nvir,), np.float64)
        gx = ctypes.c_double()
        if _on_cuda(Y) and not self._shared_stream:
            _torch_sync()
        _check(lib.adc_sigma_adjoint(self._h, _ptr(Y, np.complex128), g.ctypes.data_as(ctypes.c_void_p), k,
                                     _ptr(gB, np.complex128), _ptr(geo, np.float64), _ptr(gev, np.float64),
                                     ctypes.byref(gx)), self._h)
        return gB, geo, gev, gx.value

    def transition_density(self, Y):
        """Ground-to-excited transition densities [k][nmo][nmo] of EE vectors Y [k][N]
        (``adc_transition_density``, Sec. 2.2)."""
        Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.complex128)
        nmo = self.nocc + self.nvir
        rho = np.empty((Y.shape[0], nmo, nmo), dtype=np.complex128)
        _check(lib.adc_transition_density(self._h, _ptr(Y, np.complex128), Y.shape[0], _ptr(rho, np.complex128)),
               self._h)
        return rho

    def excited_density(self, Y):
        """State densities [k][nmo][nmo] of the vectors Y [k][N], any kind (``adc_excited_density``)."""
        Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.complex128)
        nmo = self.nocc + self.nvir
        rho = np.empty((Y.shape[0], nmo, nmo), dtype=np.complex128)
        _check(lib.adc_excited_density(self._h, _ptr(Y, np.complex128), Y.shape[0], _ptr(rho, np.complex128)),
               self._h)
        return rho

    def state_pair_density(self, YK, YL):
        """<Psi_K|a+_p a_q|Psi_L> [k][nmo][nmo] of the pairs (YK[z], YL[z]) (``adc_state_pair_density``)."""
        YK = np.ascontiguousarray(np.atleast_2d(YK), dtype=np.complex128)
        YL = np.ascontiguousarray(np.atleast_2d(YL), dtype=np.complex128)
        if YK.shape != YL.shape:
            raise ValueError("YK and YL must have the same shape")
        nmo = self.nocc + self.nvir
        rho = np.empty((YK.shape[0], nmo, nmo), dtype=np.complex128)
        _check(lib.adc_state_pair_density(self._h, _ptr(YK, np.complex128), _ptr(YL, np.complex128), YK.shape[0],
                                          _ptr(rho, np.complex128)), self._h)
        return rho

    def memory(self):
        """Bytes the context's device buffers hold now and at most since init (``adc_memory``)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.adc_memory(self._h, ctypes.byref(a), ctypes.byref(b)), self._h)
        return {"in_use": a.value, "peak": b.value}

    def direct_ladder(self):
        """Whether the context forms its ladder integrals in every product (``adc_ladder_mode``)."""
        m = ctypes.c_int()
        _check(lib.adc_ladder_mode(self._h, ctypes.byref(m)), self._h)
        return bool(m.value)

    def setup_routes(self):
        """Products adc_init ran as the sliced tensor-core product and on the FP64 cores (``adc_setup_routes``)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        fa, fb = ctypes.c_double(), ctypes.c_double()
        _check(lib.adc_setup_routes(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(fa), ctypes.byref(fb)),
               self._h)
        return {"n_sliced": a.value, "n_fp64": b.value, "flops_sliced": fa.value, "flops_fp64": fb.value}

    def spectroscopic_amplitudes(self, Y):
        """Spectroscopic amplitudes [k][nmo] of IP/EA vectors Y [k][N] (``adc_spectroscopic_amplitudes``)."""
        Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.complex128)
        x = np.empty((Y.shape[0], self.nocc + self.nvir), dtype=np.complex128)
        _check(lib.adc_spectroscopic_amplitudes(self._h, _ptr(Y, np.complex128), Y.shape[0],
                                                _ptr(x, np.complex128)), self._h)
        return x

    def state_density(self, y):
        """Virtual density of the configurations weighted by y (``adc_state_density``, Eq. 31)."""
        y = np.ascontiguousarray(y, dtype=np.complex128).reshape(-1)
        D = np.empty((self.nvir, self.nvir), dtype=np.complex128)
        _check(lib.adc_state_density(self._h, _ptr(y, np.complex128), _ptr(D, np.complex128)), self._h)
        return D

    def ssfns_density(self, y, eta_crit):
        """State-specific natural spinors of the state y (``adc_ssfns_density``, Eqs. 31, 26-30)."""
        y = np.ascontiguousarray(y, dtype=np.complex128).reshape(-1)
        nvir = self.nvir
        D = np.empty((nvir, nvir), dtype=np.complex128)
        eta = np.empty(nvir, dtype=np.float64)
        U = np.empty((nvir, nvir), dtype=np.complex128)
        en = np.empty(nvir, dtype=np.float64)
        nk = ctypes.c_int64()
        _check(lib.adc_ssfns_density(self._h, _ptr(y, np.complex128), float(eta_crit), _ptr(D, np.complex128),
                                     _ptr(eta, np.float64), ctypes.byref(nk), _ptr(U, np.complex128),
                                     _ptr(en, np.float64)), self._h)
        k = nk.value
        return {"D": D, "eta": eta, "n_keep": k, "U": U[:, :k].copy(), "eps_new": en[:k].copy()}

    def fns_vector(self, y, U):
        """y carried into the truncated basis of U [nvir][n_keep] (``adc_fns_vector``)."""
        y = np.ascontiguousarray(y, dtype=np.complex128).reshape(-1)
        U = np.ascontiguousarray(U, dtype=np.complex128)
        nk = U.shape[1]
        o = self.nocc
        n = nk + o * (nk * (nk - 1) // 2) if self.kind == "EA" else o * nk + (o * (o - 1) // 2) * (nk * (nk - 1) // 2)
        g = np.empty(n, dtype=np.complex128)
        _check(lib.adc_fns_vector(self._h, _ptr(y, np.complex128), _ptr(U, np.complex128), nk, nk,
                                  _ptr(g, np.complex128)), self._h)
        return g

    def davidson_follow(self, guess, tol=1e-8, max_iter=300, precision="fp64", raise_on_noconv=True):
        """Root-specific solve (``adc_davidson_follow``): (omega, y, err64, stats dict, rc)."""
        g = np.ascontiguousarray(guess, dtype=np.complex128).reshape(-1)
        y = np.empty(self.N, dtype=np.complex128)
        om, err = ctypes.c_double(), ctypes.c_double()
        st = adc_stats()
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        rc = lib.adc_davidson_follow(self._h, _ptr(g, np.complex128), float(tol), int(max_iter), p, ctypes.byref(om),
                                     _ptr(y, np.complex128), ctypes.byref(err), ctypes.byref(st))
        if rc != 0 and not (rc == -4 and not raise_on_noconv):
            _check(rc, self._h)
        return om.value, y, err.value, st.as_dict(), rc

    def fns_density(self, eta_crit):
        """MP2 virtual density and frozen natural spinors (``adc_fns_density``)."""
        nvir = self.nvir
        D = np.empty((nvir, nvir), dtype=np.complex128)
        eta = np.empty(nvir, dtype=np.float64)
        V = np.empty((nvir, nvir), dtype=np.complex128)
        U = np.empty((nvir, nvir), dtype=np.complex128)
        en = np.empty(nvir, dtype=np.float64)
        nk = ctypes.c_int64()
        _check(lib.adc_fns_density(self._h, _ptr(D, np.complex128), _ptr(eta, np.float64),
                                   _ptr(V, np.complex128), float(eta_crit), ctypes.byref(nk),
                                   _ptr(U, np.complex128), _ptr(en, np.float64)), self._h)
        k = nk.value
        return {"D": D, "eta": eta, "V": V, "n_keep": k, "U": U[:, :k].copy(), "eps_new": en[:k].copy()}


def _bcheck(rc, h=None):
    if rc != 0:
        msg = lib.adc_batch_last_error(h)
        raise AdcError(rc, msg.decode() if msg else "")


class Batch:
    """Several contexts solved together (``adc_batch_*``); the contexts must outlive the batch."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        self._h = ctypes.c_void_p()
        _bcheck(lib.adc_batch_create(ctypes.byref(self._h), arr, len(self.contexts)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.adc_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def use_graphs(self, on=True):
        _bcheck(lib.adc_batch_use_graphs(self._h, 1 if on else 0), self._h)

    def sigma(self, Xs, precision="bf16x3", outs=None):
        """S_i = M_i X_i for device tensors X_i [k_i][N_i] (``adc_batch_sigma``)."""
        import torch
        n = len(self.contexts)
        if len(Xs) != n:
            raise ValueError("one block per context")
        Ss = outs if outs is not None else [torch.empty_like(X) for X in Xs]
        for X, S, c in zip(Xs, Ss, self.contexts):
            if not (_is_torch(X) and X.is_cuda and _is_torch(S) and S.is_cuda):
                raise TypeError("batched sigma takes CUDA tensors")
            if X.shape[-1] != c.N or X.dtype != torch.complex128 or not X.is_contiguous():
                raise ValueError("X_i must be contiguous complex128 [k][N_i]")
        xp = (ctypes.c_void_p * n)(*[X.data_ptr() for X in Xs])
        sp = (ctypes.c_void_p * n)(*[S.data_ptr() for S in Ss])
        kk = (ctypes.c_int64 * n)(*[X.shape[0] if X.ndim == 2 else 1 for X in Xs])
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _bcheck(lib.adc_batch_sigma(self._h, xp, sp, kk, p), self._h)
        return Ss

    def davidson(self, nroots, tol=1e-8, max_iter=200, precision="bf16x3"):
        """Lowest roots of every problem (``adc_batch_davidson``): (omega, err64, status, stats list, rc)."""
        n = len(self.contexts)
        omega = np.empty((n, nroots), dtype=np.float64)
        err = np.empty((n, nroots), dtype=np.float64)
        status = np.empty(n, dtype=np.int32)
        st = (adc_stats * n)()
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        rc = lib.adc_batch_davidson(self._h, int(nroots), float(tol), int(max_iter), p,
                                    omega.ctypes.data_as(ctypes.c_void_p), err.ctypes.data_as(ctypes.c_void_p),
                                    status.ctypes.data_as(ctypes.c_void_p), st)
        if rc not in (0, -4):
            _bcheck(rc, self._h)
        return omega, err, status, [s.as_dict() for s in st], rc

    def info(self):
        i = adc_batch_info()
        _bcheck(lib.adc_batch_info_get(self._h, ctypes.byref(i)), self._h)
        return i.as_dict()


def _problems(problems):
    """adc_problem array from objects with B, eps_occ, eps_vir, kind, order, x (numpy host arrays)."""
    arr = (adc_problem * len(problems))()
    keep = []
    for i, q in enumerate(problems):
        B = np.ascontiguousarray(q.B, dtype=np.complex128)
        eo = np.ascontiguousarray(q.eps_occ, dtype=np.float64)
        ev = np.ascontiguousarray(q.eps_vir, dtype=np.float64)
        keep += [B, eo, ev]
        kind = KINDS[q.kind] if isinstance(q.kind, str) else int(q.kind)
        arr[i] = adc_problem(B.ctypes.data, B.shape[0], eo.ctypes.data, eo.shape[0], ev.ctypes.data, ev.shape[0],
                             kind, int(q.order), float(q.x))
    return arr, keep


def batch_plan(problems, nroots, mem_budget):
    """Host-only wave plan (``adc_batch_plan``): (n_waves, order, wave, mem_est, cost_est)."""
    n = len(problems)
    arr = (adc_problem * n)()
    for i, q in enumerate(problems):
        kind = KINDS[q["kind"]] if isinstance(q["kind"], str) else int(q["kind"])
        arr[i] = adc_problem(None, int(q["naux"]), None, int(q["nocc"]), None, int(q["nvir"]), kind,
                             int(q.get("order", 3)), float(q.get("x", 1.0)))
    order = np.empty(n, dtype=np.int32)
    wave = np.empty(n, dtype=np.int32)
    mem = np.empty(n, dtype=np.int64)
    cost = np.empty(n, dtype=np.float64)
    rc = lib.adc_batch_plan(n, arr, int(nroots), int(mem_budget), order.ctypes.data_as(ctypes.c_void_p),
                            wave.ctypes.data_as(ctypes.c_void_p), mem.ctypes.data_as(ctypes.c_void_p),
                            cost.ctypes.data_as(ctypes.c_void_p))
    if rc < 0:
        _bcheck(rc)
    return rc, order, wave, mem, cost


def batch_solve(problems, nroots, tol=1e-6, max_iter=300, precision="bf16x3", mem_budget=0, init_lanes=0,
                setup="fp64", refine="fp64"):
    """Solve many problems given as host arrays (``adc_batch_solve``): (omega, err64, status, info, rc)."""
    n = len(problems)
    arr, keep = _problems(problems)
    o = adc_batch_opts(int(mem_budget), int(init_lanes), 0, PRECISIONS[setup], PRECISIONS[refine])
    omega = np.empty((n, nroots), dtype=np.float64)
    err = np.empty((n, nroots), dtype=np.float64)
    status = np.empty(n, dtype=np.int32)
    info = adc_batch_info()
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    rc = lib.adc_batch_solve(n, arr, int(nroots), float(tol), int(max_iter), p, ctypes.byref(o),
                             omega.ctypes.data_as(ctypes.c_void_p), err.ctypes.data_as(ctypes.c_void_p),
                             status.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info))
    del keep
    if rc not in (0, -4):
        _bcheck(rc)
    return omega, err, status, info.as_dict(), rc


def ssfns(B, eps_occ, eps_vir, kind="EA", order=3, x=1.0, nroots=1, eta_crit=1e-5, tol=1e-8, max_iter=300,
          precision="fp64", refine="fp64"):
    """State-specific natural-spinor energies of the nroots lowest EA/EE roots (``adc_ssfns``,
    Sec. 2.4, Eqs. 31-32): a list of dicts (omega_corrected, omega_fns, omega2_canonical, omega2_fns,
    err64, n_keep, status)."""
    B = np.ascontiguousarray(B, dtype=np.complex128)
    eo = np.ascontiguousarray(eps_occ, dtype=np.float64)
    ev = np.ascontiguousarray(eps_vir, dtype=np.float64)
    o = adc_opts()
    lib.adc_opts_default(ctypes.byref(o))
    o.refine = PRECISIONS[refine] if isinstance(refine, str) else int(refine)
    out = (adc_ssfns_root * int(nroots))()
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    rc = lib.adc_ssfns(B.ctypes.data, B.shape[0], eo.ctypes.data, eo.shape[0], ev.ctypes.data, ev.shape[0],
                       KINDS[kind], int(order), float(x), int(nroots), float(eta_crit), float(tol), int(max_iter), p,
                       ctypes.byref(o), out)
    _check(rc)
    return [r.as_dict() for r in out]


def cholesky(V, tau, max_rank=None):
    """Pivoted Cholesky vectors of the PSD matrix V [n][n] (``adc_cholesky``, Eq. 41): (L [rank][n], pivots)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    n = V.shape[0]
    mr = n if max_rank is None else int(max_rank)
    L = np.zeros((mr, n), dtype=np.float64)
    piv = np.zeros(mr, dtype=np.int64)
    r = ctypes.c_int64()
    _check(lib.adc_cholesky(V.ctypes.data, n, float(tau), mr, L.ctypes.data, piv.ctypes.data, ctypes.byref(r)))
    return L[:r.value].copy(), piv[:r.value].copy()


def cholesky_mo(L, nao, C):
    """Cholesky vectors in the spinor basis C [nao][nmo] (``adc_cholesky_mo``, Eq. 42): B [rank][nmo][nmo]."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.complex128)
    rank, nmo = L.shape[0], C.shape[1]
    B = np.empty((rank, nmo, nmo), dtype=np.complex128)
    _check(lib.adc_cholesky_mo(L.ctypes.data, rank, int(nao), C.ctypes.data, nmo, B.ctypes.data))
    return B


def diag_gemm(which, M, N, K, seed=1, reps=3):
    """Accuracy and time of one contraction kernel (``adc_diag_gemm``): (rel_err, ms)."""
    e, t = ctypes.c_double(), ctypes.c_double()
    rc = lib.adc_diag_gemm(int(which), int(M), int(N), int(K), int(seed), int(reps), ctypes.byref(e),
                           ctypes.byref(t))
    _check(rc)
    return e.value, t.value


def diag_blockops(which, m, nb, n, seed=1, reps=3):
    """Accuracy and time of a Davidson block kernel (``adc_diag_blockops``; 0 gram, 1 combine): (rel_err, ms)."""
    e, t = ctypes.c_double(), ctypes.c_double()
    _check(lib.adc_diag_blockops(int(which), int(m), int(nb), int(n), int(seed), int(reps), ctypes.byref(e),
                                 ctypes.byref(t)))
    return e.value, t.value


def diag_eigh(which, A):
    """Small Hermitian eigensolver on the device (``adc_diag_eigh``; 0 FP64 Jacobi, 1 FP32 start + FP64
    refinement): (w ascending, V with eigenvectors as columns, ms, refinement steps; -1 = the FP64 Jacobi
    took over, 0 for which 0)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n = A.shape[0]
    w = np.empty(n, dtype=np.float64)
    V = np.empty((n, n), dtype=np.complex128)
    t = ctypes.c_double()
    st = ctypes.c_int()
    _check(lib.adc_diag_eigh(int(which), A.ctypes.data, n, w.ctypes.data, V.ctypes.data, ctypes.byref(t),
                             ctypes.byref(st)))
    return w, V, t.value, st.value


def diag_fp64_peak(blocks, iters):
    """FP64 FMA throughput probe (``adc_diag_fp64_peak``): (TFLOP/s, ms)."""
    f, t = ctypes.c_double(), ctypes.c_double()
    _check(lib.adc_diag_fp64_peak(int(blocks), int(iters), ctypes.byref(f), ctypes.byref(t)))
    return f.value, t.value


def launch_count():
    """Kernels launched by the library in this process (``adc_launch_count``)."""
    return int(lib.adc_launch_count())


__all__ = ["Context", "Batch", "batch_plan", "batch_solve", "AdcError", "diag_gemm", "diag_blockops", "diag_eigh", "diag_fp64_peak",
           "launch_count", "lib", "LIB_PATH", "ADC_IP", "ADC_EA", "ADC_EE",
           "ADC_PREC_FP64", "ADC_PREC_BF16X3", "ADC_PREC_BF16X6"]
