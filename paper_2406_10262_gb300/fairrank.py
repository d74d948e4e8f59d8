"""ctypes binding of libfairrank (include/fairrank.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays / torch tensors to
pointers, passes torch's current CUDA stream, and turns error statuses into exceptions. It loads
paper_2406_10262_gb300/_build/libfairrank.so and raises if the library is missing -- there is no
fallback path.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfairrank.so")

PARAM_FULL_C, PARAM_ITEM = 0, 1
GRAD_IMPLICIT, GRAD_UNROLLED = 0, 1
ADAM, SGD = 0, 1
F32, BF16, F64 = 0, 1, 2
STATUS = {0: "FR_OK", 1: "FR_EINVAL", 2: "FR_ENOMEM", 3: "FR_ECUDA", 4: "FR_ENUMERIC",
          5: "FR_ETIMEOUT", 6: "FR_ESTATE", 7: "FR_EUNSUPPORTED"}


class Config(ct.Structure):
    _fields_ = [
        ("n_users", ct.c_int32), ("n_items", ct.c_int32), ("n_slots", ct.c_int32),
        ("param", ct.c_int32), ("epsilon", ct.c_double), ("sinkhorn_iters", ct.c_int32),
        ("warm_start", ct.c_int32), ("grad_mode", ct.c_int32), ("ckpt_every", ct.c_int32),
        ("optimizer", ct.c_int32), ("lr", ct.c_double), ("beta1", ct.c_double),
        ("beta2", ct.c_double), ("adam_eps", ct.c_double), ("rel_dtype", ct.c_int32),
        ("max_wait_polls", ct.c_int32), ("reserved", ct.c_int32 * 6),
    ]


class FairRankError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_vp, _dp, _fp = ct.c_void_p, ct.POINTER(ct.c_double), ct.c_void_p


def lib():
    """The loaded shared library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfairrank is not built ({LIB_PATH} missing): run "
                               "`python -m paper_2406_10262_gb300.build`")
        L = ct.CDLL(LIB_PATH)
        i32, i64, d = ct.c_int32, ct.c_int64, ct.c_double
        sig = {
            "fr_config_default": (None, [ct.POINTER(Config), i32, i32, i32, i32]),
            "fr_num_cols": (i32, [i32, i32]),
            "fr_create": (i32, [ct.POINTER(Config), _vp, ct.POINTER(_vp)]),
            "fr_destroy": (i32, [_vp]),
            "fr_reset": (i32, [_vp]),
            "fr_set_relevance": (i32, [_vp, _vp, i32, i64, i32]),
            "fr_set_exposure": (i32, [_vp, _dp, i32]),
            "fr_step": (i32, [_vp, i32, _dp]),
            "fr_solve": (i32, [_vp, d, i32, ct.POINTER(i32), _dp]),
            "fr_impacts": (i32, [_vp, _dp, _dp, _dp]),
            "fr_policy": (i32, [_vp, i32, i32, _vp, i32]),
            "fr_grad": (i32, [_vp, _vp, _vp, _vp, i32]),
            "fr_set_state": (i32, [_vp, _vp, _vp, _vp, _vp, i64, i32]),
            "fr_get_state": (i32, [_vp, _vp, _vp, _vp, _vp, ct.POINTER(i64), i32]),
            "fr_metrics": (i32, [_vp, _dp, _dp, _dp, _dp]),
            "fr_item_envy": (i32, [_vp, _dp]),
            "fr_trace": (i32, [_vp, i32, _dp, _dp, ct.POINTER(i32)]),
            "fr_certificate": (i32, [_vp, _dp, _dp]),
            "fr_last_error": (ct.c_char_p, [_vp]),
            "fr_launch_count": (i64, [_vp]),
            "fr_measure_ex2_rate": (i32, [_dp]),
            "fr_time_kernels": (i32, [_vp, i32, _dp]),
            "fr_kernel_variant": (i32, [_vp, ct.POINTER(i32)]),
            "fr_sweep_stats": (i32, [_vp, ct.POINTER(i64)]),
            "fr_set_wait_limit": (i32, [_vp, i32]),
            "fr_measure_peaks": (i32, [_dp, i32]),
            "fr_check_log2_near1": (i32, [_dp]),
            "fr_batch_create": (i32, [ct.POINTER(Config), i32, _vp, ct.POINTER(_vp)]),
            "fr_batch_destroy": (i32, [_vp]),
            "fr_batch_reset": (i32, [_vp]),
            "fr_batch_set_relevance": (i32, [_vp, i32, _vp, i32, i64, i32]),
            "fr_batch_set_exposure": (i32, [_vp, i32, _dp, i32]),
            "fr_batch_autotune": (i32, [_vp]),
            "fr_batch_step": (i32, [_vp, i32, _dp]),
            "fr_batch_impacts": (i32, [_vp, i32, _dp, _dp, _dp]),
            "fr_batch_policy": (i32, [_vp, i32, i32, i32, _vp, i32]),
            "fr_batch_get_theta": (i32, [_vp, i32, _vp]),
            "fr_batch_tuning": (i32, [_vp, ct.POINTER(i32), _vp, i32]),
            "fr_batch_last_error": (ct.c_char_p, [_vp]),
            "fr_batch_launch_count": (i64, [_vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ct.c_void_p(0)


def _ptr(x, dtype=None):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None, 0, None
    if isinstance(x, np.ndarray):
        if dtype is not None:
            x = np.ascontiguousarray(x, dtype=dtype)
        else:
            x = np.ascontiguousarray(x)
        return ct.c_void_p(x.ctypes.data), 0, x
    import torch
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ct.c_void_p(x.data_ptr()), int(x.is_cuda), x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _rows(x):
    """(pointer, on_device, keepalive, ld) of a 2-D row-major numpy array or torch tensor whose
    rows may be padded (unit stride within a row, ld >= n_cols elements between rows): views such
    as wide[:, :n] pass without a copy; other layouts are copied to a dense array first."""
    if isinstance(x, np.ndarray):
        if (x.ndim == 2 and x.strides[1] == x.itemsize and x.strides[0] % x.itemsize == 0
                and x.strides[0] >= x.shape[1] * x.itemsize):
            return ct.c_void_p(x.ctypes.data), 0, x, x.strides[0] // x.itemsize
        c = np.ascontiguousarray(x)
        return ct.c_void_p(c.ctypes.data), 0, c, c.shape[1]
    import torch
    if isinstance(x, torch.Tensor):
        if x.dim() == 2 and x.stride(1) == 1 and x.stride(0) >= x.shape[1]:
            return ct.c_void_p(x.data_ptr()), int(x.is_cuda), x, x.stride(0)
        c = x.contiguous()
        return ct.c_void_p(c.data_ptr()), int(c.is_cuda), c, c.shape[1]
    raise TypeError(f"unsupported buffer type {type(x)}")


def num_cols(n_items: int, n_slots: int) -> int:
    return lib().fr_num_cols(n_items, n_slots)


def measure_ex2_rate() -> float:
    out = ct.c_double()
    st = lib().fr_measure_ex2_rate(ct.byref(out))
    if st:
        raise FairRankError(st, lib().fr_last_error(None).decode())
    return out.value


def measure_peaks() -> dict:
    """Measured on-chip rates of the current device (fr_measure_peaks)."""
    out = (ct.c_double * 6)()
    st = lib().fr_measure_peaks(out, 6)
    if st:
        raise FairRankError(st, lib().fr_last_error(None).decode())
    keys = ["ex2_per_s", "smem_bytes_per_s_8B", "smem_bytes_per_s_16B", "ffma_per_s",
            "ffma2_fmas_per_s", "sm_mhz"]
    return dict(zip(keys, list(out)))


def check_log2_near1() -> dict:
    """Self-check of the column updates' log2 near 1 over every float of its short path
    (fr_check_log2_near1)."""
    out = (ct.c_double * 3)()
    st = lib().fr_check_log2_near1(out)
    if st:
        raise FairRankError(st, lib().fr_last_error(None).decode())
    return {"max_rel_err": out[0], "log2f_max_rel_err": out[1], "nonzero_at_one": int(out[2])}


class FairRank:
    """One fair-ranking problem on the current CUDA device (wraps an fr_ctx)."""

    def __init__(self, n_users, n_items, n_slots, param=PARAM_FULL_C, **overrides):
        L = lib()
        cfg = Config()
        L.fr_config_default(ct.byref(cfg), n_users, n_items, n_slots, param)
        for k, v in overrides.items():
            if not hasattr(cfg, k):
                raise KeyError(k)
            setattr(cfg, k, v)
        self.cfg = cfg
        self.U, self.I, self.K = n_users, n_items, n_slots
        self.m = num_cols(n_items, n_slots)
        self.param = param
        h = ct.c_void_p()
        st = L.fr_create(ct.byref(cfg), _current_stream(), ct.byref(h))
        if st:
            raise FairRankError(st, L.fr_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().fr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st:
            raise FairRankError(st, lib().fr_last_error(self.h).decode())

    @property
    def nparam(self):
        return self.I if self.param == PARAM_ITEM else self.U * self.I * self.m

    # ---- inputs ---------------------------------------------------------------------------
    def set_relevance(self, r, dtype=None):
        """r: (U, I) numpy float32/float64, uint16 bfloat16 bits, or a torch tensor (host or CUDA);
        rows may be padded (a view of a wider array), which passes as the C ABI's ld."""
        import_dtype = dtype
        if import_dtype is None:
            kind = str(getattr(r, "dtype", ""))
            import_dtype = {"float32": F32, "torch.float32": F32, "float64": F64, "torch.float64": F64,
                            "uint16": BF16, "torch.bfloat16": BF16}.get(kind)
            if import_dtype is None:
                raise TypeError(f"unsupported relevance dtype {kind}")
        p, dev, keep, ld = _rows(r)
        self._check(lib().fr_set_relevance(self.h, p, import_dtype, ld, dev))

    def set_exposure(self, e):
        e = np.ascontiguousarray(e, dtype=np.float64)
        self._check(lib().fr_set_exposure(self.h, e.ctypes.data_as(_dp), e.shape[0]))

    def reset(self):
        self._check(lib().fr_reset(self.h))

    def set_wait_limit(self, max_wait_polls: int):
        """Polls of the bounded device-side waits (fr_config.max_wait_polls; 0 = default)."""
        self._check(lib().fr_set_wait_limit(self.h, max_wait_polls))

    # ---- Algorithm 1 ----------------------------------------------------------------------
    def step(self, n: int, trace: bool = True):
        F = np.zeros(max(n, 1))
        self._check(lib().fr_step(self.h, n, F.ctypes.data_as(_dp) if trace else None))
        return F[:n] if trace else None

    def solve(self, t: float, max_steps: int):
        done = ct.c_int32()
        F = ct.c_double()
        self._check(lib().fr_solve(self.h, t, max_steps, ct.byref(done), ct.byref(F)))
        return done.value, F.value

    def impacts(self):
        imp = np.zeros(self.I)
        util, F = ct.c_double(), ct.c_double()
        self._check(lib().fr_impacts(self.h, imp.ctypes.data_as(_dp), ct.byref(util), ct.byref(F)))
        return imp, util.value, F.value

    def policy(self, u0=0, n_u=None, out=None):
        n_u = self.U - u0 if n_u is None else n_u
        if out is None:
            out = np.zeros((n_u, self.I, self.m), dtype=np.float32)
        p, dev, keep = _ptr(out)
        self._check(lib().fr_policy(self.h, u0, n_u, p, dev))
        return out

    def grad(self, omega=None, want_dr=False, device=False):
        if device:
            import torch
            shape = (self.I,) if self.param == PARAM_ITEM else (self.U, self.I, self.m)
            dp = torch.zeros(shape, dtype=torch.float32, device="cuda")
            dr = torch.zeros((self.U, self.I), dtype=torch.float32, device="cuda") if want_dr else None
        else:
            shape = (self.I,) if self.param == PARAM_ITEM else (self.U, self.I, self.m)
            dp = np.zeros(shape, dtype=np.float32)
            dr = np.zeros((self.U, self.I), dtype=np.float32) if want_dr else None
        om = None if omega is None else (omega if not isinstance(omega, np.ndarray)
                                         else np.ascontiguousarray(omega, dtype=np.float32))
        po, _, k1 = _ptr(om)
        pp, dev, k2 = _ptr(dp)
        pr, _, k3 = _ptr(dr)
        self._check(lib().fr_grad(self.h, po, pp, pr, dev))
        return (dp, dr) if want_dr else dp

    def set_state(self, param=None, m1=None, m2=None, g=None, t=0):
        conv = lambda a: None if a is None else (np.ascontiguousarray(a, dtype=np.float32)
                                                 if isinstance(a, np.ndarray) else a)
        ps = [_ptr(conv(a)) for a in (param, m1, m2, g)]
        dev = max([q[1] for q in ps if q[0] is not None] or [0])
        self._check(lib().fr_set_state(self.h, ps[0][0], ps[1][0], ps[2][0], ps[3][0], t, dev))

    def get_state(self):
        shape = (self.I,) if self.param == PARAM_ITEM else (self.U, self.I, self.m)
        p, m1, m2 = (np.zeros(shape, np.float32) for _ in range(3))
        g = np.zeros((self.U, self.m), np.float32)
        t = ct.c_int64()
        self._check(lib().fr_get_state(self.h, ct.c_void_p(p.ctypes.data), ct.c_void_p(m1.ctypes.data),
                                       ct.c_void_p(m2.ctypes.data), ct.c_void_p(g.ctypes.data),
                                       ct.byref(t), 0))
        return p, m1, m2, g, t.value

    def metrics(self):
        vals = [ct.c_double() for _ in range(4)]
        self._check(lib().fr_metrics(self.h, *[ct.byref(v) for v in vals]))
        return dict(zip(["utility", "mean_envy", "better_pct", "worse_pct"], [v.value for v in vals]))

    def trace(self):
        """(F after each step, gradient norm of each step) of the last step() / solve() call."""
        n = ct.c_int32()
        self._check(lib().fr_trace(self.h, 0, None, None, ct.byref(n)))
        F, gn = np.zeros(n.value), np.zeros(n.value)
        self._check(lib().fr_trace(self.h, n.value, F.ctypes.data_as(_dp), gn.ctypes.data_as(_dp), None))
        return F, gn

    def item_envy(self):
        """Per-item envy max_j (Imp_i(X_j) - Imp_i(X_i)) at the current policy, [n_items] doubles."""
        out = np.zeros(self.I)
        self._check(lib().fr_item_envy(self.h, out.ctypes.data_as(_dp)))
        return out

    def certificate(self):
        """(gap, column residual): Frank-Wolfe bound on F* - F at the current policy."""
        gap, res = ct.c_double(), ct.c_double()
        self._check(lib().fr_certificate(self.h, ct.byref(gap), ct.byref(res)))
        return gap.value, res.value

    def time_kernels(self, n_steps: int):
        ms = np.zeros(3)
        self._check(lib().fr_time_kernels(self.h, n_steps, ms.ctypes.data_as(_dp)))
        return ms

    def launch_count(self) -> int:
        return lib().fr_launch_count(self.h)

    def kernel_variant(self) -> dict:
        """The compiled Sinkhorn-sweep variant serving this context (see fr_kernel_variant)."""
        o = (ct.c_int32 * 6)()
        self._check(lib().fr_kernel_variant(self.h, o))
        return {"n_cols_kernel": o[0], "rows_per_thread": o[1], "exact": bool(o[2]),
                "threads": o[3], "tile_stride": o[4], "grid": o[5]}

    def log_form_solves(self) -> int:
        """Tile-sweep solves since the last reset that finished in the log form (fr_sweep_stats)."""
        o = ct.c_int64()
        self._check(lib().fr_sweep_stats(self.h, ct.byref(o)))
        return o.value


class FairRankBatch:
    """Many independent markets advanced together (wraps an fr_batch), all FR_PARAM_ITEM or all
    FR_PARAM_FULL_C.

    sizes: sequence of (n_users, n_items, n_slots); overrides apply to every market's config."""

    def __init__(self, sizes, param=PARAM_ITEM, **overrides):
        L = lib()
        n = len(sizes)
        cfgs = (Config * n)()
        for j, (U, I, K) in enumerate(sizes):
            L.fr_config_default(ct.byref(cfgs[j]), U, I, K, param)
            for k, v in overrides.items():
                if not hasattr(cfgs[j], k):
                    raise KeyError(k)
                setattr(cfgs[j], k, v)
        self.sizes = [tuple(x) for x in sizes]
        self.M = n
        h = ct.c_void_p()
        st = L.fr_batch_create(cfgs, n, _current_stream(), ct.byref(h))
        if st:
            raise FairRankError(st, L.fr_batch_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().fr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st:
            raise FairRankError(st, lib().fr_batch_last_error(self.h).decode())

    def set_relevance(self, market, r):
        kind = str(getattr(r, "dtype", ""))
        dt = {"float32": F32, "float64": F64, "uint16": BF16, "torch.float32": F32,
              "torch.float64": F64, "torch.bfloat16": BF16}.get(kind)
        if dt is None:
            raise TypeError(f"unsupported relevance dtype {kind}")
        p, dev, keep, ld = _rows(r)
        self._check(lib().fr_batch_set_relevance(self.h, market, p, dt, ld, dev))

    def set_exposure(self, market, e):
        e = np.ascontiguousarray(e, dtype=np.float64)
        self._check(lib().fr_batch_set_exposure(self.h, market, e.ctypes.data_as(_dp), e.shape[0]))

    def reset(self):
        self._check(lib().fr_batch_reset(self.h))

    def autotune(self):
        self._check(lib().fr_batch_autotune(self.h))

    def step(self, n: int, trace: bool = True):
        F = np.zeros((max(n, 1), self.M))
        self._check(lib().fr_batch_step(self.h, n, F.ctypes.data_as(_dp) if trace else None))
        return F[:n] if trace else None

    def impacts(self, market):
        imp = np.zeros(self.sizes[market][1])
        util, F = ct.c_double(), ct.c_double()
        self._check(lib().fr_batch_impacts(self.h, market, imp.ctypes.data_as(_dp), ct.byref(util),
                                           ct.byref(F)))
        return imp, util.value, F.value

    def policy(self, market, u0=0, n_u=None):
        U, I, K = self.sizes[market]
        n_u = U - u0 if n_u is None else n_u
        out = np.zeros((n_u, I, num_cols(I, K)), dtype=np.float32)
        self._check(lib().fr_batch_policy(self.h, market, u0, n_u, ct.c_void_p(out.ctypes.data), 0))
        return out

    def theta(self, market):
        out = np.zeros(self.sizes[market][1], dtype=np.float32)
        self._check(lib().fr_batch_get_theta(self.h, market, ct.c_void_p(out.ctypes.data)))
        return out

    def tuning(self):
        n = ct.c_int32()
        self._check(lib().fr_batch_tuning(self.h, ct.byref(n), None, 0))
        t = np.zeros((max(n.value, 1), 6), dtype=np.int32)
        self._check(lib().fr_batch_tuning(self.h, ct.byref(n), ct.c_void_p(t.ctypes.data), n.value))
        keys = ["n_cols_kernel", "markets", "max_items", "rows_per_thread", "threads",
                "consumers_per_chunk"]
        return [dict(zip(keys, map(int, row))) for row in t[:n.value]]

    def launch_count(self) -> int:
        return lib().fr_batch_launch_count(self.h)
