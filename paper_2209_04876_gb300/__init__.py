"""GB300 (sm_103a) Kronecker regression: Python binding of libkron.

Thin ctypes layer over the C ABI declared in include/kron.h: every function here
only marshals tensors and options into the C structures and calls the entry point
of the same name. All computation runs in the library's CUDA kernels. PyTorch is
used for device memory and streams only. If libkron.so has not been built, every
entry point raises: there is no fallback implementation.
"""
import ctypes
import math
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkron.so")
MAX_MODES = 8

STATUS = {0: "KR_OK", 1: "KR_EINVAL", 2: "KR_ENOMEM", 3: "KR_ECUDA", 4: "KR_ENONFINITE", 5: "KR_ERANK",
          6: "KR_ENOTCONV", 7: "KR_EDIVERGED", 8: "KR_ETIMEOUT", 9: "KR_ENOTIMPL"}
KERNEL_KINDS = {"resid": 0, "modeprod": 1, "sample": 2, "scatter": 3, "dedup": 4, "tables": 5, "vector": 6,
                "slab": 7}
OPT_SLAB_PASS, OPT_SLAB_TILE_ENTRIES, OPT_DEVICE_LOOP, OPT_BATCH_WORKERS, OPT_GROUPING, OPT_HOST_GATHER = 1, 2, 3, 4, 5, 6
OPT_JL_K, OPT_JL_SEED, OPT_TENSOR_CORES, OPT_BATCH_MODE, OPT_AUTOTUNE = 7, 8, 9, 10, 11
EXPORTED = ["kr_create", "kr_destroy", "kr_set_stream", "kr_last_error", "kr_launch_count", "kr_tc_launch_count", "kr_graph_count", "kr_autotune_report", "kr_timing_enable",
            "kr_timing_read", "kr_timing_reset", "kr_set_option", "kron_sample_count", "kron_leverage",
            "kron_sample", "kron_sample_noalloc", "kron_sketch", "kron_sketch_distinct", "kron_sketch_export", "kron_sketch_residual",
            "kron_sketch_free", "kron_matmul", "kron_precond", "kron_objective", "kron_regress", "kron_ridge", "kron_regress_async", "kron_ridge_async",
            "kron_ridge_batched", "tucker_factor_update", "tucker_als_sweep", "tucker_als_exact_sweep", "tucker_rre"]


class KronError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status
        self.name = STATUS.get(status, str(status))


class KrFactors(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("I", ctypes.c_int64 * MAX_MODES), ("R", ctypes.c_int32 * MAX_MODES),
                ("A", ctypes.c_void_p * MAX_MODES)]


class KrOpts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("delta", ctypes.c_double), ("lam", ctypes.c_double),
                ("sample_scale", ctypes.c_double), ("num_samples", ctypes.c_int64), ("max_iter", ctypes.c_int32),
                ("tol", ctypes.c_double), ("step", ctypes.c_double), ("precision", ctypes.c_int32),
                ("host_io", ctypes.c_int32), ("seed", ctypes.c_uint64), ("call_id", ctypes.c_uint64),
                ("partition_T", ctypes.c_int32), ("deterministic", ctypes.c_int32), ("stop_rule", ctypes.c_int32),
                ("theta", ctypes.c_double)]


class KrReport(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("s", ctypes.c_int64),
                ("distinct", ctypes.c_int64), ("obj_sampled", ctypes.c_double), ("rel_update", ctypes.c_double),
                ("t_ms", ctypes.c_float * 8), ("iters_reduced", ctypes.c_int32), ("precision_used", ctypes.c_int32)]

    def as_dict(self):
        names = ["leverage", "sample_group_gather", "unused", "init", "iterate", "final_check", "copies", "total"]
        return dict(iters=self.iters, converged=bool(self.converged), stop=int(self.converged), s=self.s,
                    distinct=self.distinct,
                    obj_sampled=self.obj_sampled, rel_update=self.rel_update,
                    iters_reduced=self.iters_reduced, precision_used=self.precision_used,
                    t_ms={k: float(v) for k, v in zip(names, self.t_ms)})


class KrDevReport(ctypes.Structure):
    """kr_dev_report: an asynchronous solve's report, written in device memory."""
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("iters_reduced", ctypes.c_int32), ("precision_used", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("s", ctypes.c_int64), ("distinct", ctypes.c_int64), ("obj_sampled", ctypes.c_double),
                ("rel_update", ctypes.c_double)]


_lib = None
_ctx = {}


def lib():
    """The loaded libkron (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libkron.so is missing (%s): build it with __graft_entry__.build() or "
                               "python -m paper_2209_04876_gb300.build" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        P = ctypes.POINTER
        sig = {
            "kr_create": (i32, [P(vp), vp, ctypes.c_size_t]),
            "kron_sample_count": (i64, [i64, dbl, dbl]),
            "kr_destroy": (None, [vp]),
            "kr_set_stream": (i32, [vp, vp]),
            "kr_last_error": (ctypes.c_char_p, [vp]),
            "kr_launch_count": (i64, [vp]),
            "kr_tc_launch_count": (i64, [vp]),
            "kr_graph_count": (i64, [vp]),
            "kr_autotune_report": (i64, [vp, ctypes.c_char_p, i64]),
            "kr_timing_enable": (i32, [vp, i32]),
            "kr_timing_read": (i32, [vp, i32, P(dbl), P(i64)]),
            "kr_timing_reset": (i32, [vp]),
            "kr_set_option": (i32, [vp, i32, i64]),
            "kron_leverage": (i32, [vp, P(KrFactors), P(vp), P(vp), P(vp), P(i32)]),
            "kron_sample": (i32, [vp, i32, P(i64), P(vp), P(vp), i64, u64, u64, i32, vp, vp]),
            "kron_sample_noalloc": (i32, [vp, i32, P(i64), P(vp), P(vp), i64, u64, u64, i32, vp, vp]),
            "kron_sketch": (i32, [vp, P(KrFactors), P(vp), P(vp), vp, i64, u64, u64, i32, P(vp)]),
            "kron_sketch_distinct": (i64, [vp]),
            "kron_sketch_export": (i32, [vp, vp, vp, vp, vp, vp]),
            "kron_sketch_residual": (i32, [vp, vp, P(KrFactors), vp, vp, P(dbl)]),
            "kron_sketch_free": (None, [vp]),
            "kron_matmul": (i32, [vp, i32, P(i64), P(i64), P(vp), P(i32), vp, vp]),
            "kron_precond": (i32, [vp, P(KrFactors), dbl, vp, vp]),
            "kron_objective": (i32, [vp, P(KrFactors), vp, vp, dbl, P(dbl)]),
            "kron_regress": (i32, [vp, P(KrFactors), vp, P(KrOpts), vp, P(KrReport)]),
            "kron_ridge": (i32, [vp, P(KrFactors), vp, P(KrOpts), vp, P(KrReport)]),
            "kron_regress_async": (i32, [vp, P(KrFactors), vp, P(KrOpts), vp, vp]),
            "kron_ridge_async": (i32, [vp, P(KrFactors), vp, P(KrOpts), vp, vp]),
            "kron_ridge_batched": (i32, [vp, i32, P(KrFactors), P(vp), P(KrOpts), P(vp), P(KrReport)]),
            "tucker_factor_update": (i32, [vp, i32, P(i64), P(i32), vp, P(vp), vp, i32, P(KrOpts), P(KrReport)]),
            "tucker_als_sweep": (i32, [vp, i32, P(i64), P(i32), vp, P(vp), vp, P(KrOpts), i32, P(KrReport)]),
            "tucker_als_exact_sweep": (i32, [vp, i32, P(i64), P(i32), vp, P(vp), vp, dbl, i32, P(dbl)]),
            "tucker_rre": (i32, [vp, i32, P(i64), P(i32), vp, P(vp), vp, P(dbl)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


_lib_streams = {}


def _stream_for(dev):
    """The stream the library runs on: torch's current stream, or, when that is the legacy
    default stream (which CUDA graphs cannot capture, so the device-side loops would fall
    back to host loops), a per-device library stream that first waits for the current
    stream's work. Every library call synchronises its stream before it returns, so results
    are complete when the call returns."""
    cur = torch.cuda.current_stream(dev)
    if cur.cuda_stream != 0:
        return cur
    s = _lib_streams.get(dev)
    if s is None:
        s = _lib_streams[dev] = torch.cuda.Stream(dev)
    s.wait_stream(cur)
    return s


def context(device=None):
    """Per-device library context, bound at each call to torch's current stream (or to the
    library stream that stands in for the legacy default stream)."""
    dev = torch.cuda.current_device() if device is None else int(device)
    L = lib()
    if dev not in _ctx:
        with torch.cuda.device(dev):
            h = ctypes.c_void_p()
            st = L.kr_create(ctypes.byref(h), ctypes.c_void_p(_stream_for(dev).cuda_stream), 0)
            if st != 0:
                raise KronError(st, "kr_create failed")
            _ctx[dev] = h
    h = _ctx[dev]
    L.kr_set_stream(h, ctypes.c_void_p(_stream_for(dev).cuda_stream))
    return h


def launch_count():
    """Kernels launched by the library on this device's context so far."""
    return int(lib().kr_launch_count(context()))


def tc_launch_count():
    """Launches of the tcgen05 tensor-core mode product on this device's context so far."""
    return int(lib().kr_tc_launch_count(context()))


def graph_count():
    """CUDA graphs the library launched on this device's context so far."""
    return int(lib().kr_graph_count(context()))


def autotune_report():
    """The autotuner's choices (OPT_AUTOTUNE): one dict per shape class with its key
    (N, I_{N-1}, R_{N-1}, I_N, R_N, floor(log2 s)), the chosen slab tile budget and the
    measured slab-pass milliseconds at each candidate budget."""
    h = context()
    n = int(lib().kr_autotune_report(h, None, 0))
    buf = ctypes.create_string_buffer(n + 1)
    lib().kr_autotune_report(h, buf, n + 1)
    out = []
    for line in buf.value.decode().splitlines():
        f = line.split()
        out.append(dict(key=tuple(int(v) for v in f[:6]), budget=int(f[6]),
                        ms={c: float(v) for c, v in zip((2048, 4096, 8192, 16384, 32768), f[7:])}))
    return out


def timing_enable(on=True):
    h = context()
    _check(lib().kr_timing_enable(h, int(bool(on))), h)


def set_option(key, value):
    """Context option (OPT_SLAB_PASS: 1 fused slab pass where the shape allows, 0 the
    per-cell residual pass; OPT_SLAB_TILE_ENTRIES: entry budget of a slab-pass tile;
    OPT_DEVICE_LOOP: 1 Richardson steps as one CUDA graph, 0 host loop; OPT_BATCH_WORKERS:
    problems of kron_ridge_batched solved concurrently, 1..32; OPT_GROUPING: draws grouped
    by 0 automatic choice, 1 radix sort, 2 ranks in a bitmap of the key space, 3 ranks with dense
    per-key counters; OPT_HOST_GATHER: 1 host-buffer solves gather the sampled entries of a
    page-locked b in place, 0 copy b; OPT_JL_K: 0 exact leverage scores, k in [1, 64]
    JL-approximate scores with k sign columns; OPT_JL_SEED: their Philox key; OPT_TENSOR_CORES:
    1 contiguous-index mode products of KronMatMul on tcgen05 in 3xTF32, 0 CUDA cores;
    OPT_BATCH_MODE: kron_ridge_batched 0 on worker contexts, 1 fused (one context per problem,
    all Richardson loops as concurrent nodes of one CUDA graph); OPT_AUTOTUNE: 1 chooses the
    slab tile budget per shape class by measurement, see autotune_report())."""
    h = context()
    _check(lib().kr_set_option(h, int(key), int(value)), h)


def timing_reset():
    h = context()
    _check(lib().kr_timing_reset(h), h)


def timing_read():
    """{kind: (total_ms, launches)} from the library's per-launch event pairs."""
    h = context()
    out = {}
    for name, k in KERNEL_KINDS.items():
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(lib().kr_timing_read(h, k, ctypes.byref(ms), ctypes.byref(n)), h)
        out[name] = (ms.value, n.value)
    return out


def _check(st, h):
    if st != 0:
        raise KronError(st, lib().kr_last_error(h).decode(errors="replace"))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dev_f32(t, device=None):
    t = torch.as_tensor(t)
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        t = t.to(device="cuda" if device is None else device, dtype=torch.float32).contiguous()
    return t


def _inout(t, name):
    """In-place arguments must already be contiguous float32 device tensors (no copy)."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("%s must be a contiguous float32 CUDA tensor (it is updated in place)" % name)
    return t


def _factors(As, host=False):
    f = KrFactors()
    f.N = len(As)
    if not 1 <= f.N <= MAX_MODES:
        raise ValueError("between 1 and %d factors" % MAX_MODES)
    for n, A in enumerate(As):
        f.I[n] = A.shape[0]
        f.R[n] = A.shape[1]
        f.A[n] = A.data_ptr()
    return f


def _ptr_array(ts):
    arr = (ctypes.c_void_p * max(1, len(ts)))()
    for i, t in enumerate(ts):
        arr[i] = t.data_ptr() if t is not None else None
    return arr


STOP_STEP, STOP_EPS = 0, 1


def _opts(eps=0.1, lam=0.0, seed=0, call_id=0, sample_scale=4.0, num_samples=0, max_iter=100, tol=1e-7, step=0.0,
          precision=0, host_io=False, delta=0.01, partition_T=0, deterministic=1, stop_rule=STOP_STEP, theta=0.0):
    o = KrOpts()
    o.eps, o.delta, o.lam, o.sample_scale = eps, delta, lam, sample_scale
    o.num_samples, o.max_iter, o.tol, o.step = int(num_samples), int(max_iter), tol, step
    o.precision, o.host_io, o.seed, o.call_id = int(precision), int(bool(host_io)), int(seed), int(call_id)
    o.partition_T, o.deterministic, o.stop_rule, o.theta = int(partition_T), int(deterministic), int(stop_rule), theta
    return o


def kron_sample_count(R, eps, c=4.0):
    """The library's default sample count for R unknowns (kron_sample_count in kron.h)."""
    v = int(lib().kron_sample_count(int(R), float(eps), float(c)))
    if v < 0:
        raise ValueError("kron_sample_count: eps must lie in (0, 1) and R >= 1")
    return v


# ---------------------------------------------------------------------------- entry points

def kron_leverage(As):
    """Leverage scores, CDFs, probabilities and ranks of the factors (device tensors)."""
    As = [_dev_f32(A) for A in As]
    h = context()
    lev = [torch.empty(A.shape[0], dtype=torch.float64, device=A.device) for A in As]
    cdf = [torch.empty_like(l) for l in lev]
    prob = [torch.empty_like(l) for l in lev]
    rank = (ctypes.c_int32 * len(As))()
    f = _factors(As)
    st = lib().kron_leverage(h, ctypes.byref(f), _ptr_array(lev), _ptr_array(cdf), _ptr_array(prob), rank)
    _check(st, h)
    return dict(lev=lev, cdf=cdf, prob=prob, rank=list(rank))


def kron_sample(cdfs, probs, s, seed, call_id, row=0, want_idx=True, want_w=True):
    h = context()
    N = len(cdfs)
    I = (ctypes.c_int64 * N)(*[c.shape[0] for c in cdfs])
    dev = cdfs[0].device
    idx = torch.empty((s, N), dtype=torch.int32, device=dev) if want_idx else None
    w = torch.empty(s, dtype=torch.float32, device=dev) if want_w else None
    st = lib().kron_sample(h, N, I, _ptr_array(cdfs), _ptr_array(probs) if probs is not None else None, int(s),
                           int(seed), int(call_id), int(row), _ptr(idx), _ptr(w))
    _check(st, h)
    return idx, w


def _require(t, name, dtype, numel, dev):
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or t.device != dev \
            or not t.is_contiguous() or t.numel() < numel:
        raise ValueError("%s must be a contiguous %s tensor on %s with at least %d elements" % (name, dtype, dev, numel))


def kron_sample_noalloc(cdfs, probs, s, seed, call_id, row=0, idx=None, w=None):
    """kron_sample for callers that cannot allocate device memory: the outputs are the
    caller's (pass preallocated `idx` (s x N int32) / `w` (s float32) tensors, or let this
    wrapper create them before the call), and the library's only scratch is a fixed
    static device array (sum of table sizes <= 16384 rows). The kernel writes through the
    raw pointers, so every tensor is checked first (dtype, device, contiguity, size)."""
    N = len(cdfs)
    if N < 1:
        raise ValueError("kron_sample_noalloc: at least one table")
    dev = cdfs[0].device
    for m, c in enumerate(cdfs):
        _require(c, "cdfs[%d]" % m, torch.float64, c.shape[0] if c.dim() == 1 else -1, dev)
        if c.dim() != 1:
            raise ValueError("cdfs[%d] must be one-dimensional" % m)
    if probs is not None:
        if len(probs) != N:
            raise ValueError("kron_sample_noalloc: one probability table per CDF")
        for m, (p, c) in enumerate(zip(probs, cdfs)):
            _require(p, "probs[%d]" % m, torch.float64, c.shape[0], dev)
    h = context()
    I = (ctypes.c_int64 * N)(*[c.shape[0] for c in cdfs])
    if idx is None:
        idx = torch.empty((s, N), dtype=torch.int32, device=dev)
    if w is None and probs is not None:
        w = torch.empty(s, dtype=torch.float32, device=dev)
    _require(idx, "idx", torch.int32, int(s) * N, dev)
    if w is not None:
        if probs is None:
            raise ValueError("kron_sample_noalloc: weights need the probability tables")
        _require(w, "w", torch.float32, int(s), dev)
    st = lib().kron_sample_noalloc(h, N, I, _ptr_array(cdfs), _ptr_array(probs) if probs is not None else None,
                                   int(s), int(seed), int(call_id), int(row), _ptr(idx), _ptr(w))
    _check(st, h)
    return idx, w


class Sketch:
    """A sampled, grouped sketch of K's rows held in device memory by the library."""

    def __init__(self, handle, As):
        self.handle = handle
        self.As = As

    @property
    def distinct(self):
        return int(lib().kron_sketch_distinct(self.handle))

    def export(self):
        h = context()
        n = self.distinct
        dev = self.As[0].device
        keys = torch.empty(n, dtype=torch.int64, device=dev)
        counts = torch.empty(n, dtype=torch.int32, device=dev)
        omega = torch.empty(n, dtype=torch.float32, device=dev)
        bt = torch.empty(n, dtype=torch.float32, device=dev)
        _check(lib().kron_sketch_export(h, self.handle, _ptr(keys), _ptr(counts), _ptr(omega), _ptr(bt)), h)
        return keys, counts, omega, bt

    def residual(self, x, As=None):
        """g = K~^T Omega (b~ - K~ x) and sum omega (b~ - K~x)^2."""
        h = context()
        As = self.As if As is None else [_dev_f32(A) for A in As]
        x = _dev_f32(x)
        g = torch.empty_like(x)
        obj = ctypes.c_double()
        f = _factors(As)
        _check(lib().kron_sketch_residual(h, self.handle, ctypes.byref(f), _ptr(x), _ptr(g), ctypes.byref(obj)), h)
        return g, obj.value

    def free(self):
        if self.handle:
            lib().kron_sketch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def kron_sketch(As, cdfs, probs, b, s, seed, call_id, row=0):
    As = [_dev_f32(A) for A in As]
    b = _dev_f32(b) if b is not None else None
    h = context()
    out = ctypes.c_void_p()
    f = _factors(As)
    st = lib().kron_sketch(h, ctypes.byref(f), _ptr_array(cdfs), _ptr_array(probs), _ptr(b), int(s), int(seed),
                           int(call_id), int(row), ctypes.byref(out))
    _check(st, h)
    return Sketch(out, As)


def kron_matmul(Bs, x, trans=None):
    """(B1 (x) ... (x) BN) x; trans[n] = 1 uses Bn^T."""
    Bs = [_dev_f32(B) for B in Bs]
    x = _dev_f32(x)
    N = len(Bs)
    trans = [0] * N if trans is None else [int(t) for t in trans]
    J = [B.shape[1] if t else B.shape[0] for B, t in zip(Bs, trans)]
    K = [B.shape[0] if t else B.shape[1] for B, t in zip(Bs, trans)]
    y = torch.empty(int(math.prod(J)), dtype=torch.float32, device=x.device)
    h = context()
    st = lib().kron_matmul(h, N, (ctypes.c_int64 * N)(*J), (ctypes.c_int64 * N)(*K), _ptr_array(Bs),
                           (ctypes.c_int32 * N)(*trans), _ptr(x), _ptr(y))
    _check(st, h)
    return y


def kron_precond(As, g, lam=0.0):
    As = [_dev_f32(A) for A in As]
    g = _dev_f32(g)
    d = torch.empty_like(g)
    h = context()
    f = _factors(As)
    _check(lib().kron_precond(h, ctypes.byref(f), float(lam), _ptr(g), _ptr(d)), h)
    return d


def kron_objective(As, b, x, lam=0.0):
    As = [_dev_f32(A) for A in As]
    h = context()
    f = _factors(As)
    out = ctypes.c_double()
    _check(lib().kron_objective(h, ctypes.byref(f), _ptr(_dev_f32(b)), _ptr(_dev_f32(x)), float(lam),
                                ctypes.byref(out)), h)
    return out.value


def _solve(fn, As, b, raise_notconv, host_io, **kw):
    h = context()
    if host_io:
        As = [torch.as_tensor(A, dtype=torch.float32).contiguous() for A in As]
        b = torch.as_tensor(b, dtype=torch.float32).contiguous()
        R = int(math.prod(A.shape[1] for A in As))
        x = torch.empty(R, dtype=torch.float32, pin_memory=True)
    else:
        As = [_dev_f32(A) for A in As]
        b = _dev_f32(b)
        R = int(math.prod(A.shape[1] for A in As))
        x = torch.empty(R, dtype=torch.float32, device=b.device)
    f = _factors(As)
    o = _opts(host_io=host_io, **kw)
    rep = KrReport()
    st = fn(h, ctypes.byref(f), _ptr(b), ctypes.byref(o), _ptr(x), ctypes.byref(rep))
    if st != 0 and (raise_notconv or st != 6):
        _check(st, h)
    return x, rep.as_dict()


def kron_regress(As, b, eps=0.1, seed=0, call_id=0, raise_notconv=True, host_io=False, **kw):
    """Alg. 2 with lambda = 0; returns (x, report)."""
    return _solve(lib().kron_regress, As, b, raise_notconv, host_io, eps=eps, seed=seed, call_id=call_id, **kw)


def kron_ridge(As, b, lam, eps=0.1, seed=0, call_id=0, raise_notconv=True, host_io=False, **kw):
    """Alg. 2 with lambda > 0; returns (x, report)."""
    return _solve(lib().kron_ridge, As, b, raise_notconv, host_io, eps=eps, lam=lam, seed=seed, call_id=call_id,
                  **kw)


def _solve_async(fn, As, b, x, report, **kw):
    h = context()
    # no staging copies: the solve may still be running (or be replayed) after this returns
    As = [_inout(A, "As[%d]" % k) for k, A in enumerate(As)]
    b = _inout(b, "b")
    R = int(math.prod(A.shape[1] for A in As))
    if x is None:
        x = torch.empty(R, dtype=torch.float32, device=b.device)
    _inout(x, "x")
    if x.numel() != R:
        raise ValueError("x must hold prod R = %d floats" % R)
    nb = ctypes.sizeof(KrDevReport)
    if report is None:
        report = torch.zeros(nb, dtype=torch.uint8, device=b.device)
    if not (report.is_cuda and report.dtype == torch.uint8 and report.is_contiguous() and report.numel() >= nb):
        raise ValueError("report must be a contiguous CUDA uint8 tensor of at least %d bytes" % nb)
    f = _factors(As)
    o = _opts(**kw)
    _check(fn(h, ctypes.byref(f), _ptr(b), ctypes.byref(o), _ptr(x), _ptr(report)), h)
    dev = b.device.index if b.device.index is not None else torch.cuda.current_device()
    cur = torch.cuda.current_stream(dev)
    if cur.cuda_stream == 0 and dev in _lib_streams:  # later work on the current stream follows the solve
        cur.wait_stream(_lib_streams[dev])
    return x, report


def kron_regress_async(As, b, eps=0.1, seed=0, call_id=0, x=None, report=None, **kw):
    """kron_regress enqueued without waiting (or captured into the caller's CUDA graph when
    torch's current stream is capturing). Returns (x, report): report is a device uint8
    tensor holding a kr_dev_report once the solve has run; read it with read_dev_report."""
    return _solve_async(lib().kron_regress_async, As, b, x, report, eps=eps, seed=seed, call_id=call_id, **kw)


def kron_ridge_async(As, b, lam, eps=0.1, seed=0, call_id=0, x=None, report=None, **kw):
    """kron_ridge enqueued without waiting; see kron_regress_async."""
    return _solve_async(lib().kron_ridge_async, As, b, x, report, eps=eps, lam=lam, seed=seed, call_id=call_id,
                        **kw)


def read_dev_report(report):
    """The kr_dev_report in a device tensor, as a dict (copies it to the host: waits for the solve)."""
    nb = ctypes.sizeof(KrDevReport)
    r = KrDevReport.from_buffer_copy(bytes(report[:nb].cpu().numpy()))
    return dict(status=STATUS.get(r.status, r.status), iters=r.iters, converged=bool(r.converged),
                stop=int(r.converged), iters_reduced=r.iters_reduced, precision_used=r.precision_used, s=r.s,
                distinct=r.distinct, obj_sampled=r.obj_sampled, rel_update=r.rel_update)


def kron_ridge_batched(problems, lam, eps=0.1, seed=0, call_id=0, **kw):
    """problems: list of (As, b). Returns (list of x, list of reports)."""
    h = context()
    n = len(problems)
    fs = (KrFactors * n)()
    keep, bs, xs = [], [], []
    for p, (As, b) in enumerate(problems):
        As = [_dev_f32(A) for A in As]
        b = _dev_f32(b)
        keep.append((As, b))
        fs[p] = _factors(As)
        bs.append(b)
        xs.append(torch.empty(int(math.prod(A.shape[1] for A in As)), dtype=torch.float32, device=b.device))
    reps = (KrReport * n)()
    o = _opts(eps=eps, lam=lam, seed=seed, call_id=call_id, **kw)
    st = lib().kron_ridge_batched(h, n, fs, _ptr_array(bs), ctypes.byref(o), _ptr_array(xs), reps)
    if st not in (0, 6):
        _check(st, h)
    return xs, [r.as_dict() for r in reps]


def tucker_factor_update(X, As, G, n, lam, eps=0.1, seed=0, call_id=0, raise_notconv=True, **kw):
    """Alg. 3 for mode n: overwrites As[n] (device float32) in place; returns the report."""
    h = context()
    N = len(As)
    X = _dev_f32(X)
    for k, A in enumerate(As):
        _inout(A, "As[%d]" % k)
    _inout(G, "G")
    I = (ctypes.c_int64 * N)(*[A.shape[0] for A in As])
    R = (ctypes.c_int32 * N)(*[A.shape[1] for A in As])
    o = _opts(eps=eps, lam=lam, seed=seed, call_id=call_id, **kw)
    rep = KrReport()
    st = lib().tucker_factor_update(h, N, I, R, _ptr(X), _ptr_array(As), _ptr(G), int(n), ctypes.byref(o),
                                    ctypes.byref(rep))
    if st != 0 and (raise_notconv or st != 6):
        _check(st, h)
    return rep.as_dict()


def tucker_als_sweep(X, As, G, lam, eps=0.1, sweeps=1, seed=0, call_id=0, **kw):
    """Sampled TuckerALS sweeps (Alg. 1 with Alg. 3 factor steps and Alg. 2 core steps).
    As and G are updated in place (device float32 tensors); returns the report."""
    h = context()
    N = len(As)
    X = _dev_f32(X)
    for k, A in enumerate(As):
        _inout(A, "As[%d]" % k)
    _inout(G, "G")
    I = (ctypes.c_int64 * N)(*[A.shape[0] for A in As])
    R = (ctypes.c_int32 * N)(*[A.shape[1] for A in As])
    o = _opts(eps=eps, lam=lam, seed=seed, call_id=call_id, **kw)
    rep = KrReport()
    st = lib().tucker_als_sweep(h, N, I, R, _ptr(X), _ptr_array(As), _ptr(G), ctypes.byref(o), int(sweeps),
                                ctypes.byref(rep))
    _check(st, h)
    return rep.as_dict()


def tucker_als_exact_sweep(X, As, G, lam, sweeps=1):
    """Exact TuckerALS sweeps (KronMatMul factor and core updates); As and G are updated in
    place (device float32 tensors). Returns the RRE after each sweep."""
    h = context()
    N = len(As)
    X = _dev_f32(X)
    for k, A in enumerate(As):
        _inout(A, "As[%d]" % k)
    _inout(G, "G")
    I = (ctypes.c_int64 * N)(*[A.shape[0] for A in As])
    R = (ctypes.c_int32 * N)(*[A.shape[1] for A in As])
    rre = (ctypes.c_double * max(1, int(sweeps)))()
    st = lib().tucker_als_exact_sweep(h, N, I, R, _ptr(X), _ptr_array(As), _ptr(G), float(lam), int(sweeps), rre)
    _check(st, h)
    return [rre[k] for k in range(int(sweeps))]


def tucker_rre(X, As, G):
    """||X - G x_1 A(1) ... x_N A(N)||^2 / ||X||^2 (FP64 sums on the device)."""
    h = context()
    N = len(As)
    X = _dev_f32(X)
    As = [_dev_f32(A) for A in As]
    G = _dev_f32(G)
    I = (ctypes.c_int64 * N)(*[A.shape[0] for A in As])
    R = (ctypes.c_int32 * N)(*[A.shape[1] for A in As])
    out = ctypes.c_double()
    _check(lib().tucker_rre(h, N, I, R, _ptr(X), _ptr_array(As), _ptr(G), ctypes.byref(out)), h)
    return out.value
