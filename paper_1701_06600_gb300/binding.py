"""Thin ctypes binding of libcprand (include/cprand.h): argument marshalling only.

Every function below has the name of the C entry point it calls.  Torch supplies device buffers
(inputs, outputs, workspace) and the current CUDA stream; all arithmetic runs in the library's
CUDA kernels.  There is no CPU path: if the library is missing, loading fails with an error.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcprand.so")

MAX_ORDER = 8
MAX_RANK = 64
F64, F32, BF16 = 0, 1, 2
OK, EINVAL, EWORKSPACE, ESINGULAR, ENONFINITE, ETIMEOUT, ECUDA = range(7)
METHOD_CPRAND, METHOD_CPRAND_MIX, METHOD_UPDATE, METHOD_FIT, METHOD_NORM, METHOD_CP_ALS, METHOD_MTTKRP = range(7)

_DTYPES = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}


class CprTensor(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("order", ctypes.c_int32),
                ("dims", ctypes.c_int64 * MAX_ORDER)]


class CprKtensor(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("rank", ctypes.c_int32), ("dims", ctypes.c_int64 * MAX_ORDER),
                ("lambda_", ctypes.c_void_p), ("factors", ctypes.c_void_p * MAX_ORDER)]


class CprOpts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int32), ("fixed_iters", ctypes.c_int32), ("fit_tol", ctypes.c_double),
                ("noise_eta", ctypes.c_double), ("stall_iters", ctypes.c_int32),
                ("init_from_out", ctypes.c_int32), ("fit_samples", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("batch_index", ctypes.c_uint32), ("first_iter", ctypes.c_uint32),
                ("fit_trace_dev", ctypes.c_void_p), ("loop_path", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("user_samples", ctypes.c_void_p), ("user_S", ctypes.c_int64), ("wait_budget", ctypes.c_int64)]

LOOP_AUTO, LOOP_CLUSTER, LOOP_GRAPH, LOOP_STREAM, LOOP_CLUSTER_DIST, LOOP_GRID = range(6)
MIX_AUTO, MIX_FFT, MIX_DENSE = range(3)
CONTRACT_AUTO, CONTRACT_TC, CONTRACT_FMA = range(3)


class CprResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("fit_est", ctypes.c_double),
                ("norm_x", ctypes.c_double), ("kernel_launches", ctypes.c_int64), ("ms_setup", ctypes.c_double),
                ("ms_iterate", ctypes.c_double), ("ms_finish", ctypes.c_double)]


class CprSchedule(ctypes.Structure):
    _fields_ = [("loop_path", ctypes.c_int32), ("split_per_sm", ctypes.c_int32), ("grid_min_split", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("ms_per_iter", ctypes.c_double)]


class CprError(RuntimeError):
    def __init__(self, status, where):
        super().__init__("%s failed: %s (status %d)" % (where, cpr_status_string(status), status))
        self.status = status


_lib = None

_SIGS = {
    "cpr_default_opts": (None, [ctypes.POINTER(CprOpts)]),
    "cpr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cpr_sample_size": (ctypes.c_int64, [ctypes.c_int]),
    "cpr_workspace_size": (ctypes.c_size_t, [ctypes.c_int, ctypes.POINTER(CprTensor), ctypes.c_int,
                                             ctypes.c_int64, ctypes.POINTER(CprOpts)]),
    "cpr_cp_als": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.c_int, ctypes.POINTER(CprOpts),
                                  ctypes.POINTER(CprKtensor), ctypes.POINTER(CprResult), ctypes.c_void_p,
                                  ctypes.c_size_t, ctypes.c_void_p]),
    "cpr_mttkrp": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.POINTER(CprKtensor), ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "cpr_cprand": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.c_int, ctypes.c_int64, ctypes.POINTER(CprOpts),
                                  ctypes.POINTER(CprKtensor), ctypes.POINTER(CprResult), ctypes.c_void_p,
                                  ctypes.c_size_t, ctypes.c_void_p]),
    "cpr_cprand_mix": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.c_int, ctypes.c_int64,
                                      ctypes.POINTER(CprOpts), ctypes.POINTER(CprKtensor),
                                      ctypes.POINTER(CprResult), ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.c_void_p]),
    "cpr_cprand_mix_fft": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.c_int, ctypes.c_int64,
                                      ctypes.POINTER(CprOpts), ctypes.POINTER(CprKtensor),
                                      ctypes.POINTER(CprResult), ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.c_void_p]),
    "cpr_cprand_mix_fft_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(CprTensor), ctypes.c_int, ctypes.c_int64,
                                                          ctypes.POINTER(CprOpts)]),
    "cpr_batched_workspace_size": (ctypes.c_size_t, [ctypes.c_int, ctypes.POINTER(CprTensor),
                                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                                                     ctypes.POINTER(CprOpts), ctypes.c_int]),
    "cpr_cprand_batched": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(CprTensor), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(CprOpts), ctypes.c_int,
                                          ctypes.POINTER(CprKtensor), ctypes.POINTER(CprResult),
                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "cpr_cprand_mix_batched": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(CprTensor), ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(CprOpts),
                                              ctypes.POINTER(CprKtensor), ctypes.POINTER(CprResult),
                                              ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "cpr_sample_indices": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                          ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "cpr_gather_fibers": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "cpr_sampled_update": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.POINTER(CprKtensor), ctypes.c_int,
                                          ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.POINTER(CprResult), ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p]),
    "cpr_fit_estimate": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.POINTER(CprKtensor), ctypes.c_int64,
                                        ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.c_void_p]),
    "cpr_mix_tensor": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "cpr_unmix_factors": (ctypes.c_int, [ctypes.POINTER(CprKtensor), ctypes.POINTER(CprKtensor), ctypes.c_uint64,
                                         ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "cpr_tensor_norm": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                                       ctypes.c_size_t, ctypes.c_void_p]),
    "cpr_fit_estimate_noalloc": (ctypes.c_int, [ctypes.POINTER(CprTensor), ctypes.POINTER(CprKtensor), ctypes.c_int64,
                                                ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                                ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "cpr_set_mix_engine": (ctypes.c_int, [ctypes.c_int]),
    "cpr_set_contract_engine": (ctypes.c_int, [ctypes.c_int]),
    "cpr_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(CprTensor), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(CprOpts), ctypes.c_int,
                                    ctypes.POINTER(CprKtensor), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                    ctypes.c_int, ctypes.POINTER(CprSchedule)]),
    "cpr_tune_lookup": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(CprTensor), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.POINTER(CprSchedule)]),
    "cpr_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "cpr_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "cpr_tune_clear": (None, []),
    "cpr_profile_begin": (ctypes.c_int, [ctypes.c_uint]),
    "cpr_profile_end": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
}

KERNEL_CLASSES = ["mix", "sample_skr", "contract", "chol", "solve", "normalize", "fit", "other", "loop"]


def lib():
    """Load libcprand.so (built in tree by build.py); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcprand.so not built (run __graft_entry__.build()); there is no CPU path")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def exported_symbols():
    return list(_SIGS)


# ------------------------------------------------------------------------------------------------
# marshalling helpers
# ------------------------------------------------------------------------------------------------

def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def tensor_desc(X, dims):
    """cpr_tensor for a flat, contiguous, column-major tensor X (torch, on the GPU)."""
    if X.dtype not in _DTYPES:
        raise TypeError("tensor dtype must be float64, float32 or bfloat16")
    if not X.is_contiguous():
        raise ValueError("tensor must be contiguous (column-major flat storage)")
    d = CprTensor()
    d.data = X.data_ptr() if X.numel() > 0 else None
    d.dtype = _DTYPES[X.dtype]
    d.order = len(dims)
    for n, v in enumerate(dims):
        d.dims[n] = int(v)
    return d


def ktensor_desc(lam, factors):
    k = CprKtensor()
    k.order = len(factors)
    k.rank = int(lam.numel())
    for n, A in enumerate(factors):
        assert A.dtype == torch.float64 and A.is_contiguous()
        k.dims[n] = A.shape[0]
        k.factors[n] = A.data_ptr()
    k.lambda_ = lam.data_ptr()
    return k


def alloc_ktensor(dims, R, device):
    lam = torch.empty(R, dtype=torch.float64, device=device)
    factors = [torch.empty((int(I), R), dtype=torch.float64, device=device) for I in dims]
    return lam, factors


def workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _check(st, where):
    if st != OK:
        raise CprError(st, where)


# ------------------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ------------------------------------------------------------------------------------------------

def cpr_default_opts(**kw):
    o = CprOpts()
    lib().cpr_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def cpr_status_string(st):
    return lib().cpr_status_string(int(st)).decode()


def cpr_sample_size(R):
    return int(lib().cpr_sample_size(int(R)))


def cpr_workspace_size(method, X, dims, R, S, opts=None):
    d = tensor_desc(X, dims)
    o = opts if opts is not None else cpr_default_opts()
    return int(lib().cpr_workspace_size(method, ctypes.byref(d), int(R), int(S), ctypes.byref(o)))


def _run_whole(fn_name, method, X, dims, R, S, opts, init, ws, stream):
    d = tensor_desc(X, dims)
    o = opts if opts is not None else cpr_default_opts()
    lam, factors = alloc_ktensor(dims, R, X.device)
    if init is not None:
        for n in range(1, len(dims)):
            factors[n].copy_(init[n])
        o.init_from_out = 1
    k = ktensor_desc(lam, factors)
    need = lib().cpr_workspace_size(method, ctypes.byref(d), int(R), int(S), ctypes.byref(o))
    if need == 0:
        raise CprError(EINVAL, fn_name)
    if ws is None or ws.numel() < need:
        ws = workspace(need, X.device)
    res = CprResult()
    st = getattr(lib(), fn_name)(ctypes.byref(d), int(R), int(S), ctypes.byref(o), ctypes.byref(k),
                                 ctypes.byref(res), ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()),
                                 _stream(stream))
    _check(st, fn_name)
    return {"lam": lam, "factors": factors, "ws": ws, **result_dict(res)}


def result_dict(res):
    return {"iters": res.iters, "status": res.status, "fit_est": res.fit_est, "norm_x": res.norm_x,
            "kernel_launches": res.kernel_launches, "ms_setup": res.ms_setup, "ms_iterate": res.ms_iterate,
            "ms_finish": res.ms_finish}


class PreparedRun:
    """A whole-algorithm call with every buffer (workspace, outputs, descriptors) allocated once, so
    repeated calls do no host-side allocation: used by the benchmark's timed loop."""

    def __init__(self, X, dims, R, S, opts=None, mix=True):
        self.fn = lib().cpr_cprand_mix if mix else lib().cpr_cprand
        self.desc = tensor_desc(X, dims)
        self.opts = opts if opts is not None else cpr_default_opts()
        self.R, self.S = int(R), int(S)
        self.lam, self.factors = alloc_ktensor(dims, R, X.device)
        self.k = ktensor_desc(self.lam, self.factors)
        method = METHOD_CPRAND_MIX if mix else METHOD_CPRAND
        need = lib().cpr_workspace_size(method, ctypes.byref(self.desc), self.R, self.S, ctypes.byref(self.opts))
        if need == 0:
            raise CprError(EINVAL, "cpr_workspace_size")
        self.ws = workspace(need, X.device)
        self.res = CprResult()

    def set_input(self, X):
        self.desc.data = X.data_ptr()

    def __call__(self, stream=None):
        st = self.fn(ctypes.byref(self.desc), self.R, self.S, ctypes.byref(self.opts), ctypes.byref(self.k),
                     ctypes.byref(self.res), ctypes.c_void_p(self.ws.data_ptr()), ctypes.c_size_t(self.ws.numel()),
                     _stream(stream))
        _check(st, "cpr_cprand_mix")
        return result_dict(self.res)


def cpr_set_mix_engine(engine):
    """Select the mixing engine process-wide (MIX_AUTO, MIX_FFT, MIX_DENSE); returns the previous one."""
    prev = lib().cpr_set_mix_engine(int(engine))
    if prev < 0:
        raise ValueError("unknown mixing engine %r" % (engine,))
    return prev


def cpr_set_contract_engine(engine):
    """Select the contraction engine of the whole-GPU loop (CONTRACT_AUTO, CONTRACT_TC, CONTRACT_FMA);
    returns the previous one."""
    prev = lib().cpr_set_contract_engine(int(engine))
    if prev < 0:
        raise ValueError("unknown contraction engine %r" % (engine,))
    return prev


def cpr_profile_begin(mask=0xFF):
    _check(lib().cpr_profile_begin(int(mask)), "cpr_profile_begin")


def cpr_profile_end():
    ms = (ctypes.c_double * len(KERNEL_CLASSES))()
    cnt = (ctypes.c_int64 * len(KERNEL_CLASSES))()
    _check(lib().cpr_profile_end(ms, cnt), "cpr_profile_end")
    return {c: (ms[i], cnt[i]) for i, c in enumerate(KERNEL_CLASSES)}


def cpr_cp_als(X, dims, R, opts=None, init=None, ws=None, stream=None):
    """CP-ALS (Alg. 1) with the exact fit.  init: optional list of initial factors (modes 2..N used)."""
    d = tensor_desc(X, dims)
    o = opts if opts is not None else cpr_default_opts()
    lam, factors = alloc_ktensor(dims, R, X.device)
    if init is not None:
        for n in range(1, len(dims)):
            factors[n].copy_(init[n])
        o.init_from_out = 1
    k = ktensor_desc(lam, factors)
    need = lib().cpr_workspace_size(METHOD_CP_ALS, ctypes.byref(d), int(R), 0, ctypes.byref(o))
    if need == 0:
        raise CprError(EINVAL, "cpr_cp_als")
    if ws is None or ws.numel() < need:
        ws = workspace(need, X.device)
    res = CprResult()
    st = lib().cpr_cp_als(ctypes.byref(d), int(R), ctypes.byref(o), ctypes.byref(k), ctypes.byref(res),
                          ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(st, "cpr_cp_als")
    return {"lam": lam, "factors": factors, "ws": ws, **result_dict(res)}


def cpr_mttkrp(X, dims, factors, mode, stream=None):
    """M = X_(mode) Z^(mode) (exact MTTKRP) over the given FP64 factors; returns I_mode x R FP64."""
    R = int(factors[0].shape[1])
    lam = torch.ones(R, dtype=torch.float64, device=X.device)
    d = tensor_desc(X, dims)
    fs = [f.contiguous() for f in factors]
    k = ktensor_desc(lam, fs)
    o = cpr_default_opts()
    need = lib().cpr_workspace_size(METHOD_MTTKRP, ctypes.byref(d), R, 0, ctypes.byref(o))
    if need == 0:
        raise CprError(EINVAL, "cpr_workspace_size")
    ws = workspace(need, X.device)
    M = torch.empty((int(dims[mode]), R), dtype=torch.float64, device=X.device)
    st = lib().cpr_mttkrp(ctypes.byref(d), ctypes.byref(k), int(mode), ctypes.c_void_p(M.data_ptr()),
                          ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(st, "cpr_mttkrp")
    return M


def cpr_cprand(X, dims, R, S, opts=None, init=None, ws=None, stream=None):
    """CPRAND (Alg. 3) on the flat column-major tensor X; returns lam, factors (FP64) and the run
    summary.  init: optional initial factors (list; entries 1..N-1 used)."""
    return _run_whole("cpr_cprand", METHOD_CPRAND, X, dims, R, S, opts, init, ws, stream)


def cpr_cprand_mix(X, dims, R, S, opts=None, init=None, ws=None, stream=None):
    """CPRAND-MIX, real-transform form (Alg. 5); factors are returned unmixed."""
    return _run_whole("cpr_cprand_mix", METHOD_CPRAND_MIX, X, dims, R, S, opts, init, ws, stream)


def cpr_cprand_mix_fft(X, dims, R, S, opts=None, ws=None, stream=None):
    """CPRAND-MIX, complex-transform form (Alg. 4): unitary-DFT mixing, real factors."""
    d = tensor_desc(X, dims)
    o = opts if opts is not None else cpr_default_opts()
    lam, factors = alloc_ktensor(dims, R, X.device)
    k = ktensor_desc(lam, factors)
    need = lib().cpr_cprand_mix_fft_workspace_size(ctypes.byref(d), int(R), int(S), ctypes.byref(o))
    if need == 0:
        raise CprError(EINVAL, "cpr_cprand_mix_fft_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, X.device)
    res = CprResult()
    st = lib().cpr_cprand_mix_fft(ctypes.byref(d), int(R), int(S), ctypes.byref(o), ctypes.byref(k), ctypes.byref(res),
                                  ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(st, "cpr_cprand_mix_fft")
    return {"lam": lam, "factors": factors, "ws": ws, **result_dict(res)}


def cpr_cprand_batched(Xs, dims_list, Rs, Ss, opts_list=None, mix=False, ws=None, stream=None):
    """Many independent decompositions advancing together (one set of launches per step)."""
    B = len(Xs)
    descs = (CprTensor * B)(*[tensor_desc(X, d) for X, d in zip(Xs, dims_list)])
    Rarr = (ctypes.c_int * B)(*[int(r) for r in Rs])
    Sarr = (ctypes.c_int64 * B)(*[int(s) for s in Ss])
    if opts_list is None:
        opts_list = [cpr_default_opts(batch_index=b) for b in range(B)]
    oarr = (CprOpts * B)(*opts_list)
    outs = [alloc_ktensor(d, r, Xs[0].device) for d, r in zip(dims_list, Rs)]
    karr = (CprKtensor * B)(*[ktensor_desc(l, f) for l, f in outs])
    need = lib().cpr_batched_workspace_size(B, descs, Rarr, Sarr, oarr, int(bool(mix)))
    if need == 0:
        raise CprError(EINVAL, "cpr_batched_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, Xs[0].device)
    rarr = (CprResult * B)()
    st = lib().cpr_cprand_batched(B, descs, Rarr, Sarr, oarr, int(bool(mix)), karr, rarr,
                                  ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(st, "cpr_cprand_batched")
    return [{"lam": l, "factors": f, **result_dict(r)} for (l, f), r in zip(outs, rarr)], ws


def cpr_sample_indices(dims, mode, S, seed, b=0, t=0, device="cuda", stream=None):
    N = len(dims)
    d = CprTensor()
    d.order = N
    d.dtype = F32
    for n, v in enumerate(dims):
        d.dims[n] = int(v)
    idx = torch.empty((max(S, 1), N), dtype=torch.int32, device=device)
    off = torch.empty(max(S, 1), dtype=torch.int64, device=device)
    st = lib().cpr_sample_indices(ctypes.byref(d), int(mode), int(S), ctypes.c_uint64(seed), int(b), int(t),
                                  ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(off.data_ptr()),
                                  _stream(stream))
    _check(st, "cpr_sample_indices")
    return idx[:S], off[:S]


def cpr_gather_fibers(X, dims, mode, off, out=None, stream=None):
    """X_S (I_n x S view; column j = fiber j).  `out`: an optional caller buffer of S * I_n elements
    of X's dtype that receives the fibers (reused across calls)."""
    d = tensor_desc(X, dims)
    S = off.numel()
    if out is None:
        out = torch.empty((S, int(dims[mode])), dtype=X.dtype, device=X.device)
    elif out.numel() != S * int(dims[mode]) or out.dtype != X.dtype or not out.is_contiguous():
        raise ValueError("out must be a contiguous buffer of S * I_n elements of X's dtype")
    st = lib().cpr_gather_fibers(ctypes.byref(d), int(mode), int(S), ctypes.c_void_p(off.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), _stream(stream))
    _check(st, "cpr_gather_fibers")
    return out.view(S, int(dims[mode])).T   # I_n x S view


def cpr_sampled_update(X, dims, lam, factors, mode, S, seed, b=0, t=0, ws=None, stream=None):
    """One mode update of Alg. 3, in place on (lam, factors[mode]).  Returns the device status."""
    d = tensor_desc(X, dims)
    k = ktensor_desc(lam, factors)
    o = cpr_default_opts()
    need = lib().cpr_workspace_size(METHOD_UPDATE, ctypes.byref(d), int(lam.numel()), int(S), ctypes.byref(o))
    if need == 0:
        raise CprError(EINVAL, "cpr_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, X.device)
    res = CprResult()
    st = lib().cpr_sampled_update(ctypes.byref(d), ctypes.byref(k), int(mode), int(S), ctypes.c_uint64(seed),
                                  int(b), int(t), ctypes.byref(res), ctypes.c_void_p(ws.data_ptr()),
                                  ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(st, "cpr_sampled_update")
    return res.status


def cpr_fit_estimate(X, dims, lam, factors, P_hat, seed, b=0, norm_x=-1.0, stream=None):
    d = tensor_desc(X, dims)
    k = ktensor_desc(lam, factors)
    o = cpr_default_opts(fit_samples=int(P_hat))
    need = lib().cpr_workspace_size(METHOD_FIT, ctypes.byref(d), int(lam.numel()), 0, ctypes.byref(o))
    if need == 0:
        raise CprError(EINVAL, "cpr_workspace_size")
    ws = workspace(need, X.device)
    fit = ctypes.c_double()
    st = lib().cpr_fit_estimate(ctypes.byref(d), ctypes.byref(k), int(P_hat), ctypes.c_uint64(seed), int(b),
                                float(norm_x), ctypes.byref(fit), ctypes.c_void_p(ws.data_ptr()),
                                ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(st, "cpr_fit_estimate")
    return fit.value


def cpr_fit_estimate_noalloc(X, dims, lam, factors, P_hat, seed, b=0, norm_x=-1.0, stream=None):
    """The sampled fit without a workspace: the library's fixed device scratch array is used instead, so
    nothing is allocated for this call (see include/cprand.h for the sharing rules)."""
    d = tensor_desc(X, dims)
    k = ktensor_desc(lam, factors)
    fit = ctypes.c_double()
    st = lib().cpr_fit_estimate_noalloc(ctypes.byref(d), ctypes.byref(k), int(P_hat), ctypes.c_uint64(seed), int(b),
                                        float(norm_x), ctypes.byref(fit), _stream(stream))
    _check(st, "cpr_fit_estimate_noalloc")
    return fit.value


def cpr_mix_tensor(X, dims, seed, b=0, stream=None):
    d = tensor_desc(X, dims)
    o = cpr_default_opts()
    need = lib().cpr_workspace_size(METHOD_CPRAND_MIX, ctypes.byref(d), 1, 1, ctypes.byref(o))
    ws = workspace(need, X.device)
    out = torch.empty_like(X)
    st = lib().cpr_mix_tensor(ctypes.byref(d), ctypes.c_void_p(out.data_ptr()), ctypes.c_uint64(seed), int(b),
                              ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(st, "cpr_mix_tensor")
    return out


def cpr_unmix_factors(lam, factors_hat, seed, b=0, stream=None):
    dims = [A.shape[0] for A in factors_hat]
    R = lam.numel()
    out_lam, out_f = alloc_ktensor(dims, R, lam.device)
    kh = ktensor_desc(lam, factors_hat)
    ko = ktensor_desc(out_lam, out_f)
    need = sum(((8 * I * I + 255) // 256) * 256 + ((8 * I + 255) // 256) * 256 + ((32 * I + 255) // 256) * 256
               for I in dims) + 256
    ws = workspace(need, lam.device)
    st = lib().cpr_unmix_factors(ctypes.byref(kh), ctypes.byref(ko), ctypes.c_uint64(seed), int(b),
                                 ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(st, "cpr_unmix_factors")
    return out_lam, out_f


def cpr_tensor_norm(X, dims, stream=None):
    d = tensor_desc(X, dims)
    need = lib().cpr_workspace_size(METHOD_NORM, ctypes.byref(d), 1, 1, None)
    ws = workspace(need, X.device)
    out = ctypes.c_double()
    st = lib().cpr_tensor_norm(ctypes.byref(d), ctypes.byref(out), ctypes.c_void_p(ws.data_ptr()),
                               ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(st, "cpr_tensor_norm")
    return out.value


def _schedule_dict(sc):
    return {"loop_path": sc.loop_path, "split_per_sm": sc.split_per_sm, "grid_min_split": sc.grid_min_split,
            "ms_per_iter": sc.ms_per_iter}


def _batch_descs(Xs, dims_list, Rs, Ss):
    B = len(Xs)
    descs = (CprTensor * B)(*[tensor_desc(X, d) for X, d in zip(Xs, dims_list)])
    Rarr = (ctypes.c_int * B)(*[int(r) for r in Rs])
    Sarr = (ctypes.c_int64 * B)(*[int(s) for s in Ss])
    return B, descs, Rarr, Sarr


def cpr_autotune(Xs, dims_list, Rs, Ss, opts_list=None, mix=False, trial_iters=3, ws=None, stream=None):
    """Time the candidate schedules on this batch and record the fastest for its bucket; returns the
    chosen schedule (dict) and the workspace."""
    B, descs, Rarr, Sarr = _batch_descs(Xs, dims_list, Rs, Ss)
    if opts_list is None:
        opts_list = [cpr_default_opts(batch_index=b) for b in range(B)]
    oarr = (CprOpts * B)(*opts_list)
    outs = [alloc_ktensor(d, r, Xs[0].device) for d, r in zip(dims_list, Rs)]
    karr = (CprKtensor * B)(*[ktensor_desc(l, f) for l, f in outs])
    need = lib().cpr_batched_workspace_size(B, descs, Rarr, Sarr, oarr, int(bool(mix)))
    if need == 0:
        raise CprError(EINVAL, "cpr_batched_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, Xs[0].device)
    sc = CprSchedule()
    st = lib().cpr_autotune(B, descs, Rarr, Sarr, oarr, int(bool(mix)), karr, ctypes.c_void_p(ws.data_ptr()),
                            ctypes.c_size_t(ws.numel()), _stream(stream), int(trial_iters), ctypes.byref(sc))
    _check(st, "cpr_autotune")
    return _schedule_dict(sc), ws


def cpr_tune_lookup(dims_list, Rs, Ss, dtype=F32, mix=False):
    """The recorded schedule of a batch's bucket (dict), or None.  Host-side only."""
    B = len(dims_list)
    descs = (CprTensor * B)()
    for b, dims in enumerate(dims_list):
        descs[b].order = len(dims)
        descs[b].dtype = dtype
        for n, v in enumerate(dims):
            descs[b].dims[n] = int(v)
    Rarr = (ctypes.c_int * B)(*[int(r) for r in Rs])
    Sarr = (ctypes.c_int64 * B)(*[int(s) for s in Ss])
    sc = CprSchedule()
    st = lib().cpr_tune_lookup(B, descs, Rarr, Sarr, int(bool(mix)), ctypes.byref(sc))
    return _schedule_dict(sc) if st == OK else None


def cpr_tune_save(path):
    _check(lib().cpr_tune_save(str(path).encode()), "cpr_tune_save")


def cpr_tune_load(path):
    _check(lib().cpr_tune_load(str(path).encode()), "cpr_tune_load")


def cpr_tune_clear():
    lib().cpr_tune_clear()
