"""Python binding of the gbsmps C ABI (``include/gbsmps.h``).

Argument marshalling only: every step of the Gaussian-state -> MPS path runs
in the CUDA kernels of ``libgbsmps.so``.  Buffers may be numpy arrays (host
memory) or torch tensors (host or CUDA); PyTorch is used for device memory
and streams.  There is no CPU fallback: if the library is missing the first
call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbsmps.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gbsmps.h")

OK, ERR_ARG, ERR_NOT_SYMMETRIC, ERR_NOT_PURE, ERR_OOM = 0, 1, 2, 3, 4
ERR_NOT_CONVERGED, ERR_BOUNDS, ERR_CUDA, ERR_NUMERIC, ERR_STATE, ERR_TIMEOUT = 5, 6, 7, 8, 9, 10
MEM_HOST, MEM_DEVICE = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
NE_MAX = 24
QS = 2 * NE_MAX + 1


class ServerOpts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("hbm_budget", C.c_size_t),
                ("simulate_s_per_tensor", C.c_double), ("batch_max", C.c_int32)]


class JobInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("slot", C.c_int32),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("hbm_bytes", C.c_size_t), ("detail", C.c_char * 128), ("batch", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("running", C.c_int64), ("queued", C.c_int64), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("busy_s", C.c_double),
                ("tensors", C.c_double), ("samples", C.c_double), ("hbm_in_use", C.c_size_t),
                ("hbm_budget", C.c_size_t), ("hbm_peak", C.c_size_t)]


class GbsmpsError(RuntimeError):
    def __init__(self, code, detail):
        super().__init__(f"gbsmps error {code}: {detail}")
        self.code = code


class Opts(C.Structure):
    _fields_ = [("d", C.c_int32), ("chi_max", C.c_int32), ("eps_trunc", C.c_double),
                ("lambda2_freeze", C.c_double), ("precision", C.c_int32),
                ("validate", C.c_int32), ("purity_tol", C.c_double)]


class Request(C.Structure):
    _fields_ = [("gamma", C.c_void_p), ("N", C.c_int32), ("opts", Opts), ("samples", C.c_int64),
                ("seed", C.c_uint64), ("counter0", C.c_uint64), ("out", C.c_void_p),
                ("flags", C.c_void_p)]


_lib = None


def lib():
    """Load libgbsmps.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2512_10643_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    sig = {
        "gbsmps_opts_default": (C.c_int, [C.POINTER(Opts)]),
        "gbsmps_create": (C.c_int, [C.c_int, vp, C.POINTER(vp)]),
        "gbsmps_destroy": (C.c_int, [vp]),
        "gbsmps_build_from_cov": (C.c_int, [vp, i32, vp, C.c_int, C.POINTER(Opts), C.POINTER(vp)]),
        "gbsmps_build_from_Q": (C.c_int, [vp, i32, vp, C.c_int, C.POINTER(Opts), C.POINTER(vp)]),
        "gbsmps_info": (C.c_int, [vp, vp, vp, vp, vp, vp]),
        "gbsmps_get_tensor": (C.c_int, [vp, i32, vp, C.c_size_t, C.c_int]),
        "gbsmps_get_gsvd": (C.c_int, [vp, vp, vp, vp]),
        "gbsmps_get_basis": (C.c_int, [vp, i32, vp, vp]),
        "gbsmps_amplitudes": (C.c_int, [vp, i64, vp, vp, C.c_int]),
        "gbsmps_sample": (C.c_int, [vp, i64, u64, u64, vp, vp, vp, C.c_int]),
        "gbsmps_release": (C.c_int, [vp]),
        "gbsmps_offload": (C.c_int, [vp, vp]),
        "gbsmps_filter": (C.c_int, [vp, i32, i32, vp, dbl, dbl, i32, vp, vp, vp, C.c_int]),
        "gbsmps_build_site": (C.c_int, [vp, i32, i32, i32, vp, dbl, i32, vp, i32, vp, i32, vp, C.c_int]),
        "gbsmps_strerror": (C.c_char_p, [C.c_int]),
        "gbsmps_last_error_detail": (C.c_char_p, []),
        "gbsmps_launch_count": (i64, [vp]),
        "gbsmps_build_site_noalloc": (C.c_int, [vp, i32, i32, i32, vp, dbl, i32, vp, i32, vp, i32, vp]),
        "gbsmps_trace": (C.c_int, [vp, C.c_int]),
        "gbsmps_trace_read": (C.c_int, [vp, vp, vp, vp, vp]),
        "gbsmps_trace_read_kernel": (C.c_int, [vp, C.c_int32, vp, vp, vp, vp]),
        "gbsmps_server_opts_default": (C.c_int, [C.POINTER(ServerOpts)]),
        "gbsmps_server_create": (C.c_int, [C.c_int, C.POINTER(ServerOpts), C.POINTER(vp)]),
        "gbsmps_server_submit": (C.c_int, [vp, C.POINTER(Request), C.POINTER(i64)]),
        "gbsmps_server_wait": (C.c_int, [vp, i64, dbl, C.POINTER(JobInfo)]),
        "gbsmps_server_drain": (C.c_int, [vp, dbl]),
        "gbsmps_server_stats_read": (C.c_int, [vp, C.POINTER(ServerStats)]),
        "gbsmps_server_destroy": (C.c_int, [vp]),
        "gbsmps_estimate_bytes": (C.c_size_t, [i32, C.POINTER(Opts), i64]),
        "gbsmps_build_batch": (C.c_int, [vp, i32, vp, vp, C.c_int, vp, vp]),
        "gbsmps_build_sample_stream": (C.c_int, [vp, i32, vp, vp, vp, i64, vp, vp, vp, C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_symbols():
    """Entry points declared in include/gbsmps.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\*\s]+?\b(gbsmps_\w+)\s*\(", txt, re.M)))


def _check(rc):
    if rc != OK:
        L = lib()
        raise GbsmpsError(rc, f"{L.gbsmps_strerror(rc).decode()} ({L.gbsmps_last_error_detail().decode()})")


def _ptr(x):
    """(pointer, mem_kind) of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None, MEM_HOST
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, MEM_HOST
    import torch
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (MEM_DEVICE if x.is_cuda else MEM_HOST)
    raise TypeError(type(x))


def opts_default(**kw) -> Opts:
    o = Opts()
    _check(lib().gbsmps_opts_default(C.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def gbsmps_create(device: int = 0, stream=None):
    h = C.c_void_p()
    _check(lib().gbsmps_create(device, C.c_void_p(stream or 0), C.byref(h)))
    return h


def gbsmps_destroy(ctx):
    _check(lib().gbsmps_destroy(ctx))


def gbsmps_build_from_cov(ctx, gamma, opts: Opts):
    p, kind = _ptr(gamma)
    N = gamma.shape[0] // 2
    h = C.c_void_p()
    _check(lib().gbsmps_build_from_cov(ctx, N, C.c_void_p(p), kind, C.byref(opts), C.byref(h)))
    return h


def gbsmps_build_batch(ctx, gammas, opts_list):
    """Build many states at once: gammas is a list of (2N, 2N) float64 numpy
    arrays (host) or CUDA tensors (device), opts_list one Opts per state.
    Returns the list of handles."""
    n = len(gammas)
    if n != len(opts_list):
        raise ValueError("one Opts per state")
    if n == 0:
        return []
    ptrs = [_ptr(x) for x in gammas]
    kinds = {k for _, k in ptrs}
    if len(kinds) != 1:
        raise ValueError("all covariances must live in the same memory")
    Ns = (C.c_int32 * n)(*[x.shape[0] // 2 for x in gammas])
    gp = (C.c_void_p * n)(*[p for p, _ in ptrs])
    op = (Opts * n)(*opts_list)
    hs = (C.c_void_p * n)()
    _check(lib().gbsmps_build_batch(ctx, n, Ns, gp, kinds.pop(), op, hs))
    return [C.c_void_p(h) for h in hs]


def gbsmps_build_sample_stream(ctx, gammas, opts_list, S: int, seeds, counter0s, outs):
    """Build and sample a stream of states (the next state's Gaussian-SVD
    chain runs beside the current state's sampling).  gammas: (2N, 2N)
    float64 arrays or tensors, outs: (S, N) uint8 arrays or tensors, all in
    the same memory; seeds / counter0s: one Philox key and first counter per
    state.  Patterns equal those of separate build + sample calls."""
    n = len(gammas)
    if not (n == len(opts_list) == len(seeds) == len(counter0s) == len(outs)):
        raise ValueError("one Opts, seed, counter0 and output per state")
    if n == 0:
        return
    ptrs = [_ptr(x) for x in gammas] + [_ptr(x) for x in outs]
    kinds = {k for _, k in ptrs}
    if len(kinds) != 1:
        raise ValueError("all covariances and outputs must live in the same memory")
    for x, o in zip(gammas, outs):
        if tuple(o.shape) != (S, x.shape[0] // 2):
            raise ValueError("outs[k] must have shape (S, N_k)")
    Ns = (C.c_int32 * n)(*[x.shape[0] // 2 for x in gammas])
    gp = (C.c_void_p * n)(*[p for p, _ in ptrs[:n]])
    op = (Opts * n)(*opts_list)
    sd = (C.c_uint64 * n)(*[int(v) for v in seeds])
    c0 = (C.c_uint64 * n)(*[int(v) for v in counter0s])
    outp = (C.c_void_p * n)(*[p for p, _ in ptrs[n:]])
    _check(lib().gbsmps_build_sample_stream(ctx, n, Ns, gp, op, int(S), sd, c0, outp, kinds.pop()))


def gbsmps_build_from_Q(ctx, Q, opts: Opts):
    """Q: complex128 (N, N) numpy array, or float64 (N, N, 2) tensor."""
    if isinstance(Q, np.ndarray) and np.iscomplexobj(Q):
        Q = np.ascontiguousarray(Q.astype(np.complex128)).view(np.float64).reshape(Q.shape + (2,))
    p, kind = _ptr(Q)
    h = C.c_void_p()
    _check(lib().gbsmps_build_from_Q(ctx, Q.shape[0], C.c_void_p(p), kind, C.byref(opts), C.byref(h)))
    return h


def gbsmps_info(mps):
    N, d = C.c_int32(), C.c_int32()
    _check(lib().gbsmps_info(mps, C.byref(N), C.byref(d), None, None, None))
    dims = np.zeros(N.value + 1, dtype=np.int32)
    ne = np.zeros(max(N.value - 1, 1), dtype=np.int32)
    eps = np.zeros(max(N.value - 1, 1), dtype=np.float64)
    _check(lib().gbsmps_info(mps, None, None, dims.ctypes.data, ne.ctypes.data, eps.ctypes.data))
    return {"N": N.value, "d": d.value, "bond_dims": dims, "n_e": ne[:max(N.value - 1, 0)],
            "eps": eps[:max(N.value - 1, 0)]}


def gbsmps_get_tensor(mps, site: int, dst=None):
    info = gbsmps_info(mps)
    Dl, Dr, d = int(info["bond_dims"][site]), int(info["bond_dims"][site + 1]), info["d"]
    if dst is None:
        dst = np.zeros((Dl, d, Dr), dtype=np.complex128)
    p, kind = _ptr(dst)
    nbytes = dst.nbytes if isinstance(dst, np.ndarray) else dst.numel() * dst.element_size()
    _check(lib().gbsmps_get_tensor(mps, site, C.c_void_p(p), nbytes, kind))
    return dst


def gbsmps_get_gsvd(mps):
    N = gbsmps_info(mps)["N"]
    lam2 = np.zeros(max(N - 1, 1) * NE_MAX)
    Qm = np.zeros(N * QS * QS, dtype=np.complex128)
    cm = np.zeros(N)
    _check(lib().gbsmps_get_gsvd(mps, lam2.ctypes.data, Qm.ctypes.data, cm.ctypes.data))
    return lam2[:(N - 1) * NE_MAX].reshape(max(N - 1, 0), NE_MAX), Qm.reshape(N, QS, QS), cm


def gbsmps_get_basis(mps, bond: int):
    """(occ uint8 (D_b, n_e_b), E float64 (D_b,)) of the kept basis of bond b."""
    info = gbsmps_info(mps)
    D = int(info["bond_dims"][bond])
    ne = 0 if bond in (0, info["N"]) else int(info["n_e"][bond - 1])
    occ = np.zeros((D, ne), dtype=np.uint8)
    E = np.zeros(D, dtype=np.float64)
    _check(lib().gbsmps_get_basis(mps, int(bond), occ.ctypes.data if ne else None, E.ctypes.data))
    return occ, E


def gbsmps_amplitudes(mps, patterns, out=None):
    P = patterns.shape[0]
    if out is None:
        out = np.zeros(P, dtype=np.complex128) if isinstance(patterns, np.ndarray) else None
    pp, kind = _ptr(patterns)
    op, okind = _ptr(out)
    if okind != kind:
        raise ValueError("patterns and out must live in the same memory")
    _check(lib().gbsmps_amplitudes(mps, P, C.c_void_p(pp), C.c_void_p(op), kind))
    return out


def gbsmps_sample(mps, S: int, seed: int = 0, counter0: int = 0, uniforms=None, out=None,
                  flags=None):
    N = gbsmps_info(mps)["N"]
    if out is None:
        out = np.zeros((S, N), dtype=np.uint8)
    op, kind = _ptr(out)
    up, ukind = _ptr(uniforms)
    fp, fkind = _ptr(flags)
    if uniforms is not None and ukind != kind:
        raise ValueError("uniforms and out must live in the same memory")
    if flags is not None and fkind != kind:
        raise ValueError("flags and out must live in the same memory")
    _check(lib().gbsmps_sample(mps, S, seed, counter0, C.c_void_p(up or 0), C.c_void_p(op),
                               C.c_void_p(fp or 0), kind))
    return out


def gbsmps_release(mps):
    _check(lib().gbsmps_release(mps))


def gbsmps_offload(mps) -> int:
    """Move a mixed-precision MPS's sampler planes to pinned host memory;
    later samplings stream them through a three-site device ring.  Returns
    the bytes each sampling streams."""
    n = C.c_size_t()
    _check(lib().gbsmps_offload(mps, C.byref(n)))
    return n.value


def gbsmps_build_site(ctx, Qm, c, occ_l, occ_r, d, precision=PREC_FP64):
    """Expert entry on host numpy arrays: Qm complex (n, n), occ_l (Dl, nl)
    and occ_r (Dr, nr) uint8 down-closed bases starting at the vacuum."""
    Qm = np.ascontiguousarray(Qm, dtype=np.complex128)
    occ_l = np.ascontiguousarray(occ_l, dtype=np.uint8)
    occ_r = np.ascontiguousarray(occ_r, dtype=np.uint8)
    nl, nr = occ_l.shape[1], occ_r.shape[1]
    Dl, Dr = occ_l.shape[0], occ_r.shape[0]
    out = np.zeros((Dl, d, Dr), dtype=np.complex128)
    _check(lib().gbsmps_build_site(ctx, nl, nr, d, Qm.ctypes.data, float(c), Dl,
                                   occ_l.ctypes.data if nl else None, Dr,
                                   occ_r.ctypes.data if nr else None, precision,
                                   out.ctypes.data, MEM_HOST))
    return out


def gbsmps_build_site_noalloc(ctx, Qm, c, occ_l, occ_r, d, out, precision=PREC_FP64):
    """Allocation-free single-site build.  Qm (complex (n, n) as float64
    (n, n, 2)), occ_l (Dl, nl) and occ_r (Dr, nr) uint8, and out (Dl, d, Dr, 2)
    float64 are contiguous CUDA tensors; the library allocates nothing."""
    nl, nr = occ_l.shape[1], occ_r.shape[1]
    Dl, Dr = occ_l.shape[0], occ_r.shape[0]
    ptrs = [_ptr(x) for x in (Qm, occ_l, occ_r, out)]
    if any(k != MEM_DEVICE for _, k in ptrs):
        raise ValueError("all buffers must be device tensors")
    _check(lib().gbsmps_build_site_noalloc(ctx, nl, nr, d, C.c_void_p(ptrs[0][0]), float(c), Dl,
                                           C.c_void_p(ptrs[1][0] if nl else 0), Dr,
                                           C.c_void_p(ptrs[2][0] if nr else 0), precision,
                                           C.c_void_p(ptrs[3][0])))
    return out


def gbsmps_filter(ctx, gammas, alpha: float, eps: float = 0.0, max_iter: int = 100000, out=None):
    """Mixed -> pure decomposition of a batch of covariances of equal N:
    gammas (count, 2N, 2N) float64 numpy array or CUDA tensor.  Returns
    (S (count, 2N, 2N), iters (count,), loss (count,)); Gamma_p = S S^T / 2."""
    count, n = int(gammas.shape[0]), int(gammas.shape[1])
    if isinstance(gammas, np.ndarray):
        gammas = np.ascontiguousarray(gammas, dtype=np.float64)
    if out is None:
        if isinstance(gammas, np.ndarray):
            out = np.zeros((count, n, n), dtype=np.float64)
        else:
            import torch
            out = torch.zeros((count, n, n), dtype=torch.float64, device=gammas.device)
    gp, kind = _ptr(gammas)
    op, okind = _ptr(out)
    if kind != okind:
        raise ValueError("gammas and out must live in the same memory")
    iters = np.zeros(count, dtype=np.int32)
    loss = np.zeros(count, dtype=np.float64)
    _check(lib().gbsmps_filter(ctx, count, n // 2, C.c_void_p(gp), float(alpha), float(eps),
                               int(max_iter), C.c_void_p(op), iters.ctypes.data, loss.ctypes.data,
                               kind))
    return out, iters, loss


def gbsmps_launch_count(ctx=None) -> int:
    return int(lib().gbsmps_launch_count(ctx))


def gbsmps_trace(ctx, enable: bool):
    _check(lib().gbsmps_trace(ctx, int(bool(enable))))


def gbsmps_trace_read(ctx):
    ms, fl, by = C.c_double(), C.c_double(), C.c_double()
    n = C.c_int64()
    _check(lib().gbsmps_trace_read(ctx, C.byref(ms), C.byref(n), C.byref(fl), C.byref(by)))
    return {"ms": ms.value, "launches": n.value, "flops": fl.value, "bytes": by.value}


def gbsmps_trace_read_kernel(ctx, which: int):
    """which = 0: the sampler GEMM (as gbsmps_trace_read); 1: the environment
    products (two passes per site: slicing, GEMM and k-split reduction on the
    tensor cores, or one double-float GEMM launch); 2: the PCO tensor build
    (time and launches only)."""
    ms, fl, by = C.c_double(), C.c_double(), C.c_double()
    n = C.c_int64()
    _check(lib().gbsmps_trace_read_kernel(ctx, int(which), C.byref(ms), C.byref(n), C.byref(fl),
                                          C.byref(by)))
    return {"ms": ms.value, "launches": n.value, "flops": fl.value, "bytes": by.value}


class Context:
    """Owns a gbsmps context bound to a device and a CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        self.h = gbsmps_create(device, stream)

    def close(self):
        if self.h:
            gbsmps_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class MPS:
    """A device-resident MPS built by the library."""

    def __init__(self, h):
        self.h = h
        self.info = gbsmps_info(h)

    @classmethod
    def from_cov(cls, ctx: Context, gamma, **opts):
        return cls(gbsmps_build_from_cov(ctx.h, gamma, opts_default(**opts)))

    @classmethod
    def batch(cls, ctx: Context, gammas, opts_list):
        """Batched build; opts_list holds one keyword dict per state."""
        return [cls(h) for h in gbsmps_build_batch(ctx.h, gammas,
                                                    [opts_default(**o) for o in opts_list])]

    @classmethod
    def from_Q(cls, ctx: Context, Q, **opts):
        return cls(gbsmps_build_from_Q(ctx.h, Q, opts_default(**opts)))

    def tensor(self, site: int):
        return gbsmps_get_tensor(self.h, site)

    def tensors(self):
        return [self.tensor(m) for m in range(self.info["N"])]

    def amplitudes(self, patterns, out=None):
        return gbsmps_amplitudes(self.h, patterns, out)

    def sample(self, S, seed=0, counter0=0, uniforms=None, out=None, flags=None):
        return gbsmps_sample(self.h, S, seed, counter0, uniforms, out, flags)

    def offload(self):
        """Out-of-core sampling from here on; returns the bytes streamed per sampling."""
        return gbsmps_offload(self.h)

    def release(self):
        if self.h:
            gbsmps_release(self.h)
            self.h = None


def gbsmps_estimate_bytes(N: int, opts: Opts, samples: int) -> int:
    return int(lib().gbsmps_estimate_bytes(N, C.byref(opts), samples))


class Server:
    """Continuous-batching request loop of the library (gbsmps_server_*):
    requests (host Gamma, options, sample count) are admitted by free device
    memory into `slots` concurrent streams; results land in host arrays."""

    def __init__(self, device: int = 0, slots: int = 4, hbm_budget: int = 0,
                 simulate_s_per_tensor: float = 0.0, batch_max: int = 1):
        o = ServerOpts()
        _check(lib().gbsmps_server_opts_default(C.byref(o)))
        o.slots, o.hbm_budget, o.simulate_s_per_tensor = slots, hbm_budget, simulate_s_per_tensor
        o.batch_max = batch_max
        self.h = C.c_void_p()
        _check(lib().gbsmps_server_create(device, C.byref(o), C.byref(self.h)))
        self._keep = {}

    def submit(self, gamma, samples: int, seed: int = 0, counter0: int = 0, N: int | None = None,
               **opts) -> int:
        """Queue one request; returns its id.  gamma: host float64 (2N, 2N)
        numpy array or None (simulation mode, then N is required)."""
        if gamma is not None:
            gamma = np.ascontiguousarray(gamma, dtype=np.float64)
            N = gamma.shape[0] // 2
        out = np.zeros((samples, N), dtype=np.uint8)
        flags = np.zeros(samples, dtype=np.uint8)
        r = Request()
        r.gamma = gamma.ctypes.data if gamma is not None else None
        r.N, r.opts, r.samples, r.seed, r.counter0 = N, opts_default(**opts), samples, seed, counter0
        r.out = out.ctypes.data if samples else None
        r.flags = flags.ctypes.data if samples else None
        jid = C.c_int64()
        _check(lib().gbsmps_server_submit(self.h, C.byref(r), C.byref(jid)))
        self._keep[jid.value] = (gamma, out, flags)
        return jid.value

    def wait(self, jid: int, timeout_s: float = -1.0):
        """(samples, info dict) of request jid; raises on a failed job.  The
        info dict carries the job's boundary flags under "flags"."""
        info = JobInfo()
        rc = lib().gbsmps_server_wait(self.h, jid, timeout_s, C.byref(info))
        d = {k: getattr(info, k) for k, _ in JobInfo._fields_ if k != "detail"}
        d["detail"] = info.detail.decode(errors="replace")
        if rc != OK:
            raise GbsmpsError(rc, f"{lib().gbsmps_strerror(rc).decode()} ({d['detail']})")
        gamma, out, flags = self._keep.pop(jid)
        d["flags"] = flags
        return out, d

    def drain(self, timeout_s: float = -1.0):
        _check(lib().gbsmps_server_drain(self.h, timeout_s))

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().gbsmps_server_stats_read(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            _check(lib().gbsmps_server_destroy(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
