"""ctypes binding of libls (include/ls.h): the same entry points, argument marshalling only.

Every function here forwards to the C function of the same name; device buffers are torch CUDA
tensors (passed by data_ptr()), host buffers numpy arrays, and streams torch.cuda streams (the
current stream by default).  Negative return codes raise LSError with ls_last_error(); warnings
(LS_WARN_*) are returned.  Importing this module loads the in-tree library and fails loudly if
it has not been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LS_OK = 0
LS_WARN_UNDERFLOW = 1
LS_WARN_OVERFLOW = 2
LS_ERR_ARG = -1
LS_ERR_PARAM_MISMATCH = -2
LS_ERR_DIRECTION = -3
LS_ERR_LOCUS_MISMATCH = -4
LS_ERR_RANGE = -5
LS_ERR_CUDA = -6
LS_ERR_OOM = -7
LS_ERR_STATE = -8
LS_ERR_DEVICE = -9
LS_ERR_UNSUPPORTED = -10
LS_STATUS_UNDERFLOW = 1
LS_STATUS_OVERFLOW = 2
LS_STATUS_TIMEOUT = 4
LS_FWD = 0
LS_BWD = 1
LS_NOALLOC_MAX_N = 65536
LS_CKPT_F32 = 0
LS_PRIOR_FP32 = 0
LS_PRIOR_BF16 = 1
LS_CKPT_F16 = 1
LS_MLP_PARAMS = 68353

EXPORTED = [
    "ls_version", "ls_last_error", "ls_create", "ls_create_packed", "ls_destroy", "ls_info", "ls_query",
    "ls_export_packed", "ls_calc_rho", "ls_set_params", "ls_set_prior_format", "ls_table_create", "ls_table_destroy", "ls_table_copy",
    "ls_table_reset", "ls_table_info", "ls_table_read", "ls_forward", "ls_backward", "ls_posterior", "ls_distance",
    "ls_checkpoints", "ls_ckpt_info", "ls_ckpt_read", "ls_ckpt_replay", "ls_ckpt_destroy",
    "ls_run_all", "ls_run_all_noalloc", "ls_pac_grad", "ls_set_profiling", "ls_profile_read",
    "ls_posterior_rows", "ls_mlp_create", "ls_mlp_destroy", "ls_mlp_get", "ls_mlp_set", "ls_mlp_forward",
    "ls_mlp_grad", "ls_mlp_train", "ls_propose_window", "ls_propose_labels", "ls_propose", "ls_sparse_run_all",
]


class LSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libls error %d: %s" % (code, msg))
        self.code = code


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("libls is not built (%s missing); run __graft_entry__.build() first" % path)
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    sig = {
        "ls_version": ([], ctypes.c_char_p),
        "ls_last_error": ([], ctypes.c_char_p),
        "ls_create": ([P, P, I, I], I),
        "ls_create_packed": ([P, P, I, I, I], I),
        "ls_destroy": ([P], I),
        "ls_info": ([P, P, P, P, P], I),
        "ls_query": ([P, P, I, P, I, P], I),
        "ls_export_packed": ([P, P], I),
        "ls_calc_rho": ([P, I, D, D, P], I),
        "ls_set_params": ([P, P, P, I, P, P], I),
        "ls_set_prior_format": ([P, I], I),
        "ls_table_create": ([P, I, I, I, P], I),
        "ls_table_destroy": ([P], I),
        "ls_table_copy": ([P, P, P], I),
        "ls_table_reset": ([P], I),
        "ls_table_info": ([P, P, P, P, P, P], I),
        "ls_table_read": ([P, P, P, P], I),
        "ls_forward": ([P, P, I, P, I, P, P, P], I),
        "ls_backward": ([P, P, I, P, I, P, P, P], I),
        "ls_checkpoints": ([P, P, I, I, I, P, P, P], I),
        "ls_ckpt_info": ([P, P, P, P, P, P, P], I),
        "ls_ckpt_read": ([P, I, P, P, P], I),
        "ls_ckpt_replay": ([P, P, P, I, P, P], I),
        "ls_ckpt_destroy": ([P], I),
        "ls_posterior": ([P, P, P, P, P], I),
        "ls_distance": ([P, P, P, P, P], I),
        "ls_run_all": ([P, P, I, P, P, P, P], I),
        "ls_run_all_noalloc": ([P, P, I, P, P, P, P], I),
        "ls_pac_grad": ([P, I, I, P, I, P, P, P, P], I),
        "ls_posterior_rows": ([P, P, P, I, I, P, P], I),
        "ls_mlp_create": ([P, ctypes.c_uint64, P], I),
        "ls_mlp_destroy": ([P], I),
        "ls_mlp_get": ([P, P], I),
        "ls_mlp_set": ([P, P], I),
        "ls_mlp_forward": ([P, P, ctypes.c_int64, P, P], I),
        "ls_mlp_grad": ([P, P, P, I, P, P, P], I),
        "ls_mlp_train": ([P, P, P, ctypes.c_int64, I, I, ctypes.c_float, ctypes.c_uint64, P, P], I),
        "ls_propose_window": ([P, I, I, P, P, P], I),
        "ls_propose_labels": ([P, P, P, I, P, P], I),
        "ls_propose": ([P, I, I, P, P, P], I),
        "ls_sparse_run_all": ([P, P, I, I, I, I, P, I, P, ctypes.c_float, P, P, P, P, ctypes.c_float, P, P, P], I),
        "ls_set_profiling": ([P, I], I),
        "ls_profile_read": ([P, P, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()
LIBRARY_PATH = _build.LIB


def _check(rc):
    if rc < 0:
        raise LSError(rc, _lib.ls_last_error().decode())
    return rc


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype=None, name="tensor"):
    """device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    return ctypes.c_void_p(t.data_ptr())


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def ls_version():
    return _lib.ls_version().decode()


def ls_last_error():
    return _lib.ls_last_error().decode()


def ls_create(haps):
    """haps: host uint8 [L, N] 0/1.  Returns a context handle."""
    h, hp = _host(haps, np.uint8)
    L, N = h.shape
    out = ctypes.c_void_p()
    _check(_lib.ls_create(ctypes.byref(out), hp, N, L))
    return out


def ls_create_packed(packed, N, L, row_words):
    import torch
    out = ctypes.c_void_p()
    _check(_lib.ls_create_packed(ctypes.byref(out), _dev(packed, torch.int32, "packed"), N, L, row_words))
    return out


def ls_destroy(ctx):
    return _check(_lib.ls_destroy(ctx))


def ls_info(ctx):
    N, L, rw, nb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
    _check(_lib.ls_info(ctx, ctypes.byref(N), ctypes.byref(L), ctypes.byref(rw), ctypes.byref(nb)))
    return dict(N=N.value, L=L.value, row_words=rw.value, device_bytes=nb.value)


def ls_query(ctx, loci, haps):
    loci, lp = _host(loci, np.int32)
    haps, hp = _host(haps, np.int32)
    out = np.zeros((loci.size, haps.size), dtype=np.uint8)
    _check(_lib.ls_query(ctx, lp, loci.size, hp, haps.size, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def ls_export_packed(ctx):
    info = ls_info(ctx)
    out = np.zeros((info["L"], info["row_words"]), dtype=np.uint32)
    _check(_lib.ls_export_packed(ctx, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def ls_calc_rho(m, Ne=1.0, gamma=1.0):
    m, mp = _host(np.atleast_1d(m), np.float64)
    out = np.zeros_like(m)
    _check(_lib.ls_calc_rho(mp, m.size, float(Ne), float(gamma), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def ls_set_params(ctx, rho, mu, Pi=None):
    """rho host [L-1], mu scalar or [L]; Pi None (uniform) or a CUDA float32 [N, N] tensor."""
    import torch
    rho, rp = _host(np.atleast_1d(rho) if np.size(rho) else np.zeros(1), np.float64)
    mu, mp = _host(np.atleast_1d(mu), np.float64)
    h = ctypes.c_uint64()
    _check(_lib.ls_set_params(ctx, rp, mp, mu.size, _dev(Pi, torch.float32, "Pi"), ctypes.byref(h)))
    return h.value


def ls_set_prior_format(ctx, fmt):
    """LS_PRIOR_FP32 or LS_PRIOR_BF16 (applied by the next ls_set_params)."""
    return _check(_lib.ls_set_prior_format(ctx, int(fmt)))


def ls_table_create(ctx, kind, t_from, t_to):
    out = ctypes.c_void_p()
    _check(_lib.ls_table_create(ctx, kind, t_from, t_to, ctypes.byref(out)))
    return out


def ls_table_destroy(t):
    return _check(_lib.ls_table_destroy(t))


def ls_table_copy(dst, src, stream=None):
    return _check(_lib.ls_table_copy(dst, src, _stream(stream)))


def ls_table_reset(t):
    return _check(_lib.ls_table_reset(t))


def ls_table_info(t):
    k, l, a, b, h = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_uint64()
    _check(_lib.ls_table_info(t, ctypes.byref(k), ctypes.byref(l), ctypes.byref(a), ctypes.byref(b), ctypes.byref(h)))
    return dict(kind=k.value, locus=l.value, t_from=a.value, t_to=b.value, hash=h.value)


def ls_table_read(t, state=None, logscale=None, stream=None):
    import torch
    return _check(_lib.ls_table_read(t, _dev(state, torch.float32, "state"), _dev(logscale, torch.float64, "logscale"),
                                     _stream(stream)))


def _prop(fn, ctx, t, to_locus, store_loci, out, status, stream):
    import torch
    sl = np.ascontiguousarray(store_loci if store_loci is not None else np.zeros(0), dtype=np.int32)
    return _check(fn(ctx, t, int(to_locus), sl.ctypes.data_as(ctypes.c_void_p) if sl.size else None, sl.size,
                     _dev(out, torch.float32, "out"), _dev(status, torch.int32, "status"), _stream(stream)))


def ls_forward(ctx, fwd, to_locus, store_loci=None, alpha_out=None, status_out=None, stream=None):
    return _prop(_lib.ls_forward, ctx, fwd, to_locus, store_loci, alpha_out, status_out, stream)


def ls_backward(ctx, bck, to_locus, store_loci=None, beta_out=None, status_out=None, stream=None):
    return _prop(_lib.ls_backward, ctx, bck, to_locus, store_loci, beta_out, status_out, stream)


def ls_checkpoints(ctx, fwd, a, b, dtype=LS_CKPT_F32, status_out=None, stream=None):
    """snapshots of alpha at the recursive-bisection loci of [a, b]; returns the checkpoint handle."""
    import torch
    out = ctypes.c_void_p()
    _check(_lib.ls_checkpoints(ctx, fwd, int(a), int(b), int(dtype), ctypes.byref(out),
                               _dev(status_out, torch.int32, "status"), _stream(stream)))
    return out


def ls_ckpt_info(ck):
    n, dt, a, b, nb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
    _check(_lib.ls_ckpt_info(ck, ctypes.byref(n), None, None, None, None, None))
    loci = np.zeros(n.value, dtype=np.int32)
    _check(_lib.ls_ckpt_info(ck, ctypes.byref(n), loci.ctypes.data_as(ctypes.c_void_p), ctypes.byref(dt),
                             ctypes.byref(a), ctypes.byref(b), ctypes.byref(nb)))
    return dict(n=n.value, loci=loci, dtype=dt.value, t_from=a.value, t_to=b.value, device_bytes=nb.value)


def ls_ckpt_read(ck, k, alpha_out=None, logF_out=None, stream=None):
    import torch
    return _check(_lib.ls_ckpt_read(ck, int(k), _dev(alpha_out, torch.float32, "alpha_out"),
                                    _dev(logF_out, torch.float64, "logF_out"), _stream(stream)))


def ls_ckpt_replay(ctx, ck, fwd, locus, status_out=None, stream=None):
    import torch
    return _check(_lib.ls_ckpt_replay(ctx, ck, fwd, int(locus), _dev(status_out, torch.int32, "status"),
                                      _stream(stream)))


def ls_ckpt_destroy(ck):
    return _check(_lib.ls_ckpt_destroy(ck))


def ls_posterior(ctx, fwd, bck, p_out, stream=None):
    import torch
    return _check(_lib.ls_posterior(ctx, fwd, bck, _dev(p_out, torch.float32, "p_out"), _stream(stream)))


def ls_distance(ctx, fwd, bck, d_out, stream=None):
    import torch
    return _check(_lib.ls_distance(ctx, fwd, bck, _dev(d_out, torch.float32, "d_out"), _stream(stream)))


def ls_run_all(ctx, decode_loci, d_out, want_pac=True, status_out=None, stream=None):
    """d_out: CUDA float32 tensor or host float32 numpy array [D, N, N].  Returns (rc, pac)."""
    import torch
    dl = np.ascontiguousarray(decode_loci, dtype=np.int32)
    if isinstance(d_out, np.ndarray):
        if d_out.dtype != np.float32 or not d_out.flags["C_CONTIGUOUS"]:
            raise TypeError("host d_out must be a contiguous float32 array")
        dp = ctypes.c_void_p(d_out.ctypes.data)
    else:
        dp = _dev(d_out, torch.float32, "d_out")
    pac = ctypes.c_double(0.0)
    rc = _check(_lib.ls_run_all(ctx, dl.ctypes.data_as(ctypes.c_void_p) if dl.size else None, dl.size, dp,
                                ctypes.byref(pac) if want_pac else None, _dev(status_out, torch.int32, "status"),
                                _stream(stream)))
    return rc, (pac.value if want_pac else None)


def ls_run_all_noalloc(ctx, decode_loci, d_out, want_pac=True, status_out=None, stream=None):
    """The allocation-free pipeline: d_out must be a CUDA float32 tensor [D, N, N].  Returns (rc, pac)."""
    import torch
    dl = np.ascontiguousarray(decode_loci, dtype=np.int32)
    pac = ctypes.c_double(0.0)
    rc = _check(_lib.ls_run_all_noalloc(ctx, dl.ctypes.data_as(ctypes.c_void_p) if dl.size else None, dl.size,
                                        _dev(d_out, torch.float32, "d_out"), ctypes.byref(pac) if want_pac else None,
                                        _dev(status_out, torch.int32, "status"), _stream(stream)))
    return rc, (pac.value if want_pac else None)


def ls_pac_grad(ctx, interval_of, K, t_from=0, t_to=None, stream=None):
    """PAC log-likelihood of targets [t_from, t_to) and its gradient: returns
    (rc, pac, dlogmu, dlogrho [K] float64)."""
    io = np.ascontiguousarray(interval_of, dtype=np.int32)
    if t_to is None:
        t_to = ls_info(ctx)["N"]
    pac, gm = ctypes.c_double(), ctypes.c_double()
    gr = np.zeros(int(K), dtype=np.float64)
    rc = _check(_lib.ls_pac_grad(ctx, int(t_from), int(t_to), io.ctypes.data_as(ctypes.c_void_p) if io.size else None,
                                 int(K), ctypes.byref(pac), ctypes.byref(gm), gr.ctypes.data_as(ctypes.c_void_p),
                                 _stream(stream)))
    return rc, pac.value, gm.value, gr


def ls_posterior_rows(ctx, alpha, beta, t_from, p_out, stream=None):
    import torch
    T = alpha.shape[0]
    return _check(_lib.ls_posterior_rows(ctx, _dev(alpha, torch.float32, "alpha"), _dev(beta, torch.float32, "beta"),
                                         int(t_from), int(T), _dev(p_out, torch.float32, "p_out"), _stream(stream)))


def ls_mlp_create(params=None, seed=0):
    out = ctypes.c_void_p()
    pp = None
    if params is not None:
        params, pp = _host(params, np.float32)
        if params.size != LS_MLP_PARAMS:
            raise ValueError("need %d parameters" % LS_MLP_PARAMS)
    _check(_lib.ls_mlp_create(pp, ctypes.c_uint64(seed), ctypes.byref(out)))
    return out


def ls_mlp_destroy(m):
    return _check(_lib.ls_mlp_destroy(m))


def ls_mlp_get(m):
    out = np.zeros(LS_MLP_PARAMS, dtype=np.float32)
    _check(_lib.ls_mlp_get(m, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def ls_mlp_set(m, params):
    params, pp = _host(params, np.float32)
    return _check(_lib.ls_mlp_set(m, pp))


def ls_mlp_forward(m, X, scores, stream=None):
    import torch
    return _check(_lib.ls_mlp_forward(m, _dev(X, torch.float32, "X"), ctypes.c_int64(X.shape[0]),
                                      _dev(scores, torch.float32, "scores"), _stream(stream)))


def ls_mlp_grad(m, X, y, stream=None):
    """(grad [LS_MLP_PARAMS] float32, loss) of the half mean squared error at the current weights."""
    import torch
    g = np.zeros(LS_MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_double()
    _check(_lib.ls_mlp_grad(m, _dev(X, torch.float32, "X"), _dev(y, torch.float32, "y"), int(X.shape[0]),
                            g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss), _stream(stream)))
    return g, loss.value


def ls_mlp_train(m, X, y, steps, batch, lr, seed=0, stream=None):
    import torch
    loss = ctypes.c_double()
    _check(_lib.ls_mlp_train(m, _dev(X, torch.float32, "X"), _dev(y, torch.float32, "y"), ctypes.c_int64(X.shape[0]),
                             int(steps), int(batch), ctypes.c_float(lr), ctypes.c_uint64(seed), ctypes.byref(loss),
                             _stream(stream)))
    return loss.value


def ls_propose_window(ctx, C, w, cand_out, feat_out=None, stream=None):
    import torch
    return _check(_lib.ls_propose_window(ctx, int(C), int(w), _dev(cand_out, torch.int32, "cand_out"),
                                         _dev(feat_out, torch.float32, "feat_out"), _stream(stream)))


def ls_propose_labels(ctx, P, cand, C, y_out, stream=None):
    import torch
    return _check(_lib.ls_propose_labels(ctx, _dev(P, torch.float32, "P"), _dev(cand, torch.int32, "cand"), int(C),
                                         _dev(y_out, torch.float32, "y_out"), _stream(stream)))


def ls_propose(ctx, C, K, mlp, idx_out, stream=None):
    import torch
    return _check(_lib.ls_propose(ctx, int(C), int(K), mlp, _dev(idx_out, torch.int32, "idx_out"), _stream(stream)))


def ls_sparse_run_all(ctx, idx, K, WS, decode_loci, d_out, lost_tol=-1.0, lost_out=None, status_out=None,
                      lookahead=2, pool=True, d_trust=float("inf"), trust_out=None, pout_out=None, stream=None):
    """Returns (rc, pac of the restricted chains, number of dense-fallback targets).  trust_out: an
    int32 CUDA tensor [D, N, ceil(N/32)] receiving the trust bits (see include/ls.h)."""
    import torch
    dl = np.ascontiguousarray(decode_loci, dtype=np.int32)
    pac = ctypes.c_double()
    nf = ctypes.c_int32()
    rc = _check(_lib.ls_sparse_run_all(ctx, _dev(idx, torch.int32, "idx"), int(K), int(WS), int(lookahead), int(bool(pool)),
                                       dl.ctypes.data_as(ctypes.c_void_p), dl.size, _dev(d_out, torch.float32, "d_out"),
                                       ctypes.c_float(lost_tol), _dev(lost_out, torch.float32, "lost_out"),
                                       ctypes.byref(pac), _dev(status_out, torch.int32, "status_out"), ctypes.byref(nf),
                                       ctypes.c_float(d_trust), _dev(trust_out, torch.int32, "trust_out"),
                                       _dev(pout_out, torch.float32, "pout_out"), _stream(stream)))
    return rc, pac.value, nf.value


def trust_bits(mask, N):
    """Unpack trust_out words ([D, N, ceil(N/32)] int32 tensor) into a bool tensor [D, N, N]."""
    import torch
    m = mask.to(torch.int64) & 0xFFFFFFFF
    bits = (m.unsqueeze(-1) >> torch.arange(32, device=mask.device)) & 1
    return bits.reshape(mask.shape[0], mask.shape[1], -1)[:, :, :N].bool()


def ls_set_profiling(ctx, enable=True):
    return _check(_lib.ls_set_profiling(ctx, 1 if enable else 0))


def ls_profile_read(ctx):
    """(ms [4], launches [4]) of the last profiled ls_run_all: forward, backward, decode, symmetrise."""
    ms = (ctypes.c_float * 4)()
    n = (ctypes.c_int32 * 4)()
    _check(_lib.ls_profile_read(ctx, ms, n))
    return list(ms), list(n)
