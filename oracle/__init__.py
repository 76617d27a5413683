"""Plain FP64 CPU oracle for the Li & Stephens all-vs-all hot path (arXiv 2212.11403).

TEST INFRASTRUCTURE ONLY: the product library never imports, links or runs anything here.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` leg use it.

The arithmetic lives in ``ls_oracle.c`` (plain C, double precision, one routine per equation
of the paper, each citing its equation).  This module compiles it with gcc and marshals numpy
arrays through ctypes; it adds no arithmetic of the method except the closed forms used as
pins in the tests (which live in the tests, not here).

Array conventions (all host numpy):
  h     uint8 [L, N], variant-major 0/1 haplotypes (Sec. 3.2 "haplotypes in columns")
  rho   float64 [L-1], rho[l] between loci l and l+1 (0-based)
  mu    float64 scalar or [L]
  Pi    None (uniform 1/(N-1)) or float64 [N, N] recipient-major: Pi[i, j] = paper's Pi_ji
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ls_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libls_oracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_U32 = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile ls_oracle.c into a shared library (gcc, -O2, OpenMP, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.lso_calc_rho.argtypes = [_D, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D]
        lib.lso_pack_paper_layout.argtypes = [_U8, ctypes.c_int, ctypes.c_int, _U32]
        lib.lso_pack_paper_layout.restype = ctypes.c_long
        common = [_U8, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int, _D, ctypes.c_int]
        lib.lso_forward_target.argtypes = common + [_I, _D, _D]
        lib.lso_forward_target.restype = ctypes.c_double
        lib.lso_backward_target.argtypes = common + [_I, _D, _D]
        lib.lso_backward_target.restype = ctypes.c_double
        lib.lso_raw_forward_target.argtypes = common + [_D, _D]
        lib.lso_raw_backward_target.argtypes = common + [_D, _D]
        lib.lso_posterior.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, _D]
        lib.lso_distance_pair.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.lso_distance_pair.restype = ctypes.c_double
        lib.lso_distance_block.argtypes = [_D, _I, ctypes.c_int, ctypes.c_int, _D]
        lib.lso_run.argtypes = [_U8, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int, _D, _I, ctypes.c_int, _I,
                                ctypes.c_int, _D, _D, _D, _D, _D, _D, _D, ctypes.c_int]
        lib.lso_run.restype = ctypes.c_int
        lib.lso_run_rows.argtypes = lib.lso_run.argtypes
        lib.lso_run_rows.restype = ctypes.c_int
        lib.lso_grad_target.argtypes = common + [_I, _D, _D]
        lib.lso_grad_target.restype = ctypes.c_double
        lib.lso_pac_grad.argtypes = [_U8, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int, _D, _I, ctypes.c_int, _I,
                                     ctypes.c_int, _D, _D, _D, ctypes.c_int]
        _lib = lib
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


def _prep(h, rho, mu, Pi):
    h = np.ascontiguousarray(h, dtype=np.uint8)
    L, N = h.shape
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    if L > 1 and rho.size != L - 1:
        raise ValueError("rho must have L-1 entries")
    if rho.size == 0:
        rho = np.zeros(1)
    mu = np.ascontiguousarray(np.atleast_1d(mu), dtype=np.float64)
    if mu.size not in (1, L):
        raise ValueError("mu must be scalar or length L")
    if Pi is not None:
        Pi = np.ascontiguousarray(Pi, dtype=np.float64)
        if Pi.shape != (N, N):
            raise ValueError("Pi must be N x N")
    return h, L, N, rho, mu, Pi


def calc_rho(m, Ne=1.0, gamma=1.0):
    """Eq. rho: -expm1(-Ne * m**gamma), m in Morgans."""
    m = np.ascontiguousarray(m, dtype=np.float64).reshape(-1)
    out = np.empty_like(m)
    _get().lso_calc_rho(_p(m, _D), m.size, float(Ne), float(gamma), _p(out, _D))
    return out


def pack_paper_layout(h):
    """Paper's packed cache (Sec. 4.1.1): returns (bytes, words[L, stride_words])."""
    h = np.ascontiguousarray(h, dtype=np.uint8)
    L, N = h.shape
    nbytes = _get().lso_pack_paper_layout(_p(h, _U8), N, L, None)
    out = np.zeros(nbytes // 4, dtype=np.uint32)
    _get().lso_pack_paper_layout(_p(h, _U8), N, L, _p(out, _U32))
    return int(nbytes), out.reshape(L, -1)


def _slots(L, loci):
    slot = np.full(L, -1, dtype=np.int32)
    for k, l in enumerate(loci):
        slot[l] = k
    return slot


def forward_target(h, rho, mu, i, loci=(), Pi=None):
    """alpha at `loci` ([len(loci), N]), log F at those loci, and the final log F (Eq. fwd0/fwd1)."""
    h, L, N, rho, mu, Pi = _prep(h, rho, mu, Pi)
    loci = list(loci)
    slot = _slots(L, loci)
    A = np.zeros((max(len(loci), 1), N))
    lf = np.zeros(max(len(loci), 1))
    ll = _get().lso_forward_target(_p(h, _U8), N, L, _p(rho, _D), _p(mu, _D), mu.size, _p(Pi, _D), int(i),
                                   _p(slot, _I), _p(A, _D), _p(lf, _D))
    return A[: len(loci)], lf[: len(loci)], ll


def backward_target(h, rho, mu, i, loci=(), Pi=None):
    """beta at `loci`, log G at those loci, and the backward log-likelihood (Eq. bck0/bck1)."""
    h, L, N, rho, mu, Pi = _prep(h, rho, mu, Pi)
    loci = list(loci)
    slot = _slots(L, loci)
    B = np.zeros((max(len(loci), 1), N))
    lg = np.zeros(max(len(loci), 1))
    ll = _get().lso_backward_target(_p(h, _U8), N, L, _p(rho, _D), _p(mu, _D), mu.size, _p(Pi, _D), int(i),
                                    _p(slot, _I), _p(B, _D), _p(lg, _D))
    return B[: len(loci)], lg[: len(loci)], ll


def raw_forward_target(h, rho, mu, i, Pi=None):
    """Unscaled alpha~ [L, N] and F [L] (Eq. raw_forward, Eq. F).  Tiny L only."""
    h, L, N, rho, mu, Pi = _prep(h, rho, mu, Pi)
    A = np.zeros((L, N))
    F = np.zeros(L)
    _get().lso_raw_forward_target(_p(h, _U8), N, L, _p(rho, _D), _p(mu, _D), mu.size, _p(Pi, _D), int(i),
                                  _p(A, _D), _p(F, _D))
    return A, F


def raw_backward_target(h, rho, mu, i, Pi=None):
    """Unscaled beta~ [L, N] and G [L] (Eq. raw_backward, Eq. G).  Tiny L only."""
    h, L, N, rho, mu, Pi = _prep(h, rho, mu, Pi)
    B = np.zeros((L, N))
    G = np.zeros(L)
    _get().lso_raw_backward_target(_p(h, _U8), N, L, _p(rho, _D), _p(mu, _D), mu.size, _p(Pi, _D), int(i),
                                   _p(B, _D), _p(G, _D))
    return B, G


def run(h, rho, mu, loci, targets=None, Pi=None, nthreads=0, want=("post",), Pi_rows=None):
    """Forward + backward for `targets` (default: all), results at `loci`.

    The prior is Pi (recipient-major [N, N]), or Pi_rows ([nt, N]: row t = the prior row of
    recipient targets[t], for N too large for a host matrix), or neither (uniform).
    Returns a dict with the requested keys among alpha, beta, post ([nt, nl, N]), logF, logG
    ([nt, nl]), llf, llb ([nt]).
    """
    h, L, N, rho, mu, Pi = _prep(h, rho, mu, Pi)
    targets = np.arange(N, dtype=np.int32) if targets is None else np.ascontiguousarray(targets, dtype=np.int32)
    fn = _get().lso_run
    if Pi_rows is not None:
        if Pi is not None:
            raise ValueError("give Pi or Pi_rows, not both")
        Pi = np.ascontiguousarray(Pi_rows, dtype=np.float64)
        if Pi.shape != (targets.size, N):
            raise ValueError("Pi_rows must be [len(targets), N]")
        fn = _get().lso_run_rows
    loci = np.ascontiguousarray(loci, dtype=np.int32)
    nt, nl = targets.size, loci.size
    out = {}
    for key, shape in (("alpha", (nt, nl, N)), ("beta", (nt, nl, N)), ("post", (nt, nl, N)),
                       ("logF", (nt, nl)), ("logG", (nt, nl)), ("llf", (nt,)), ("llb", (nt,))):
        out[key] = np.zeros(shape) if (key in want) else None
    rc = fn(_p(h, _U8), N, L, _p(rho, _D), _p(mu, _D), mu.size, _p(Pi, _D), _p(targets, _I), nt,
                        _p(loci, _I), nl, _p(out["alpha"], _D), _p(out["beta"], _D), _p(out["post"], _D),
                        _p(out["logF"], _D), _p(out["logG"], _D), _p(out["llf"], _D), _p(out["llb"], _D),
                        int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the inputs")
    return {k: v for k, v in out.items() if v is not None}


def posterior(alpha, beta, i):
    """Eq. postprob for one recipient."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    p = np.zeros_like(alpha)
    _get().lso_posterior(_p(alpha, _D), _p(beta, _D), alpha.size, int(i), _p(p, _D))
    return p


def distance_pair(p_ji, p_ij):
    """Eq. distmat for one pair of posteriors."""
    return _get().lso_distance_pair(float(p_ji), float(p_ij))


def distance_block(post, targets):
    """Eq. distmat among `targets` at one locus; post [nt, N] = posteriors of those recipients."""
    post = np.ascontiguousarray(post, dtype=np.float64)
    targets = np.ascontiguousarray(targets, dtype=np.int32)
    nt, N = post.shape
    d = np.zeros((nt, nt))
    _get().lso_distance_block(_p(post, _D), _p(targets, _I), nt, N, _p(d, _D))
    return d


def grad_target(h, rho, mu, i, interval_of, K, Pi=None):
    """(log P_i, d/dlog mu, d/dlog rho_k [K]) by the Fisher identity, one recipient."""
    h, L, N, rho, mu, Pi = _prep(h, rho, mu, Pi)
    iv = np.ascontiguousarray(interval_of, dtype=np.int32)
    gm = np.zeros(1)
    gr = np.zeros(K)
    ll = _get().lso_grad_target(_p(h, _U8), N, L, _p(rho, _D), _p(mu, _D), mu.size, _p(Pi, _D), int(i),
                                _p(iv, _I), _p(gm, _D), _p(gr, _D))
    return ll, gm[0], gr


def pac_grad(h, rho, mu, interval_of, K, targets=None, Pi=None, nthreads=0):
    """PAC log-likelihood sum_i log P(h_i | h_-i) and its gradient w.r.t. log mu and the K log rho
    interval scales (Sec. 1 PAC; Fisher identity)."""
    h, L, N, rho, mu, Pi = _prep(h, rho, mu, Pi)
    targets = np.arange(N, dtype=np.int32) if targets is None else np.ascontiguousarray(targets, dtype=np.int32)
    iv = np.ascontiguousarray(interval_of, dtype=np.int32)
    pac = np.zeros(1)
    gm = np.zeros(1)
    gr = np.zeros(K)
    _get().lso_pac_grad(_p(h, _U8), N, L, _p(rho, _D), _p(mu, _D), mu.size, _p(Pi, _D), _p(targets, _I),
                        targets.size, _p(iv, _I), K, _p(pac, _D), _p(gm, _D), _p(gr, _D), int(nthreads))
    return pac[0], gm[0], gr
