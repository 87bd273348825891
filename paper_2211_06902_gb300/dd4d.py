"""Thin ctypes binding of libdd4d.so (C ABI in include/dd4d.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Fields may be numpy arrays (host; the library copies them in and
out) or CUDA torch tensors (device; used in place on the current stream).
Loading fails loudly when the library has not been built: there is no CPU
fallback.
"""

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdd4d.so")

DD_OK, DD_EINVAL, DD_ENOMEM, DD_ENOCONV, DD_ETIMEOUT, DD_ENAN, DD_ECUDA = range(7)
F64, F32, BF16 = 0, 1, 2
FULL, OMEGA, PHI, LAMBDA1 = 0, 1, 2, 3
SET_DPI, SET_B, SET_C, SET_OMEGA, SET_PHI, SET_LAMBDA1 = range(6)
PREC = {"f64": F64, "f32": F32, "bf16": BF16}
DOMAIN = {"full": FULL, "omega": OMEGA, "phi": PHI, "lambda1": LAMBDA1}


class GeomInfo(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("nblocks", "n_dpi", "n_B", "n_C", "n_E", "n_A",
                                        "n_lambda1", "max_omega", "max_phi")]


SOLVE_GRAPH, SOLVE_AUTOTUNE, SOLVE_NET_GUESS, SOLVE_PIPELINE = 1, 2, 4, 8
SOLVE_FGMRES, SOLVE_NET_PRECOND, SOLVE_GRAPH_LOOP, SOLVE_GRAPH_SOLVE = 16, 32, 64, 128


class SolveParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxiter", C.c_int), ("inner_prec", C.c_int),
                ("inner_tol", C.c_double), ("max_outer", C.c_int), ("check_every", C.c_int),
                ("flags", C.c_int), ("restart", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("systems", C.c_int), ("converged", C.c_int), ("max_iters", C.c_int),
                ("outer_cycles", C.c_int), ("max_relres", C.c_double), ("seconds", C.c_double),
                ("hop_variant", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HeatbathStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("matvecs", C.c_int), ("converged", C.c_int),
                ("max_relres", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MdStats(C.Structure):
    _fields_ = [("H0", C.c_double), ("H1", C.c_double), ("kinetic0", C.c_double), ("kinetic1", C.c_double),
                ("s_mb0", C.c_double), ("s_mb1", C.c_double), ("s_pf0", C.c_double), ("s_pf1", C.c_double),
                ("steps", C.c_int), ("force_evals", C.c_int), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("dd4d status %d: %s" % (status, msg))
        self.status = status


_lib = None


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libdd4d.so is not built (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
        sig = {
            "dd_create": [C.POINTER(vp), ip, C.c_int, C.c_double],
            "dd_destroy": [vp],
            "dd_strerror": [C.c_int],
            "dd_last_error": [vp],
            "dd_set_kappa": [vp, C.c_double],
            "dd_gauge_upload": [vp, vp],
            "dd_gauge_random": [vp, C.c_double, C.c_ulonglong],
            "dd_gauge_download": [vp, vp],
            "dd_set_geometry": [vp, ip, ip, ip, C.POINTER(GeomInfo)],
            "dd_geom_sites": [vp, C.c_int, C.c_int, ip, ip],
            "dd_geom_block": [vp, C.c_int, ip, ip, ip, ip],
            "dd_apply_D_block": [vp, C.c_int, ip, C.c_int, C.c_int, vp, vp, C.c_int, vp],
            "dd_solve_blocks": [vp, C.c_int, ip, C.c_int, C.c_int, vp, vp,
                                C.POINTER(SolveParams), C.POINTER(SolveStats), vp],
            "dd_apply_w": [vp, C.c_int, vp, vp, C.POINTER(SolveParams), vp],
            "dd_multiboson_action": [vp, C.c_int, dp, vp, dp, dp, dp, C.POINTER(SolveParams), vp],
            "dd_roots": [C.c_int, C.c_double, dp],
            "dd_timing_enable": [vp, C.c_int],
            "dd_timing_get": [vp, C.c_int, dp, C.POINTER(C.c_longlong), dp],
            "dd_launch_count": [C.POINTER(C.c_longlong)],
            "dd_logdet_check": [vp, C.POINTER(SolveParams), dp, dp, C.POINTER(LogdetReport), vp],
            "dd_last_solve_stats": [vp, C.POINTER(SolveStats)],
            "dd_net_create": [vp, C.c_int, ip, dp, C.POINTER(vp)],
            "dd_net_destroy": [vp],
            "dd_net_weights": [vp, dp],
            "dd_net_apply": [vp, vp, ip, C.c_int, C.c_int, vp, vp, vp],
            "dd_net_loss_grad": [vp, vp, ip, C.c_int, C.c_int, vp, vp, dp, dp, vp],
            "dd_net_train": [vp, vp, ip, C.c_int, C.c_int, vp, C.POINTER(TrainParams),
                             C.POINTER(TrainStats), vp],
            "dd_set_net": [vp, vp],
            "dd_set_hop_variant": [vp, C.c_int, C.c_int],
            "dd_hop_variants": [C.c_int],
            "dd_multiboson_heatbath": [vp, C.c_int, dp, vp, vp, C.c_double, C.c_int,
                                       C.POINTER(SolveParams), C.POINTER(HeatbathStats), vp],
            "dd_net_save": [vp, C.c_char_p],
            "dd_net_load": [vp, C.c_char_p, C.POINTER(vp)],
            "dd_hop_variant_name": [C.c_int, C.c_int],
            "dd_apply_D_block_noalloc": [vp, C.c_int, ip, C.c_int, C.c_int, vp, vp, vp],
            "dd_reweight_samples": [vp, C.c_int, C.c_double, C.c_int, vp, dp, vp,
                                    C.POINTER(SolveParams), vp],
            "dd_mb_force": [vp, C.c_int, dp, vp, vp, C.POINTER(SolveParams), vp],
            "dd_set_clover": [vp, C.c_double],
            "dd_debug_wait_fault": [vp, C.c_int],
            "dd_logdet_force": [vp, C.c_int, vp, vp, C.POINTER(SolveParams), vp],
            "dd_fp64_fma_rate": [dp],
            "dd_apply_w_part": [vp, C.c_int, C.c_int, ip, C.c_int, vp, vp, C.POINTER(SolveParams), vp],
            "dd_net_tensor_cores": [vp, C.c_int],
            "dd_pf_heatbath": [vp, vp, vp, vp],
            "dd_clover_cond": [vp, dp],
            "dd_md_trajectory": [vp, C.c_int, dp, vp, vp, vp, C.c_double, C.c_int, C.POINTER(SolveParams),
                                 C.POINTER(MdStats), vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = (C.c_char_p if name in ("dd_strerror", "dd_last_error", "dd_hop_variant_name")
                         else C.c_int)
        _lib = L
    return _lib


def exported_symbols():
    """Names of the C ABI entry points the binding expects."""
    return ["dd_create", "dd_destroy", "dd_strerror", "dd_last_error", "dd_set_kappa",
            "dd_gauge_upload", "dd_gauge_random", "dd_gauge_download", "dd_set_geometry", "dd_geom_sites", "dd_geom_block",
            "dd_apply_D_block", "dd_solve_blocks", "dd_apply_w", "dd_multiboson_action",
            "dd_roots", "dd_timing_enable", "dd_timing_get", "dd_launch_count", "dd_logdet_check",
            "dd_last_solve_stats", "dd_net_create", "dd_net_destroy", "dd_net_weights",
            "dd_net_apply", "dd_net_loss_grad", "dd_net_train", "dd_set_net", "dd_net_save", "dd_net_load", "dd_multiboson_heatbath",
            "dd_set_hop_variant", "dd_hop_variants", "dd_hop_variant_name",
            "dd_apply_D_block_noalloc", "dd_reweight_samples", "dd_mb_force", "dd_set_clover",
            "dd_debug_wait_fault", "dd_logdet_force", "dd_fp64_fma_rate", "dd_apply_w_part",
            "dd_net_tensor_cores", "dd_pf_heatbath", "dd_md_trajectory", "dd_clover_cond"]


def hop_variant_name(prec, v):
    """Description of stencil launch variant v at precision prec (None if out of range)."""
    r = lib().dd_hop_variant_name(PREC[prec] if isinstance(prec, str) else prec, v)
    return r.decode() if r else None


def _ptr(x):
    """Device or host address of a torch tensor / numpy array."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(x.ctypes.data)


def _stream(stream):
    """A CUDA stream handle: an int, a torch stream (its handle), or None for
    torch's current stream (the legacy default stream without torch)."""
    if stream is not None:
        return C.c_void_p(getattr(stream, "cuda_stream", stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return C.c_void_p(0)


def params(tol=1e-10, maxiter=2000, inner_prec="f64", inner_tol=3e-6, max_outer=None,
           check_every=8, graph=False, autotune=False, net_guess=False, pipeline=False,
           fgmres=False, restart=8, net_precond=False, graph_loop=False, graph_solve=False):
    ip = PREC[inner_prec] if isinstance(inner_prec, str) else inner_prec
    if max_outer is None:
        max_outer = 4 if ip == F64 else 30
    flags = ((SOLVE_GRAPH if graph else 0) | (SOLVE_AUTOTUNE if autotune else 0)
             | (SOLVE_NET_GUESS if net_guess else 0) | (SOLVE_PIPELINE if pipeline else 0)
             | (SOLVE_FGMRES if fgmres else 0) | (SOLVE_NET_PRECOND if net_precond else 0)
             | (SOLVE_GRAPH_LOOP if graph_loop else 0) | (SOLVE_GRAPH_SOLVE if graph_solve else 0))
    return SolveParams(tol, maxiter, ip, inner_tol, max_outer, check_every, flags, restart)


def roots(N, c):
    """u_k, k = 1..N/2 (complex numpy array)."""
    out = np.zeros(N, dtype=np.float64)
    st = lib().dd_roots(N, c, out.ctypes.data_as(C.POINTER(C.c_double)))
    if st:
        raise DDError(st, lib().dd_strerror(st).decode())
    return out[0::2] + 1j * out[1::2]


def fp64_fma_rate():
    """Measured FP64 FMA rate of the current device (TFLOP/s)."""
    t = C.c_double(0)
    st = lib().dd_fp64_fma_rate(C.byref(t))
    if st:
        raise DDError(st, "dd_fp64_fma_rate failed")
    return t.value


def launch_count():
    """Kernel launches issued by the library so far in this process."""
    n = C.c_longlong(0)
    lib().dd_launch_count(C.byref(n))
    return n.value


class LogdetReport(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("logabs_D", "logabs_W1", "logabs_Lambda1",
                                           "logabs_Omega", "logabs_Phi", "phase_D",
                                           "phase_rhs", "residual")] + \
               [(n, C.c_int) for n in ("dim_D", "dim_W1", "dim_Lambda1")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TrainParams(C.Structure):
    _fields_ = [("steps", C.c_int), ("lr", C.c_double), ("solve_tol", C.c_double)]


class TrainStats(C.Structure):
    _fields_ = [("loss_first", C.c_double), ("loss_last", C.c_double), ("steps", C.c_int),
                ("pairs", C.c_int), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Context:
    """A lattice, its gauge field and its domain decomposition on the GPU."""

    def __init__(self, L, kappa, time_bc=-1):
        self.L = tuple(int(v) for v in L)
        self._h = C.c_void_p()
        Larr = (C.c_int * 4)(*self.L)
        st = lib().dd_create(C.byref(self._h), Larr, int(time_bc), float(kappa))
        if st:
            raise DDError(st, lib().dd_strerror(st).decode())
        self.info = None

    def close(self):
        if self._h:
            lib().dd_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st and st != DD_ENOCONV:
            raise DDError(st, lib().dd_last_error(self._h).decode())
        return st

    def set_kappa(self, kappa):
        self._check(lib().dd_set_kappa(self._h, float(kappa)))

    def set_clover(self, csw):
        """Clover term c_sw (0 = off): A(x) = 1 + i kappa c_sw sum sigma F in D."""
        self._check(lib().dd_set_clover(self._h, float(csw)))

    def clover_cond(self):
        """The bound c_A >= cond_2(A) the solves divide their tolerance by (1 without the term)."""
        v = C.c_double(0)
        self._check(lib().dd_clover_cond(self._h, C.byref(v)))
        return v.value

    def gauge_upload(self, U):
        U = np.ascontiguousarray(U, dtype=np.complex128)
        if U.shape != self.L + (4, 3, 3):
            raise ValueError("gauge field shape must be L + (4, 3, 3)")
        self._check(lib().dd_gauge_upload(self._h, C.c_void_p(U.ctypes.data)))

    def gauge_random(self, eps, seed):
        """Synthetic links exp(i eps H) drawn on the device from the (seed, gauge) stream."""
        self._check(lib().dd_gauge_random(self._h, float(eps), int(seed) & 0xFFFFFFFFFFFFFFFF))

    def gauge_download(self):
        """The current links, layout L + (4, 3, 3) complex128 (time-boundary sign not applied)."""
        U = np.empty(self.L + (4, 3, 3), dtype=np.complex128)
        self._check(lib().dd_gauge_download(self._h, C.c_void_p(U.ctypes.data)))
        return U

    def set_geometry(self, cores):
        nc = (C.c_int * 4)(*[len(c) for c in cores])
        lo = [iv[0] for c in cores for iv in c]
        hi = [iv[1] for c in cores for iv in c]
        info = GeomInfo()
        self._check(lib().dd_set_geometry(self._h, nc, (C.c_int * len(lo))(*lo),
                                          (C.c_int * len(hi))(*hi), C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in info._fields_}
        return self.info

    def geom_sites(self, which, block=0):
        n = C.c_int(0)
        self._check(lib().dd_geom_sites(self._h, which, block, None, C.byref(n)))
        out = np.zeros(n.value, dtype=np.int32)
        self._check(lib().dd_geom_sites(self._h, which, block,
                                        out.ctypes.data_as(C.POINTER(C.c_int)), C.byref(n)))
        return out

    def geom_block(self, b):
        arrs = [(C.c_int * 4)() for _ in range(4)]
        self._check(lib().dd_geom_block(self._h, b, *arrs))
        return dict(zip(("origin", "side", "core_lo", "core_hi"), [list(a) for a in arrs]))

    def apply_D_block(self, kind, ids, nrhs, inp, out, prec="f64", stream=None):
        kind = DOMAIN[kind] if isinstance(kind, str) else kind
        ids = list(ids) if ids is not None else [0]
        idarr = (C.c_int * len(ids))(*ids)
        p = PREC[prec] if isinstance(prec, str) else prec
        self._check(lib().dd_apply_D_block(self._h, kind, idarr, len(ids), nrhs, _ptr(inp),
                                           _ptr(out), p, _stream(stream)))

    def apply_D_block_noalloc(self, kind, ids, nrhs, inp, out, stream=None):
        """FP64 D_X without device allocation (device tensors only)."""
        kind = DOMAIN[kind] if isinstance(kind, str) else kind
        ids = list(ids) if ids is not None else [0]
        idarr = (C.c_int * len(ids))(*ids)
        self._check(lib().dd_apply_D_block_noalloc(self._h, kind, idarr, len(ids), nrhs,
                                                   _ptr(inp), _ptr(out), _stream(stream)))

    def solve_blocks(self, kind, ids, nrhs, b, x, prm=None, stream=None):
        kind = DOMAIN[kind] if isinstance(kind, str) else kind
        ids = list(ids) if ids is not None else [0]
        idarr = (C.c_int * len(ids))(*ids)
        prm = prm or params()
        stats = SolveStats()
        st = self._check(lib().dd_solve_blocks(self._h, kind, idarr, len(ids), nrhs, _ptr(b),
                                               _ptr(x), C.byref(prm), C.byref(stats),
                                               _stream(stream)))
        d = stats.as_dict()
        d["status"] = st
        return d

    def apply_w(self, n_f, chi, w_chi, prm=None, stream=None):
        prm = prm or params()
        st = self._check(lib().dd_apply_w(self._h, n_f, _ptr(chi), _ptr(w_chi), C.byref(prm),
                                          _stream(stream)))
        return st

    W_PARTS = {"frame_q": 0, "blocks": 1, "frame": 2}

    def apply_w_part(self, part, n_f, ids, inp, out, prm=None, stream=None):
        """One stage of w for the blocks ids (None for the frame stage): see dd_apply_w_part."""
        ids = list(ids) if ids is not None else [0]
        idarr = (C.c_int * len(ids))(*ids)
        p = self.W_PARTS[part] if isinstance(part, str) else part
        return self._check(lib().dd_apply_w_part(self._h, p, n_f, idarr, len(ids), _ptr(inp), _ptr(out),
                                                 C.byref(prm or params()), _stream(stream)))

    def multiboson_heatbath(self, u, eta, chi, tol=1e-10, maxiter=200, prm=None, stream=None):
        """chi_k = W_{u_k}^{-1} eta_k for the fields of eta (layout of apply_w); stats dict."""
        u = np.asarray(u, dtype=np.complex128)
        uu = np.empty(2 * len(u))
        uu[0::2], uu[1::2] = u.real, u.imag
        prm = prm or params()
        st = HeatbathStats()
        s = self._check(lib().dd_multiboson_heatbath(
            self._h, len(u), uu.ctypes.data_as(C.POINTER(C.c_double)), _ptr(eta), _ptr(chi),
            float(tol), int(maxiter), C.byref(prm), C.byref(st), _stream(stream)))
        d = st.as_dict()
        d["status"] = s
        return d

    def mb_force(self, u, chi, F=None, prm=None, stream=None):
        """Force of the multi-boson action on the active links: F[x0,x1,x2,x3,mu,t] =
        dS/d eps at U_mu(x) -> exp(i eps lambda_t/2) U_mu(x), zero off the active links.
        chi: layout of apply_w.  F: optional device tensor of V*4*8 doubles.
        Returns (F, status); F is a numpy array unless a tensor was given."""
        u = np.asarray(u, dtype=np.complex128)
        uu = np.empty(2 * len(u))
        uu[0::2], uu[1::2] = u.real, u.imag
        out = F if F is not None else np.zeros(self.L + (4, 8))
        st = self._check(lib().dd_mb_force(
            self._h, len(u), uu.ctypes.data_as(C.POINTER(C.c_double)), _ptr(chi), _ptr(out),
            C.byref(prm or params()), _stream(stream)))
        return out, st

    def logdet_force(self, n_noise, eta, G=None, prm=None, stream=None):
        """Noise estimate of d ln|det D_Omega0^a| / d eps on the active links:
        G[x0,x1,x2,x3,mu,t], zero off the active links.  eta: n_noise noise vectors
        per framed block in the layout of solve_blocks on all blocks.  G: optional
        device tensor of V*4*8 doubles.  Returns (G, status)."""
        out = G if G is not None else np.zeros(self.L + (4, 8))
        st = self._check(lib().dd_logdet_force(self._h, n_noise, _ptr(eta), _ptr(out),
                                               C.byref(prm or params()), _stream(stream)))
        return out, st

    def pf_heatbath(self, eta, phi, stream=None):
        """phi_a = D_Omega0^a^dag eta_a for every block (layout of solve_blocks on all
        blocks with one rhs), so that the pseudofermion action equals |eta|^2."""
        self._check(lib().dd_pf_heatbath(self._h, _ptr(eta), _ptr(phi), _stream(stream)))

    def md_trajectory(self, u, chi, phi, P, tau, nsteps, prm=None, stream=None):
        """Leapfrog trajectory of the active links (links updated in place): u, chi the
        multi-boson roots and fields (layout of apply_w; None for none), phi the block
        pseudofermions (layout of pf_heatbath; None for none), P the momenta
        [x0,x1,x2,x3,mu,t] (V*4*8 doubles, in and out).  Returns the stats dict."""
        n_f = 0
        uptr = None
        if u is not None and len(u):
            u = np.asarray(u, dtype=np.complex128)
            uu = np.empty(2 * len(u))
            uu[0::2], uu[1::2] = u.real, u.imag
            n_f = len(u)
            uptr = uu.ctypes.data_as(C.POINTER(C.c_double))
        st = MdStats()
        s = self._check(lib().dd_md_trajectory(
            self._h, n_f, uptr, None if chi is None or n_f == 0 else _ptr(chi),
            None if phi is None else _ptr(phi), _ptr(P), float(tau), int(nsteps),
            C.byref(prm or params()), C.byref(st), _stream(stream)))
        d = st.as_dict()
        d["status"] = s
        return d

    def reweight_samples(self, N, c, eta, r_eta=None, prm=None, stream=None):
        """Samples s = |eta|^2 - |M eta|^2, M = 1 - R_{N+1}(W_1), one per source of eta
        (layout of apply_w); mean(exp(s)) estimates |W_N|^-2 (Eq. rw).  Returns
        (s, status); r_eta, if given, receives R_{N+1}(W_1) eta."""
        n_src = int(eta.shape[0])
        out = np.zeros(n_src)
        st = self._check(lib().dd_reweight_samples(
            self._h, int(N), float(c), n_src, _ptr(eta), out.ctypes.data_as(C.POINTER(C.c_double)),
            None if r_eta is None else _ptr(r_eta), C.byref(prm or params()), _stream(stream)))
        return out, st

    def multiboson_action(self, u, chi, prm=None, stream=None):
        u = np.asarray(u, dtype=np.complex128)
        n_f = len(u)
        uu = np.empty(2 * n_f)
        uu[0::2], uu[1::2] = u.real, u.imag
        S = C.c_double(0)
        Sr = C.c_double(0)
        nb = self.info["nblocks"]
        Sb = np.zeros(nb)
        prm = prm or params()
        st = self._check(lib().dd_multiboson_action(
            self._h, n_f, uu.ctypes.data_as(C.POINTER(C.c_double)), _ptr(chi), C.byref(S),
            Sb.ctypes.data_as(C.POINTER(C.c_double)), C.byref(Sr), C.byref(prm),
            _stream(stream)))
        return S.value, Sb, Sr.value, st

    def logdet_check(self, prm=None, stream=None):
        """Dense check of Eq. (detD): report dict plus per-block ln|det| arrays."""
        prm = prm or params(1e-12)
        nb = self.info["nblocks"]
        lo, lp = np.zeros(nb), np.zeros(nb)
        rep = LogdetReport()
        self._check(lib().dd_logdet_check(self._h, C.byref(prm),
                                          lo.ctypes.data_as(C.POINTER(C.c_double)),
                                          lp.ctypes.data_as(C.POINTER(C.c_double)),
                                          C.byref(rep), _stream(stream)))
        d = rep.as_dict()
        d["logabs_omega"] = lo
        d["logabs_phi"] = lp
        return d

    def set_hop_variant(self, prec, v):
        p = PREC[prec] if isinstance(prec, str) else prec
        self._check(lib().dd_set_hop_variant(self._h, p, v))

    def debug_wait_fault(self, on):
        """Test hook: the bundle-form stencil's bounded wait gives up (DD_ETIMEOUT)."""
        self._check(lib().dd_debug_wait_fault(self._h, 1 if on else 0))

    def last_solve_stats(self):
        st = SolveStats()
        self._check(lib().dd_last_solve_stats(self._h, C.byref(st)))
        return st.as_dict()

    def timing_enable(self, on=True):
        self._check(lib().dd_timing_enable(self._h, 1 if on else 0))

    def timing_get(self, which):
        ms = C.c_double(0)
        n = C.c_longlong(0)
        by = C.c_double(0)
        self._check(lib().dd_timing_get(self._h, which, C.byref(ms), C.byref(n), C.byref(by)))
        return ms.value, n.value, by.value


NET_CHANNELS = (4, 16, 16, 16, 4)


class Net:
    """The gauge-covariant parallel-transport convolution network on a context."""

    def __init__(self, ctx, weights, channels=NET_CHANNELS):
        self.ctx = ctx
        self.channels = tuple(channels)
        w = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.complex128).ravel()
                                                 for x in weights]))
        self.shapes = [np.asarray(x).shape for x in weights]
        self._h = C.c_void_p()
        ch = (C.c_int * len(channels))(*channels)
        ctx._check(lib().dd_net_create(ctx._h, len(channels) - 1, ch,
                                       w.view(np.float64).ctypes.data_as(C.POINTER(C.c_double)),
                                       C.byref(self._h)))

    def close(self):
        if self._h:
            lib().dd_net_destroy(self._h)
            self._h = C.c_void_p()

    def save(self, path):
        """Channels, FP32 master weights and Adam state to `path`."""
        st = lib().dd_net_save(self._h, os.fsencode(path))
        if st:
            raise DDError(st, "cannot write network file %s" % path)

    @classmethod
    def load(cls, ctx, path):
        """A network read from `path` (written by save) on ctx's device."""
        self = cls.__new__(cls)
        self.ctx = ctx
        self._h = C.c_void_p()
        ctx._check(lib().dd_net_load(ctx._h, os.fsencode(path), C.byref(self._h)))
        with open(path, "rb") as f:
            head = f.read(12)
            nl = int(np.frombuffer(head[8:12], dtype=np.int32)[0])
            ch = np.frombuffer(f.read(4 * (nl + 1)), dtype=np.int32)
        self.channels = tuple(int(c) for c in ch)
        self.shapes = [(9, self.channels[l + 1], self.channels[l]) for l in range(nl)]
        return self

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _split(self, flat):
        out, k = [], 0
        for s in self.shapes:
            n = int(np.prod(s))
            out.append(flat[k:k + n].reshape(s))
            k += n
        return out

    def weights(self):
        n = sum(int(np.prod(s)) for s in self.shapes)
        w = np.zeros(2 * n)
        lib().dd_net_weights(self._h, w.ctypes.data_as(C.POINTER(C.c_double)))
        return self._split(w.view(np.complex128))

    def tensor_cores(self, on=True):
        """Layers on the tensor cores (BF16 operands, the default) or the FP32 CUDA cores."""
        st = lib().dd_net_tensor_cores(self._h, 1 if on else 0)
        if st:
            raise DDError(st, "dd_net_tensor_cores failed")

    def apply(self, ids, nrhs, inp, out, stream=None):
        idarr = (C.c_int * len(ids))(*ids)
        self.ctx._check(lib().dd_net_apply(self.ctx._h, self._h, idarr, len(ids), nrhs, _ptr(inp),
                                           _ptr(out), _stream(stream)))

    def loss_grad(self, ids, nrhs, b, x, stream=None):
        idarr = (C.c_int * len(ids))(*ids)
        n = sum(int(np.prod(s)) for s in self.shapes)
        g = np.zeros(2 * n)
        L = C.c_double(0)
        self.ctx._check(lib().dd_net_loss_grad(self.ctx._h, self._h, idarr, len(ids), nrhs, _ptr(b),
                                               _ptr(x), C.byref(L),
                                               g.ctypes.data_as(C.POINTER(C.c_double)),
                                               _stream(stream)))
        return L.value, self._split(g.view(np.complex128))

    def train(self, ids, nrhs, b, steps=100, lr=2e-3, solve_tol=1e-10, stream=None, ctx=None):
        """Train on the framed blocks `ids` of `ctx` (default: the creating context)."""
        ctx = ctx or self.ctx
        idarr = (C.c_int * len(ids))(*ids)
        tp = TrainParams(steps, lr, solve_tol)
        ts = TrainStats()
        ctx._check(lib().dd_net_train(ctx._h, self._h, idarr, len(ids), nrhs, _ptr(b),
                                      C.byref(tp), C.byref(ts), _stream(stream)))
        return ts.as_dict()

    def attach(self, ctx=None):
        """Use this network for DD_SOLVE_NET_GUESS solves on `ctx` (default: its own)."""
        ctx = ctx or self.ctx
        ctx._check(lib().dd_set_net(ctx._h, self._h))

    def detach(self, ctx=None):
        ctx = ctx or self.ctx
        ctx._check(lib().dd_set_net(ctx._h, None))
